// Launch-side declarations of the resultant stage kernels.
#pragma once
#include "common.cuh"

namespace bs {

constexpr int kUniTile = 128;     // default threads of a univariate-resultant block
constexpr int kUniMaxThreads = 256;  // largest univariate-resultant block
constexpr int kEvalThreads = 256; // threads of a transform block
// warps of an independent-warp evaluation block; five such blocks fit an SM at 56 registers,
// so 35 warps per SM take the 80 x 65 rows of a degree-32 discriminant in one wave
constexpr int kEvalIwWarps = 7;
constexpr int kEvalIwBlocksPerSm = 5;
constexpr int kCrtWarps = 8;      // warps of a reconstruction block
constexpr int kCrtTile = 8;       // coefficients per reconstruction block
constexpr int kCrtInvSmem = 160;  // prime counts whose inverse table is staged in smem
constexpr int kCrtWarpMaxK = 160; // prime counts handled by the warp-per-coefficient kernel
constexpr int kPlanThreads = 512; // threads of the device plan block (two halves)
constexpr int kWarpLogNMax = 10;  // transforms up to 2^10 points run one per warp
// device-plan offset slots (pairs [start, end) of each stage's work list)
constexpr int kOffEvalW = 0, kOffEvalS = 2, kOffUni = 4, kOffInttW = 6, kOffInttS = 8,
              kOffCrt = 10, kNumOffs = 12;
constexpr int kInttWarps = 4;     // warps (primes) of a warp-interpolation block
constexpr int kWarpInttLogNMax = 9;  // interpolations up to 2^9 points run one per warp
constexpr int kInttSmemWords = 3;  // words per point of an interpolation block: values, twiddles, coset powers
// size classes of the warp evaluation kernels: N <= 32, 64, 128, 256, 512, 1024
constexpr int kNumEvalClasses = 6;
inline int eval_class_of(int logN) { return logN <= 5 ? 0 : logN - 5; }

// launchers (defined next to the kernels)
int uni_occupancy(int cls, int threads);
void launch_uni(int cls, int grid, int threads, cudaStream_t s, const Job* jobs, WorkList wl, Tables T);
void launch_uni_direct(int cls, int n, cudaStream_t s, const int32_t* idx, const uint32_t* a, int da,
                       int lda, const uint32_t* b, int db, int ldb, uint32_t* res, Tables T);
// transforms of N > 2^kWarpLogNMax points: blocks of `warps` = max N / 1024 warps
constexpr int kEvalBigMaxWarps = 16;
void launch_eval(int grid, int warps, cudaStream_t s, const Job* jobs, WorkList wl, Tables T);
void launch_intt(int grid, size_t smem, cudaStream_t s, const Job* jobs, WorkList wl, Tables T);
// one warp per (job, prime) for N <= 2^kWarpInttLogNMax
void launch_intt_w(int grid, cudaStream_t s, const Job* jobs, WorkList wl, Tables T);
// tile: coefficients per block (one warp each), 1 <= tile <= kCrtTile
void launch_crt_w(int grid, int tile, size_t smem, cudaStream_t s, const Job* jobs, WorkList wl,
                  Tables T, int kmax, int lmax);
// sizes for the L2 prefetch the evaluation kernel issues (kt < 0: read the first job's plan)
struct PfHint {
  int kt, N, kn;
};
constexpr int kPfIssuers = 128;   // blocks that issue one prefetch chunk each
// cls = eval_class_of(logN) for lists of one size class, -1 for any size (device plans)
// warps: rows per block (1 .. kEvalThreads / 32); the work list counts groups of that many rows
void launch_eval_w(int cls, int grid, int warps, cudaStream_t s, const Job* jobs, WorkList wl,
                   Tables T, PfHint pf);
// independent-warp evaluation: the work list counts single rows (eval_rows_per_item = 1)
void launch_eval_iw(int cls, int grid, cudaStream_t s, const Job* jobs, WorkList wl, Tables T, PfHint pf);
void launch_crt(int grid, int threads, size_t smem, cudaStream_t s, const Job* jobs, WorkList wl,
                Tables T, int kmax, int lmax, int staged, int skip_big = 0);
// eval_group: rows per item of the warp-evaluation work list (8 for k_eval_w blocks of
// eight warps, 1 for the independent-warp kernel)
void launch_plan_single(cudaStream_t s, const Job& J, Job* dst, int64_t* offs, Tables T, int eval_group);
int set_stage_smem_limits(int optin);
// launches of the stage kernels from the calling thread use programmatic dependent launch
// while on (each stage kernel waits for its predecessor before reading its results)
void set_launch_pdl(bool on);
// raise a kernel's dynamic shared memory limit to what the opt-in size leaves next to its
// static shared memory
int set_dyn_smem_limit(const void* func, int optin);

// weighted-sum reconstruction of many primes (k_need > kCrtWarpMaxK, host batches)
constexpr int kBigTabThreads = 128;  // primes per table block
constexpr int kBigGI = 32, kBigGL = 64, kBigGJ = 32;  // contraction tile: coefficients, limbs, primes
constexpr int kBigCarryWarps = 8;    // coefficients per carry block
// limbs of M_j = P / p_j for k primes (P < 2^(31 k))
inline int big_ws_len(int k) { return (31 * k + 31) / 32 + 1; }
void launch_bigcrt(int g_tab, int g_gemm, int g_carry, cudaStream_t s, const Job* jobs, WorkList tab,
                   WorkList gemm, WorkList carry, Tables T);

// degree classes of the univariate stage: max(m_e, n_e) + 1 <= class length
constexpr int kUniClasses[] = {8, 16, 24, 33, 48, 65};
constexpr int kNumUniClasses = 6;

inline int uni_class_of(int len) {
  for (int i = 0; i < kNumUniClasses; ++i)
    if (len <= kUniClasses[i]) return i;
  return -1;
}

}  // namespace bs
