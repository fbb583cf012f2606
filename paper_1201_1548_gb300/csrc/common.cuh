// Device-side data structures shared by the resultant kernels.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "modarith.cuh"
#include "plan.cuh"

namespace bs {

enum Status : int32_t {
  kOk = 0,
  kErrArg = 1,
  kErrNoMem = 2,
  kErrUnlucky = 3,
  kErrTimeout = 4,
  kErrCuda = 5,
  kErrZero = 6,
  kErrRange = 7,
  kErrInternal = 8,
  kErrCapacity = 9,
};

// per-prime constants (indexed by the prime's position in the table)
struct PrimeConst {
  uint32_t p;
  uint32_t pinv;   // p^-1 mod 2^32
  uint32_t one_m;  // 2^32 mod p   (Montgomery form of 1)
  uint32_t r2;     // 2^64 mod p
  uint32_t g;      // smallest primitive root (standard form): omega = g^((p-1)/N)
  uint32_t c_m;    // coset representative c (Montgomery form): the points are c omega^t
  uint32_t half;   // (p - 1) / 2
  uint32_t pad;
};

// device tables owned by a context
struct Tables {
  const PrimeConst* pc;  // [T]
  const uint32_t* pw;    // [T][kMaxLimbs + 1]: 2^(32 l) * 2^64 mod p
  const uint32_t* mpw;   // [T][kMaxLimbs + 1]: Montgomery form of 2^(32 l)
  const int64_t* lg_prefix;  // [T + 1]: sums of lower bounds of log2 p (Q16)
  // transform tables for the first Tt primes, row length NT
  const uint32_t* tw;    // [Tt][NT/2] omega^i, omega of order NT (Montgomery)
  const uint32_t* itw;   // [Tt][NT/2] omega^-i (Montgomery)
  const uint32_t* cp;    // [Tt][NT] c^i, c the coset representative (Montgomery)
  const uint32_t* icp;   // [Tt][NT] c^-i (standard form)
  const uint32_t* ninv;  // [Tt][kLogNMax + 1] 2^-s (Montgomery form)
  // packed twiddles [Tt][NT]: twp[len + j] = omega_{2 len}^j, itwp[len + j] = omega_{2 len}^-j
  // (len = 1, 2, ..., NT/2; j < len; entry 0 is 1), Montgomery form
  const uint32_t* twp;
  const uint32_t* itwp;
  // [Tt][64]: for j = 1 .. 31, tws[2 j] = twp[j] in standard form w and tws[2 j + 1] =
  // floor(w 2^32 / p), the pairs of Shoup's products in the transforms' short stages;
  // j = 0 holds the pair of 1
  const uint32_t* tws;
  // Garner table for the first Tg primes: ginv[a * Tg + b] = p_a^-1 mod p_b (Montgomery)
  const uint32_t* ginv;
  // prefix products of the table primes: pp[j * LPP + l] = limb l of p_0 ... p_{j-1}
  // (j = 0..Tg), zero above the product's length
  const uint32_t* pp;
  int32_t LPP;
  // weighted-sum reconstruction for the first k table primes, k = 1..WK:
  //   ws_m + ws_moff[k] : M_k[i] = (p_0 ... p_{k-1}) / p_i, k rows of ws_len(k) limbs
  //   ws_y + ws_yoff[k] : y_k[i] = M_k[i]^-1 mod p_i (standard form)
  //   q62[i] = floor(2^62 / p_i)
  const uint32_t* ws_m;
  const int64_t* ws_moff;
  const uint32_t* ws_y;
  const int32_t* ws_yoff;
  const uint32_t* q62;
  int64_t ws_m_words;  // allocation size of ws_m in words
  int32_t WK;
  int32_t T, Tt, NT, logNT, Tg;
};

// limbs of the weighted-sum tables for k primes (P_k < 2^(31 k))
__host__ __device__ __forceinline__ int ws_len(int k) { return (31 * k + 31) / 32 + 1; }

// one resultant job as the kernels see it
struct Job {
  Grid f, g;
  int32_t var;
  int32_t rows;   // (me + 1) + (ne + 1)
  Plan plan;
  uint32_t* ev;    // [k_total][rows][N] evaluations (Montgomery form)
  uint32_t* vals;  // [k_total][N] univariate resultants (Montgomery form, bit-reversed order)
  // 1 (host batches whose transforms are interpolated one warp per prime): the univariate
  // stage leaves each value's numerator in vals and its denominator in the instance's
  // first evaluation word ev[q][0][t] (read by the instance itself, then dead), and the
  // interpolating warp divides them with one inversion per prime (Montgomery's
  // simultaneous inversion); 0: vals are final
  int32_t den_in_ev;
  uint32_t* rmod;  // [k_need][D + 1] residues of the result coefficients (standard form)
  int32_t* pstat;  // [k_total] 0 = good prime, 1 = rejected
  int32_t* sel;    // [k_need] table index of the j-th selected prime
  uint32_t* out;   // [cap_deg + 1][cap_limbs]
  int32_t cap_deg, cap_limbs;
  int32_t* status;  // sticky device status word of the call
  int32_t* rejected;  // counter of rejected primes (may be null)
  // workspace capacities (device-planned jobs): the plan must fit them
  int32_t cap_k_total, cap_k_need, cap_rows, cap_logN, cap_D;
  // weighted-sum reconstruction of many primes (host batches with k_need > 160; null
  // otherwise): wsM [k_need][wsL] M_j = P / p_j, wsY [k_need] y_j (Montgomery form),
  // wsS [3][cap_deg + 1][wsL] column sums of sum_j t_j M_j
  uint32_t* wsM;
  uint32_t* wsY;
  uint32_t* wsS;
  int32_t wsL;
  // principal subresultant coefficients (psc jobs; 0 otherwise): the univariate stage
  // writes sr_i of instance t to vals[i * psc_stride + t], i < npsc
  int32_t npsc;
  int64_t psc_stride;
};

// Programmatic dependent launch: a stage kernel launched with programmatic stream
// serialisation may start while its predecessor finishes; it waits for the predecessor's
// results before touching them, and lets its own successor launch once its blocks are
// done.  Both instructions are no-ops for an ordinary launch.
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

// Asynchronous 4-byte copy from global to shared memory (cp.async, no register staging):
// a thread issues many and waits once with cp_async_wait_all (a hardware wait).
__device__ __forceinline__ void cp_async4(uint32_t* sdst, const uint32_t* gsrc) {
  const unsigned sa = (unsigned)__cvta_generic_to_shared(sdst);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(sa), "l"(gsrc) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }

// work lists: stage work of job ids[i] occupies [off[i], off[i+1]) of a flat index space
struct WorkList {
  const int32_t* ids;  // may be null: identity
  const int64_t* off;  // n + 1 entries
  int32_t n;
};

__device__ __forceinline__ int find_item(const int64_t* off, int n, int64_t item) {
  int lo = 0, hi = n - 1;
  while (lo < hi) {
    int mid = (lo + hi + 1) >> 1;
    if (off[mid] <= item)
      lo = mid;
    else
      hi = mid - 1;
  }
  return lo;
}

__device__ __forceinline__ void set_status(int32_t* st, int32_t code) {
  if (st) atomicCAS(st, 0, code);
}

// Debug bounds checks, compiled in with -DBS_DEBUG_CHECKS (the library built by
// build(debug=True)): a failed check records kErrInternal in the call's status word and
// the site number (kDbg*) in its third word, and the guarded access is skipped, so a bad
// index is reported to the host instead of faulting.  Without the flag every check is
// the constant true and costs nothing.
enum DebugSite : int32_t {
  kDbgEvalIn = 11, kDbgEvalOut = 12, kDbgEvalTab = 13, kDbgEvalPf = 14,
  kDbgUniIn = 21, kDbgUniOut = 22, kDbgUniStat = 23, kDbgUniPrime = 24,
  kDbgInttIn = 31, kDbgInttOut = 32, kDbgInttSel = 33, kDbgInttTab = 34,
  kDbgCrtIn = 41, kDbgCrtSel = 42, kDbgCrtOut = 43, kDbgCrtWs = 44, kDbgCrtGinv = 45,
  kDbgCrtPp = 46,
};
#ifdef BS_DEBUG_CHECKS
__device__ __forceinline__ bool dbg_ok(bool cond, int32_t* st, int32_t site) {
  if (!cond && st) {
    atomicCAS(st, 0, kErrInternal);
    atomicCAS(st + 2, 0, site);
  }
  return cond;
}
#else
__device__ __forceinline__ constexpr bool dbg_ok(bool, int32_t*, int32_t) { return true; }
#endif
// elements of a job's buffers, from its plan (a device-planned job's capacities are at
// least these)
__device__ __forceinline__ int64_t job_ev_words(const Job* J) {
  return (int64_t)J->plan.k_total * J->rows * J->plan.N;
}
__device__ __forceinline__ int64_t job_vals_words(const Job* J) { return (int64_t)J->plan.k_total * J->plan.N; }
__device__ __forceinline__ int64_t job_rmod_words(const Job* J) {
  return (int64_t)J->plan.k_need * (J->plan.D + 1);
}
__device__ __forceinline__ int64_t job_out_words(const Job* J) {
  return (int64_t)(J->cap_deg + 1) * J->cap_limbs;
}
__device__ __forceinline__ int64_t grid_words(const Grid& g) {
  return (int64_t)(g.dx + 1) * (g.dy + 1) * g.L;
}

}  // namespace bs
