// Host-side context of libbsres.
#pragma once
#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>

#include <string>

#include "../../include/bsres.h"
#include "common.cuh"
#include "resultant_kernels.cuh"
#include "tables.cuh"

namespace bs {

// names a host call for a profiler (an NVTX range over the call); nothing without one
struct NvtxScope {
  explicit NvtxScope(const char* name) { nvtxRangePushA(name); }
  ~NvtxScope() { nvtxRangePop(); }
  NvtxScope(const NvtxScope&) = delete;
  NvtxScope& operator=(const NvtxScope&) = delete;
};
// launch shapes of the batched stages: defaults, or what bs_autotune_batch measured best
// for a batch (the device-planned single job always uses the defaults)
struct Tune {
  int eval_warps = 8;           // rows (one warp each) per evaluation block, 1..8
  int eval_blocks_per_sm = 5;   // cap of the persistent evaluation grid
  int uni_threads[kNumUniClasses] = {128, 128, 128, 128, 128, 128};  // 64, 128 or 256
  int crt_tile = 8;             // coefficients (one warp each) per reconstruction block, 1..8
  int crt_blocks_per_sm = 4;    // cap of the persistent reconstruction grid
  int eval_independent = 1;     // 1: independent-warp evaluation (k_eval_iw), rows per item 1;
                                // 0: blocks of eval_warps rows of one prime (k_eval_w)
};
constexpr int kUniThreadChoices[3] = {64, 128, 256};
}  // namespace bs

struct bs_ctx {
  int device = 0;
  int sms = 0;
  int smem_optin = 48 * 1024;
  size_t budget = 0;
  cudaStream_t own_stream = nullptr;
  // serving slots: a second stream of the lowest priority for large batches (own_stream
  // has the highest), and grids sized by the work instead of the SMs for those batches, so
  // that blocks of small batches are scheduled between theirs
  cudaStream_t aux_stream = nullptr;
  bool fine_grids = false;
  cudaStream_t stream = nullptr;
  bs::DeviceTables own_tabs;
  bs::DeviceTables* tabs = &own_tabs;  // serving slots point at their parent's tables
  bs_ctx* parent = nullptr;            // set on the serving slots' contexts
  struct bs_server* server = nullptr;  // serving loop (bs_serve_start)
  // workspace of host-planned calls
  void* ws = nullptr;
  size_t ws_cap = 0;
  int ws_generation = 0;
  // workspace of device-planned calls
  void* dev_ws = nullptr;
  size_t dev_ws_cap = 0;
  // pinned staging
  void* h_up = nullptr;
  size_t h_up_cap = 0;
  void* h_down = nullptr;
  size_t h_down_cap = 0;
  int32_t* d_status = nullptr;  // [status, rejected, -, -] of device-planned calls
  int occ[bs::kNumUniClasses][3] = {};  // resident univariate blocks per SM (64/128/256 threads)
  bs::Tune tune;
  // cached executable graph of the batched stages
  cudaGraphExec_t graph_exec = nullptr;
  std::string err;
  bs_stats stats{};
  // per-stage timing: events 0..5 bracket plan | eval | unires | intt | crt
  bool profile = false;
  cudaEvent_t prof_ev[6] = {nullptr, nullptr, nullptr, nullptr, nullptr, nullptr};
  bool prof_rec[6] = {false, false, false, false, false, false};
};

constexpr int kProfEvents = 6;

namespace bs {

// bump layout with 256-byte alignment
struct Layout {
  size_t used = 0;
  size_t take(size_t bytes) {
    size_t off = (used + 255) & ~(size_t)255;
    used = off + bytes;
    return off;
  }
};

struct MetaBounds {
  int32_t D, logN, rows, len, k_total, k_need, out_limbs;
};

// upper bounds of a resultant job from the grids' extents and limb counts only (the sizes
// of the device-planned entry points' workspace); BS_ERR_RANGE beyond the supported sizes
int meta_bounds(const bs_bipoly* f, const bs_bipoly* g, int var, MetaBounds* mb);

struct StageLaunch {
  const Job* jobs;
  WorkList eval, intt, intt_w, crt;
  // reconstruction of many primes: tables, contraction, carries, Garner for rejections
  WorkList crt_big_tab{nullptr, nullptr, 0}, crt_big_gemm{nullptr, nullptr, 0},
      crt_big_carry{nullptr, nullptr, 0}, crt_big_fb{nullptr, nullptr, 0};
  int64_t crt_big_items[4] = {0, 0, 0, 0};
  int kmax_big = 1, lmax_big = 1;
  WorkList evw[kNumEvalClasses];  // warp evaluation, one list per transform-size class
  WorkList evw_any;               // warp evaluation of any size class (device plans)
  WorkList uni[kNumUniClasses];
  int64_t eval_items, intt_items, intt_w_items, crt_items;
  int64_t evw_items[kNumEvalClasses], evw_any_items;
  int eval_warps = 8, eval_blocks_per_sm = 8, crt_tile = kCrtTile, crt_blocks_per_sm = 4;
  bool eval_independent = false;  // k_eval_iw (work lists count single rows)
  bool pdl = false;  // programmatic dependent launch between the stage kernels
  int uni_threads[kNumUniClasses] = {kUniTile, kUniTile, kUniTile, kUniTile, kUniTile, kUniTile};
  int64_t uni_items[kNumUniClasses];
  int maxN, kmax, lmax;
  int kt_max, logN_max;  // largest prime count and transform size (L2 prefetch)
};

int launch_stages(bs_ctx* ctx, const StageLaunch& L, const Tables& Tv, bool use_graph);
// whether the reconstruction of a batch runs in the warp-per-coefficient kernel (whose
// block size is tunable) or in the block Garner kernel (tiles of kCrtTile coefficients)
bool crt_warp_kernel(const bs_ctx* ctx, int kmax, int lmax);
// shared memory of the warp-per-coefficient reconstruction block
size_t crt_warp_smem(int kmax, int lmax);
int launch_device_job(bs_ctx* ctx, const Job& J, Job* dj, int64_t* offs, const MetaBounds& mb,
                      int cls);

}  // namespace bs

int ctx_fail(bs_ctx* ctx, int code, const std::string& msg);
// the host message of a device status word [status, rejected, debug site, -]
std::string device_failure_detail(const int32_t* st);
int ctx_cuda(bs_ctx* ctx, cudaError_t e, const char* what);
int ensure_workspace(bs_ctx* ctx, size_t bytes);
void ctx_release_extra(bs_ctx* ctx);
