// Grid sizing and launch of the resultant stages (persistent kernels, optional CUDA graph).
#include <cuda_runtime.h>

#include <algorithm>

#include "ctx.cuh"

namespace bs {

// SM count that stands in for the real one when a context's grids follow the work
constexpr int kFineGridSms = 1 << 16;

static int grid_for(int64_t items, int cap) {
  if (items <= 0) return 0;
  return (int)std::min<int64_t>(items, cap);
}

// shared memory of a reconstruction block: the digit tile, three per-prime arrays and
// 3 words per limb and warp for the limb sums; when it fits, also the Garner inverses of
// the job's primes and the prefix-product rows (staged = 1)
static int crt_warps(const bs_ctx* ctx, int kmax, int lmax, size_t* smem, int* staged) {
  const size_t avail = (size_t)ctx->smem_optin - 64;
  const size_t per = (size_t)3 * lmax * sizeof(uint32_t);
  for (int st = 1; st >= 0; --st) {
    if (st && kmax > kCrtInvSmem) continue;
    const size_t fixed = ((st ? (size_t)kmax * kmax + (size_t)(kmax + 1) * lmax : 0) +
                          (size_t)kmax * kCrtTile + 3 * (size_t)kmax) * sizeof(uint32_t);
    if (fixed + per > avail) continue;
    const int w = (int)std::min<size_t>(kCrtWarps, (avail - fixed) / per);
    if (st && w < 4) continue;  // prefer more warps over staging
    *smem = fixed + per * w;
    *staged = st;
    return w;
  }
  *smem = 0;
  *staged = 0;
  return 0;
}

// shared memory of the warp-per-coefficient reconstruction block
size_t crt_warp_smem(int kmax, int lmax) {
  return ((size_t)kmax * (kmax + 1) + (size_t)kmax * kCrtTile + 3 * (size_t)kmax +
          (size_t)kCrtTile * kmax + (size_t)kCrtTile * lmax + 3 * (size_t)kmax + 4) *
         sizeof(uint32_t);
}

// NVTX ranges around each stage's launches ("bs.plan", "bs.eval", "bs.unires",
// "bs.interp", "bs.crt") let a profiler select a stage's kernels (ncu --nvtx
// --nvtx-include "bs.unires/"); without a tool attached the calls do nothing
static inline void nvtx_next(const char* name) {
  nvtxRangePop();
  nvtxRangePushA(name);
}

static inline void mark(bs_ctx* ctx, int i, cudaStream_t s) {
  if (!ctx->profile) return;
  cudaEventRecord(ctx->prof_ev[i], s);
  ctx->prof_rec[i] = true;
}

static void enqueue(bs_ctx* ctx, const StageLaunch& L, const Tables& Tv, cudaStream_t s, int crt_w,
                    size_t crt_smem, int crt_staged) {
  // fine grids: the caps below (persistent grids of a few blocks per SM) become far larger
  // than any work list, so every grid is sized by its work and each block is short
  const int sms = ctx->fine_grids ? kFineGridSms : ctx->sms;
  const size_t tsmem = sizeof(uint32_t) * (size_t)L.maxN;
  // the profiling events between the stages would separate them: no overlap then
  set_launch_pdl(L.pdl && !ctx->profile);
  mark(ctx, 1, s);
  nvtxRangePushA("bs.eval");
  int g;
  const PfHint pf{L.kt_max, 1 << L.logN_max, L.kmax};
  for (int c = 0; c < kNumEvalClasses; ++c) {
    if (L.eval_independent) {  // items are rows, kEvalIwWarps warps per block
      g = grid_for((L.evw_items[c] + kEvalIwWarps - 1) / kEvalIwWarps, (int64_t)sms * L.eval_blocks_per_sm);
      if (g) launch_eval_iw(c, g, s, L.jobs, L.evw[c], Tv, pf);
    } else {
      g = grid_for(L.evw_items[c], (int64_t)sms * L.eval_blocks_per_sm);
      if (g) launch_eval_w(c, g, L.eval_warps, s, L.jobs, L.evw[c], Tv, pf);
    }
  }
  if (L.eval_independent) {
    g = grid_for((L.evw_any_items + kEvalIwWarps - 1) / kEvalIwWarps, (int64_t)sms * kEvalIwBlocksPerSm);
    if (g) launch_eval_iw(-1, g, s, L.jobs, L.evw_any, Tv, pf);
  } else {
    g = grid_for(L.evw_any_items, (int64_t)sms * 8);
    if (g) launch_eval_w(-1, g, kEvalThreads / 32, s, L.jobs, L.evw_any, Tv, pf);
  }
  // persistent blocks of C = N / 1024 warps, about 16 warps per SM; a device plan sizes
  // this launch from the extents and usually leaves it empty, so there it stays small
  const int ecw = std::max(2, L.maxN >> 10);
  const int ebps = L.kt_max < 0 ? 2 : std::max(1, 16 / ecw);
  g = grid_for(L.eval_items, (int64_t)sms * ebps);
  if (g) launch_eval(g, ecw, s, L.jobs, L.eval, Tv);
  mark(ctx, 2, s);
  nvtx_next("bs.unires");
  for (int c = 0; c < kNumUniClasses; ++c) {
    const int th = L.uni_threads[c];
    const int ti = th == 64 ? 0 : th == 128 ? 1 : 2;
    g = grid_for((L.uni_items[c] + th - 1) / th, (int64_t)sms * ctx->occ[c][ti]);
    if (g) launch_uni(c, g, th, s, L.jobs, L.uni[c], Tv);
  }
  mark(ctx, 3, s);
  nvtx_next("bs.interp");
  g = grid_for((L.intt_w_items + kInttWarps - 1) / kInttWarps, (int64_t)sms * 8);
  if (g) launch_intt_w(g, s, L.jobs, L.intt_w, Tv);
  g = grid_for(L.intt_items, (int64_t)sms * 8);
  if (g) launch_intt(g, kInttSmemWords * tsmem, s, L.jobs, L.intt, Tv);
  mark(ctx, 4, s);
  nvtx_next("bs.crt");
  g = grid_for(L.crt_items, (int64_t)sms * L.crt_blocks_per_sm);
  const size_t wsm = crt_warp_smem(L.kmax, L.lmax);
  if (g && L.kmax <= kCrtWarpMaxK && wsm <= (size_t)ctx->smem_optin - 64)
    launch_crt_w(g, L.crt_tile, wsm, s, L.jobs, L.crt, Tv, L.kmax, L.lmax);
  else if (g)
    launch_crt(g, crt_w * 32, crt_smem, s, L.jobs, L.crt, Tv, L.kmax, L.lmax, crt_staged);
  if (L.crt_big_items[2]) {  // jobs with many primes
    launch_bigcrt(grid_for(L.crt_big_items[0], (int64_t)sms * 8),
                  grid_for(L.crt_big_items[1], (int64_t)sms * 8),
                  grid_for(L.crt_big_items[2], (int64_t)sms * 8), s, L.jobs, L.crt_big_tab,
                  L.crt_big_gemm, L.crt_big_carry, Tv);
    size_t fsm = 0;
    int fst = 0;
    const int fw = crt_warps(ctx, L.kmax_big, L.lmax_big, &fsm, &fst);
    g = grid_for(L.crt_big_items[3], (int64_t)sms * 4);
    if (g && fw) launch_crt(g, fw * 32, fsm, s, L.jobs, L.crt_big_fb, Tv, L.kmax_big, L.lmax_big, fst, 1);
  }
  set_launch_pdl(false);
  nvtxRangePop();
  mark(ctx, 5, s);
}

bool crt_warp_kernel(const bs_ctx* ctx, int kmax, int lmax) {
  return kmax <= kCrtWarpMaxK && crt_warp_smem(kmax, lmax) <= (size_t)ctx->smem_optin - 64;
}

int launch_stages(bs_ctx* ctx, const StageLaunch& L, const Tables& Tv, bool use_graph) {
  cudaStream_t s = ctx->stream;
  if (kInttSmemWords * (size_t)L.maxN * sizeof(uint32_t) > (size_t)ctx->smem_optin)  // interpolation block
    return ctx_fail(ctx, kErrRange, "transform size exceeds shared memory");
  size_t crt_smem = 0;
  int crt_staged = 0;
  const int crt_w = crt_warps(ctx, L.kmax, L.lmax, &crt_smem, &crt_staged);
  if (crt_w == 0) return ctx_fail(ctx, kErrRange, "too many primes for the reconstruction stage");
  if (ctx->profile) {
    for (int i = 0; i < kProfEvents; ++i) ctx->prof_rec[i] = false;
    mark(ctx, 0, s);
  }
  if (!use_graph || ctx->profile) {
    enqueue(ctx, L, Tv, s, crt_w, crt_smem, crt_staged);
    return ctx_cuda(ctx, cudaGetLastError(), "stage launch");
  }
  cudaGraph_t graph = nullptr;
  int rc = ctx_cuda(ctx, cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal), "capture");
  if (rc) return rc;
  enqueue(ctx, L, Tv, s, crt_w, crt_smem, crt_staged);
  cudaError_t le = cudaGetLastError();
  cudaError_t ce = cudaStreamEndCapture(s, &graph);
  if (le != cudaSuccess || ce != cudaSuccess) {
    if (graph) cudaGraphDestroy(graph);
    return ctx_cuda(ctx, le != cudaSuccess ? le : ce, "graph capture");
  }
  bool updated = false;
  if (ctx->graph_exec) {
    cudaGraphExecUpdateResultInfo info;
    if (cudaGraphExecUpdate(ctx->graph_exec, graph, &info) == cudaSuccess) {
      updated = true;
    } else {
      cudaGetLastError();
      cudaGraphExecDestroy(ctx->graph_exec);
      ctx->graph_exec = nullptr;
    }
  }
  if (!updated) {
    rc = ctx_cuda(ctx, cudaGraphInstantiate(&ctx->graph_exec, graph, 0), "graph instantiate");
    if (rc) {
      cudaGraphDestroy(graph);
      ctx->graph_exec = nullptr;
      return rc;
    }
  }
  cudaGraphDestroy(graph);
  return ctx_cuda(ctx, cudaGraphLaunch(ctx->graph_exec, s), "graph launch");
}

int launch_device_job(bs_ctx* ctx, const Job& J, Job* dj, int64_t* offs, const MetaBounds& mb,
                      int cls) {
  cudaStream_t s = ctx->stream;
  const Tables Tv = ctx->tabs->view();
  const int N = 1 << mb.logN;
  if (kInttSmemWords * (size_t)N * sizeof(uint32_t) > (size_t)ctx->smem_optin)  // interpolation block
    return ctx_fail(ctx, kErrRange, "transform size exceeds shared memory");
  if (ctx->profile)
    for (int i = 0; i < kProfEvents; ++i) ctx->prof_rec[i] = false;
  mark(ctx, 0, s);
  // the plan kernel receives the job by value, zeroes its prime flags and stores the
  // planned job for the stage kernels
  const bool indep = ctx->tune.eval_independent != 0;
  nvtxRangePushA("bs.plan");
  launch_plan_single(s, J, dj, offs, Tv, indep ? 1 : kEvalThreads / 32);
  nvtxRangePop();
  StageLaunch L;
  L.jobs = dj;
  const bool wsize = mb.logN <= kWarpLogNMax;  // the actual size is at most the bound
  for (int c = 0; c < kNumEvalClasses; ++c) {
    L.evw[c] = WorkList{nullptr, offs + kOffEvalW, 1};
    L.evw_items[c] = 0;
  }
  L.eval = WorkList{nullptr, offs + kOffEvalS, 1};
  for (int c = 0; c < kNumUniClasses; ++c) {
    L.uni[c] = WorkList{nullptr, offs + kOffUni, 1};
    L.uni_items[c] = 0;
  }
  L.uni_items[cls] = (int64_t)mb.k_total << mb.logN;  // instances
  L.intt = WorkList{nullptr, offs + kOffInttS, 1};
  L.intt_w = WorkList{nullptr, offs + kOffInttW, 1};
  L.crt = WorkList{nullptr, offs + kOffCrt, 1};
  // the transform size is known on the device only: one kernel dispatches per job
  L.evw_any = WorkList{nullptr, offs + kOffEvalW, 1};
  L.eval_independent = indep;
  L.evw_any_items = indep ? (int64_t)mb.k_total * mb.rows : (int64_t)mb.k_total * ((mb.rows + 7) / 8);
  L.eval_items = wsize ? 0 : (int64_t)mb.k_total * mb.rows;
  // a single job has few primes: one block per prime (no second, possibly empty launch)
  L.intt_w_items = 0;
  L.intt_items = mb.k_total;
  L.crt_items = ((int64_t)J.cap_deg + kCrtTile) / kCrtTile;
  L.maxN = N;
  L.kt_max = -1;  // the evaluation kernel reads the device plan for its prefetch sizes
  L.logN_max = 0;
  L.kmax = mb.k_need;
  L.lmax = J.cap_limbs;
  L.pdl = true;
  size_t crt_smem = 0;
  int crt_staged = 0;
  const int crt_w = crt_warps(ctx, L.kmax, L.lmax, &crt_smem, &crt_staged);
  if (crt_w == 0) return ctx_fail(ctx, kErrRange, "too many primes for the reconstruction stage");
  enqueue(ctx, L, Tv, s, crt_w, crt_smem, crt_staged);
  return ctx_cuda(ctx, cudaGetLastError(), "stage launch");
}

}  // namespace bs

void ctx_release_extra(bs_ctx* ctx) {
  for (int i = 0; i < kProfEvents; ++i)
    if (ctx->prof_ev[i]) cudaEventDestroy(ctx->prof_ev[i]);
  if (ctx->graph_exec) cudaGraphExecDestroy(ctx->graph_exec);
  ctx->graph_exec = nullptr;
}
