// Grid sizing and launch of the resultant stages (persistent kernels, optional CUDA graph).
#include <cuda_runtime.h>

#include <algorithm>

#include "ctx.cuh"

namespace bs {

__global__ void k_store_job(Job J, Job* dst) {
  if (threadIdx.x == 0 && blockIdx.x == 0) *dst = J;
}

static int grid_for(int64_t items, int cap) {
  if (items <= 0) return 0;
  return (int)std::min<int64_t>(items, cap);
}

static int crt_warps(const bs_ctx* ctx, int kmax, int lmax, size_t* smem) {
  const size_t per = (size_t)(4 * kmax + lmax) * sizeof(uint32_t);
  int w = (int)std::min<size_t>(kCrtWarps, (size_t)ctx->smem_optin / per);
  if (w < 1) w = 0;
  *smem = per * (w > 0 ? w : 1);
  return w;
}

static inline void mark(bs_ctx* ctx, int i, cudaStream_t s) {
  if (!ctx->profile) return;
  cudaEventRecord(ctx->prof_ev[i], s);
  ctx->prof_rec[i] = true;
}

static void enqueue(bs_ctx* ctx, const StageLaunch& L, const Tables& Tv, cudaStream_t s, int crt_w,
                    size_t crt_smem) {
  const int sms = ctx->sms;
  const size_t tsmem = sizeof(uint32_t) * (size_t)L.maxN;
  mark(ctx, 1, s);
  int g = grid_for(L.eval_items, (int64_t)sms * 8);
  if (g) launch_eval(g, tsmem, s, L.jobs, L.eval, Tv);
  mark(ctx, 2, s);
  for (int c = 0; c < kNumUniClasses; ++c) {
    g = grid_for(L.uni_items[c], (int64_t)sms * ctx->occ[c]);
    if (g) launch_uni(c, g, s, L.jobs, L.uni[c], Tv);
  }
  mark(ctx, 3, s);
  g = grid_for(L.intt_items, (int64_t)sms * 8);
  if (g) launch_intt(g, tsmem, s, L.jobs, L.intt, Tv);
  mark(ctx, 4, s);
  g = grid_for((L.crt_items + crt_w - 1) / crt_w, (int64_t)sms * 4);
  if (g) launch_crt(g, crt_w * 32, crt_smem, s, L.jobs, L.crt, Tv, L.kmax, L.lmax);
  mark(ctx, 5, s);
}

int launch_stages(bs_ctx* ctx, const StageLaunch& L, const Tables& Tv, bool use_graph) {
  cudaStream_t s = ctx->stream;
  if ((size_t)L.maxN * sizeof(uint32_t) > (size_t)ctx->smem_optin)
    return ctx_fail(ctx, kErrRange, "transform size exceeds shared memory");
  size_t crt_smem = 0;
  const int crt_w = crt_warps(ctx, L.kmax, L.lmax, &crt_smem);
  if (crt_w == 0) return ctx_fail(ctx, kErrRange, "too many primes for the reconstruction stage");
  if (ctx->profile) {
    for (int i = 0; i < kProfEvents; ++i) ctx->prof_rec[i] = false;
    mark(ctx, 0, s);
  }
  if (!use_graph || ctx->profile) {
    enqueue(ctx, L, Tv, s, crt_w, crt_smem);
    return ctx_cuda(ctx, cudaGetLastError(), "stage launch");
  }
  cudaGraph_t graph = nullptr;
  int rc = ctx_cuda(ctx, cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal), "capture");
  if (rc) return rc;
  enqueue(ctx, L, Tv, s, crt_w, crt_smem);
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
  const Tables Tv = ctx->tabs.view();
  const int N = 1 << mb.logN;
  if ((size_t)N * sizeof(uint32_t) > (size_t)ctx->smem_optin)
    return ctx_fail(ctx, kErrRange, "transform size exceeds shared memory");
  if (ctx->profile)
    for (int i = 0; i < kProfEvents; ++i) ctx->prof_rec[i] = false;
  mark(ctx, 0, s);
  k_store_job<<<1, 32, 0, s>>>(J, dj);
  cudaMemsetAsync(J.pstat, 0, sizeof(int32_t) * mb.k_total, s);
  launch_plan_single(s, dj, offs, Tv);
  StageLaunch L;
  L.jobs = dj;
  L.eval = WorkList{nullptr, offs + 0, 1};
  for (int c = 0; c < kNumUniClasses; ++c) {
    L.uni[c] = WorkList{nullptr, offs + 2, 1};
    L.uni_items[c] = 0;
  }
  L.uni_items[cls] = (((int64_t)mb.k_total << mb.logN) + kUniTile - 1) / kUniTile;
  L.intt = WorkList{nullptr, offs + 4, 1};
  L.crt = WorkList{nullptr, offs + 6, 1};
  L.eval_items = (int64_t)mb.k_total * mb.rows;
  L.intt_items = mb.k_total;
  L.crt_items = (int64_t)J.cap_deg + 1;
  L.maxN = N;
  L.kmax = mb.k_need;
  L.lmax = J.cap_limbs;
  size_t crt_smem = 0;
  const int crt_w = crt_warps(ctx, L.kmax, L.lmax, &crt_smem);
  if (crt_w == 0) return ctx_fail(ctx, kErrRange, "too many primes for the reconstruction stage");
  enqueue(ctx, L, Tv, s, crt_w, crt_smem);
  return ctx_cuda(ctx, cudaGetLastError(), "stage launch");
}

}  // namespace bs

void ctx_release_extra(bs_ctx* ctx) {
  for (int i = 0; i < kProfEvents; ++i)
    if (ctx->prof_ev[i]) cudaEventDestroy(ctx->prof_ev[i]);
  if (ctx->graph_exec) cudaGraphExecDestroy(ctx->graph_exec);
  ctx->graph_exec = nullptr;
  if (ctx->extra) cudaFree(ctx->extra);
  ctx->extra = nullptr;
  ctx->extra_cap = 0;
}
