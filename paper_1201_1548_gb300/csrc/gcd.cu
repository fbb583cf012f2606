// gcd in Z_p[x] (Sec. 5.1, "Computing gcds in Z[x]", step (b)).
//
// One block per instance.  Both polynomials sit in shared memory; every step removes
// the leading term of the longer one with the division-free update
// A <- lc(B) A - lc(A) x^(deg A - deg B) B, which keeps gcd(A, B) up to a unit.  The
// last non-zero polynomial is made monic with a single inversion.
#include <cuda_runtime.h>

#include <algorithm>
#include <vector>

#include "ctx.cuh"

namespace bs {

struct GcdJob {
  const uint32_t* a;  // standard form, ascending
  const uint32_t* b;
  int32_t da, db;     // degrees (-1: zero polynomial)
  uint32_t p, pinv, r2, one_m;
  uint32_t* g;        // output, monic, standard form, capacity max(da, db) + 1
  int32_t* dg;        // output degree
};

__device__ void gcd_block(const GcdJob& J, uint32_t* sA, uint32_t* sB) {
  const Mod M{J.p, J.pinv};
  const int cap = max(J.da, J.db) + 1;
  for (int i = threadIdx.x; i < cap; i += blockDim.x) {
    sA[i] = (i <= J.da) ? redc((uint64_t)J.a[i] * J.r2, M.p, M.pinv) : 0u;
    sB[i] = (i <= J.db) ? redc((uint64_t)J.b[i] * J.r2, M.p, M.pinv) : 0u;
  }
  __shared__ int s_la, s_lb, s_swap;
  __syncthreads();
  if (threadIdx.x == 0) {
    int la = J.da, lb = J.db;
    while (la >= 0 && sA[la] == 0) --la;
    while (lb >= 0 && sB[lb] == 0) --lb;
    s_la = la;
    s_lb = lb;
  }
  __syncthreads();
  uint32_t* A = sA;
  uint32_t* B = sB;
  int la = s_la, lb = s_lb;
  // invariant: la >= lb after the swap; stop when B is zero
  while (true) {
    if (la < lb) {
      uint32_t* t = A;
      A = B;
      B = t;
      int u = la;
      la = lb;
      lb = u;
    }
    if (lb < 0) break;
    const int k = la - lb;
    const uint32_t a0 = A[la], b0 = B[lb];
    const uint32_t na0 = mneg(a0, M.p);
    for (int i = threadIdx.x; i < la; i += blockDim.x) {
      const uint32_t bi = (i >= k) ? B[i - k] : 0u;
      A[i] = redc((uint64_t)b0 * A[i] + (uint64_t)na0 * bi, M.p, M.pinv);
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      int l = la - 1;
      while (l >= 0 && A[l] == 0) --l;
      s_la = l;
      s_swap = 0;
    }
    __syncthreads();
    la = s_la;
  }
  // A holds the gcd (degree la), or both are zero (la = -1)
  const uint32_t lc = la >= 0 ? A[la] : J.one_m;
  const uint32_t ilc = minv(lc, J.one_m, M);
  for (int i = threadIdx.x; i <= la; i += blockDim.x)
    J.g[i] = redc((uint64_t)mmul(A[i], ilc, M), M.p, M.pinv);
  if (threadIdx.x == 0) *J.dg = la;
}

__global__ void k_gcd_modp(const GcdJob* jobs, int n, int cap_words) {
  extern __shared__ uint32_t sm[];
  for (int i = blockIdx.x; i < n; i += gridDim.x) {
    gcd_block(jobs[i], sm, sm + cap_words);
    __syncthreads();
  }
}

}  // namespace bs

using namespace bs;

extern "C" int bs_gcd_modp(bs_ctx* ctx, const uint32_t* a, int da, const uint32_t* b, int db,
                           uint32_t p, uint32_t* g, int* dg) {
  if (!ctx) return BS_ERR_ARG;
  if (da < -1 || db < -1 || !g || !dg || (da >= 0 && !a) || (db >= 0 && !b) || p < 3 ||
      p >= (1u << 31) || (p & 1u) == 0)
    return ctx_fail(ctx, BS_ERR_ARG, "bad arguments");
  for (int i = 0; i <= da; ++i)
    if (a[i] >= p) return ctx_fail(ctx, BS_ERR_ARG, "input not reduced");
  for (int i = 0; i <= db; ++i)
    if (b[i] >= p) return ctx_fail(ctx, BS_ERR_ARG, "input not reduced");
  const int cap = std::max(da, db) + 1;
  if (cap == 0) {
    *dg = -1;
    return BS_OK;
  }
  if ((size_t)2 * cap * sizeof(uint32_t) > (size_t)ctx->smem_optin)
    return ctx_fail(ctx, BS_ERR_RANGE, "degree too large for one block");
  cudaSetDevice(ctx->device);
  Layout lay;
  const size_t o_a = lay.take(sizeof(uint32_t) * std::max(da + 1, 1));
  const size_t o_b = lay.take(sizeof(uint32_t) * std::max(db + 1, 1));
  const size_t o_g = lay.take(sizeof(uint32_t) * cap);
  const size_t o_dg = lay.take(sizeof(int32_t));
  const size_t o_job = lay.take(sizeof(GcdJob));
  int rc = ensure_workspace(ctx, lay.used);
  if (rc) return rc;
  char* base = (char*)ctx->ws;
  cudaStream_t s = ctx->stream;
  GcdJob J;
  J.a = (const uint32_t*)(base + o_a);
  J.b = (const uint32_t*)(base + o_b);
  J.da = da;
  J.db = db;
  J.p = p;
  J.pinv = host_pinv(p);
  J.one_m = (uint32_t)((1ull << 32) % p);
  J.r2 = (uint32_t)(((uint64_t)J.one_m << 32) % p);
  J.g = (uint32_t*)(base + o_g);
  J.dg = (int32_t*)(base + o_dg);
  if (da >= 0) rc |= ctx_cuda(ctx, cudaMemcpyAsync(base + o_a, a, sizeof(uint32_t) * (da + 1), cudaMemcpyHostToDevice, s), "h2d");
  if (db >= 0) rc |= ctx_cuda(ctx, cudaMemcpyAsync(base + o_b, b, sizeof(uint32_t) * (db + 1), cudaMemcpyHostToDevice, s), "h2d");
  rc |= ctx_cuda(ctx, cudaMemcpyAsync(base + o_job, &J, sizeof(J), cudaMemcpyHostToDevice, s), "h2d");
  if (rc) return rc;
  const size_t smem = (size_t)2 * cap * sizeof(uint32_t);
  if (smem > 48 * 1024 && set_dyn_smem_limit((const void*)k_gcd_modp, ctx->smem_optin) != 0)
    return ctx_fail(ctx, BS_ERR_CUDA, "shared memory limit");
  const int threads = std::min(1024, std::max(32, ((cap + 31) / 32) * 32));
  k_gcd_modp<<<1, threads, smem, s>>>((const GcdJob*)(base + o_job), 1, cap);
  rc = ctx_cuda(ctx, cudaGetLastError(), "launch");
  if (rc) return rc;
  int32_t hdg = -1;
  rc = ctx_cuda(ctx, cudaMemcpyAsync(&hdg, J.dg, sizeof(int32_t), cudaMemcpyDeviceToHost, s), "d2h");
  if (rc) return rc;
  rc = ctx_cuda(ctx, cudaStreamSynchronize(s), "stream");
  if (rc) return rc;
  *dg = hdg;
  if (hdg >= 0) {
    rc = ctx_cuda(ctx, cudaMemcpy(g, J.g, sizeof(uint32_t) * (hdg + 1), cudaMemcpyDeviceToHost), "d2h");
    if (rc) return rc;
  }
  return BS_OK;
}
