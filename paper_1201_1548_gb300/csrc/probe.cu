// Integer-multiply throughput probe (the denominator of the ALU roofline) and per-stage
// event timing of the resultant pipeline.
//
// The probe runs eight independent dependency chains per thread on every SM and counts
// one operation per executed instruction of the probed kind:
//   0  mad.lo.u32     (32-bit multiply-add, low word)
//   1  mad.hi.u32     (32-bit multiply-add, high word)
//   2  mad.wide.u32   (32 x 32 -> 64-bit multiply-add)
//   3  the library's Montgomery multiplication mod a 31-bit prime (one mulmod)
#include <cuda_runtime.h>

#include "ctx.cuh"

namespace bs {

template <int KIND>
__global__ void k_probe(uint32_t* out, int iters, uint32_t seed) {
  const uint32_t tid = blockIdx.x * blockDim.x + threadIdx.x;
  uint32_t a[8];
  uint64_t w[8];
#pragma unroll
  for (int c = 0; c < 8; ++c) {
    a[c] = seed * (tid + 1) + 977u * c;
    w[c] = a[c];
  }
  const uint32_t b = seed | 1u, k = 0x9e3779b9u;
  const Mod M{2147352577u, 0u};
  uint32_t pinv = 2147352577u;
  for (int i = 0; i < 5; ++i) pinv *= 2u - 2147352577u * pinv;
  const Mod MM{M.p, pinv};
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int c = 0; c < 8; ++c) {
      if (KIND == 0) {
        asm volatile("mad.lo.u32 %0, %0, %1, %2;" : "+r"(a[c]) : "r"(b), "r"(k));
      } else if (KIND == 1) {
        asm volatile("mad.hi.u32 %0, %0, %1, %2;" : "+r"(a[c]) : "r"(b), "r"(k));
      } else if (KIND == 2) {
        asm volatile("mad.wide.u32 %0, %1, %2, %0;" : "+l"(w[c]) : "r"((uint32_t)w[c]), "r"(b));
      } else {
        a[c] = mmul(a[c] & 0x3fffffffu, b & 0x3fffffffu, MM);
      }
    }
  }
  uint32_t x = 0;
#pragma unroll
  for (int c = 0; c < 8; ++c) x ^= a[c] ^ (uint32_t)w[c] ^ (uint32_t)(w[c] >> 32);
  out[tid] = x;
}

}  // namespace bs

using namespace bs;

extern "C" int bs_alu_probe(bs_ctx* ctx, int kind, double* ops_per_s) {
  if (!ctx || !ops_per_s || kind < 0 || kind > 3) return BS_ERR_ARG;
  cudaSetDevice(ctx->device);
  const int threads = 256, blocks = ctx->sms * 8, iters = 4096;
  uint32_t* out = nullptr;
  if (cudaMalloc(&out, sizeof(uint32_t) * threads * blocks) != cudaSuccess)
    return ctx_fail(ctx, BS_ERR_NOMEM, "probe buffer");
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  cudaStream_t s = ctx->stream;
  float best = 1e30f;
  for (int rep = 0; rep < 4; ++rep) {
    cudaEventRecord(e0, s);
    switch (kind) {
      case 0: k_probe<0><<<blocks, threads, 0, s>>>(out, iters, 12345u + rep); break;
      case 1: k_probe<1><<<blocks, threads, 0, s>>>(out, iters, 12345u + rep); break;
      case 2: k_probe<2><<<blocks, threads, 0, s>>>(out, iters, 12345u + rep); break;
      default: k_probe<3><<<blocks, threads, 0, s>>>(out, iters, 12345u + rep); break;
    }
    cudaEventRecord(e1, s);
    cudaEventSynchronize(e1);
    float ms = 0;
    cudaEventElapsedTime(&ms, e0, e1);
    if (rep > 0 && ms < best) best = ms;  // first launch is a warm-up
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFree(out);
  int rc = ctx_cuda(ctx, cudaGetLastError(), "probe");
  if (rc) return rc;
  const double ops = (double)threads * blocks * iters * 8.0;
  *ops_per_s = ops / (best * 1e-3);
  return BS_OK;
}

extern "C" int bs_profile(bs_ctx* ctx, int enable) {
  if (!ctx) return BS_ERR_ARG;
  if (enable && !ctx->prof_ev[0]) {
    for (int i = 0; i < kProfEvents; ++i) cudaEventCreate(&ctx->prof_ev[i]);
  }
  ctx->profile = enable != 0;
  return BS_OK;
}

extern "C" int bs_stage_times(bs_ctx* ctx, float* ms, int n) {
  if (!ctx || !ms || n < 1) return BS_ERR_ARG;
  if (!ctx->profile || !ctx->prof_ev[0]) return ctx_fail(ctx, BS_ERR_ARG, "profiling is off");
  if (cudaEventSynchronize(ctx->prof_ev[kProfEvents - 1]) != cudaSuccess)
    return ctx_fail(ctx, BS_ERR_CUDA, "event sync");
  for (int i = 0; i < n && i < kProfEvents - 1; ++i) {
    float t = 0;
    if (ctx->prof_rec[i] && ctx->prof_rec[i + 1])
      cudaEventElapsedTime(&t, ctx->prof_ev[i], ctx->prof_ev[i + 1]);
    ms[i] = t;
  }
  return BS_OK;
}
