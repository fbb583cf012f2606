// Resultant with device-resident buffers that allocates no device memory.
//
// Same computation and launches as bs_resultant_device, but every scratch buffer of the
// call (job descriptor, stage offsets, prime flags, evaluations, values, residues,
// selected primes) is carved out of one static device array compiled into the library.
#include <cuda_runtime.h>

#include <cstring>
#include <mutex>

#include "ctx.cuh"

namespace bs {
namespace {

// 32 MiB of scratch, resident on every GPU that loads the library until the process
// exits.  Device code could name it directly; host code uses the address returned by
// cudaGetSymbolAddress, looked up once per device below.
constexpr size_t kNoAllocScratchBytes = size_t(32) << 20;
__device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_scratch_mu;
void* g_scratch_addr[kMaxDevices] = {nullptr};

// device address of the static scratch array on the current device (set-up on the first
// call per device; the caller has made ctx->device current).  The address is kept for the
// life of the process: a device reset that rebuilds the primary context is not supported.
int scratch_address(int device, void** out) {
  if (device < 0 || device >= kMaxDevices) return kErrArg;
  std::lock_guard<std::mutex> lk(g_scratch_mu);
  if (!g_scratch_addr[device]) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) {
      cudaGetLastError();
      return kErrCuda;
    }
    g_scratch_addr[device] = p;
  }
  *out = g_scratch_addr[device];
  return 0;
}

}  // namespace
}  // namespace bs

using namespace bs;

extern "C" int bs_resultant_device_noalloc(bs_ctx* ctx, const bs_bipoly* f, const bs_bipoly* g,
                                           int var, bs_upoly* out) {
  if (!ctx) return BS_ERR_ARG;
  if (!out || !out->c || (var != 0 && var != 1) || !f || !g)
    return ctx_fail(ctx, BS_ERR_ARG, "bad arguments");
  for (const bs_bipoly* p : {f, g})
    if (p->deg_x < 0 || p->deg_y < 0 || p->limbs < 1 || p->limbs > kMaxLimbs || !p->c)
      return ctx_fail(ctx, BS_ERR_ARG, "bad extents, limbs or pointer");
  if (ctx->server) return ctx_fail(ctx, BS_ERR_ARG, "the context runs a serving loop");
  if (cudaSetDevice(ctx->device) != cudaSuccess) return ctx_fail(ctx, BS_ERR_CUDA, "set device");
  // size bounds from the extents, exactly as the allocating device entry point
  int32_t dcap = 0, lcap = 0;
  int rc = bs_resultant_bounds(f, g, var, &dcap, &lcap);
  if (rc) return ctx_fail(ctx, rc, "problem exceeds the supported range");
  if (out->deg < dcap || out->limbs < lcap)
    return ctx_fail(ctx, BS_ERR_CAPACITY, "output capacity below bs_resultant_bounds()");
  // the workspace bounds of the allocating device entry point, from the same function
  MetaBounds mb;
  rc = meta_bounds(f, g, var, &mb);
  if (rc) return ctx_fail(ctx, rc, "problem exceeds the supported range");
  const int cls = uni_class_of(mb.len);
  if (cls < 0) return ctx_fail(ctx, BS_ERR_RANGE, "degree in the eliminated variable above 64");
  // this call never grows the context's tables
  if (ctx->tabs->Tt < mb.k_total || ctx->tabs->Tg < mb.k_total || ctx->tabs->logNT < mb.logN)
    return ctx_fail(ctx, BS_ERR_RANGE,
                    "the context's prime tables do not cover this size yet; make one "
                    "allocating resultant call of this size on the context first");
  const int N = 1 << mb.logN;
  Layout lay;
  const size_t o_job = lay.take(sizeof(Job));
  const size_t o_offs = lay.take(sizeof(int64_t) * kNumOffs);
  const size_t o_pstat = lay.take(sizeof(int32_t) * mb.k_total);
  const size_t o_ev = lay.take(sizeof(uint32_t) * (size_t)mb.k_total * mb.rows * N);
  const size_t o_vals = lay.take(sizeof(uint32_t) * (size_t)mb.k_total * N);
  const size_t o_rmod = lay.take(sizeof(uint32_t) * (size_t)mb.k_need * (mb.D + 1));
  const size_t o_sel = lay.take(sizeof(int32_t) * mb.k_need);
  if (lay.used > kNoAllocScratchBytes)
    return ctx_fail(ctx, BS_ERR_RANGE,
                    "problem needs " + std::to_string(lay.used) +
                        " bytes of scratch; the static scratch array holds 33554432 bytes");
  void* scratch = nullptr;
  rc = scratch_address(ctx->device, &scratch);
  if (rc) {
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(ctx->stream, &cs) == cudaSuccess && cs != cudaStreamCaptureStatusNone)
      return ctx_fail(ctx, rc, "the first call on a device looks up the static scratch; make it "
                               "before the stream capture begins");
    cudaGetLastError();
    return ctx_fail(ctx, rc, "cudaGetSymbolAddress of the static scratch failed");
  }
  char* base = (char*)scratch;
  Job J;
  std::memset(&J, 0, sizeof(J));
  J.f = Grid{f->c, f->deg_x, f->deg_y, f->limbs};
  J.g = Grid{g->c, g->deg_x, g->deg_y, g->limbs};
  J.var = var;
  J.ev = (uint32_t*)(base + o_ev);
  J.vals = (uint32_t*)(base + o_vals);
  J.rmod = (uint32_t*)(base + o_rmod);
  J.pstat = (int32_t*)(base + o_pstat);  // zeroed on the stream before use
  J.sel = (int32_t*)(base + o_sel);
  J.out = out->c;
  J.cap_deg = out->deg;
  J.cap_limbs = out->limbs;
  J.status = ctx->d_status;
  J.rejected = ctx->d_status + 1;
  J.cap_k_total = mb.k_total;
  J.cap_k_need = mb.k_need;
  J.cap_rows = mb.rows;
  J.cap_logN = mb.logN;
  J.cap_D = mb.D;
  rc = launch_device_job(ctx, J, (Job*)(base + o_job), (int64_t*)(base + o_offs), mb, cls);
  if (rc) return rc;
  ctx->stats = bs_stats{};
  ctx->stats.jobs = 1;
  return BS_OK;
}
