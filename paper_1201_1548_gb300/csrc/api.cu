// C ABI of libbsres: context, workspace management and the resultant entry points.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/bsres.h"
#include "batch.cuh"
#include "host_parallel.h"
#include "common.cuh"
#include "ctx.cuh"
#include "resultant_kernels.cuh"
#include "tables.cuh"

using namespace bs;

// ------------------------------------------------------------------------------------
// context
// ------------------------------------------------------------------------------------
int ctx_fail(bs_ctx* ctx, int code, const std::string& msg) {
  if (ctx) ctx->err = msg;
  return code;
}

std::string device_failure_detail(const int32_t* st) {
  std::string m = "device stage reported a failure";
  if (st[2]) m += " (debug bounds check failed at site " + std::to_string(st[2]) + ")";
  return m;
}

int ctx_cuda(bs_ctx* ctx, cudaError_t e, const char* what) {
  if (e == cudaSuccess) return 0;
  return ctx_fail(ctx, BS_ERR_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

int ensure_workspace(bs_ctx* ctx, size_t bytes) {
  if (bytes <= ctx->ws_cap) return 0;
  if (bytes > ctx->budget) return ctx_fail(ctx, BS_ERR_NOMEM, "workspace exceeds the memory budget");
  if (ctx->ws) {
    cudaStreamSynchronize(ctx->stream);
    cudaFree(ctx->ws);
    ctx->ws = nullptr;
    ctx->ws_cap = 0;
  }
  size_t cap = std::min(ctx->budget, bytes + bytes / 4);
  if (cudaMalloc(&ctx->ws, cap) != cudaSuccess) {
    cudaGetLastError();
    ctx->ws = nullptr;
    return ctx_fail(ctx, BS_ERR_NOMEM, "cudaMalloc of the workspace failed");
  }
  ctx->ws_cap = cap;
  ++ctx->ws_generation;
  return 0;
}

// Pinned staging grows geometrically: freeing and allocating pinned memory waits for the
// whole device, so a growth step costs as long as the longest work in flight.
int ensure_pinned(bs_ctx* ctx, size_t up, size_t down) {
  if (up > ctx->h_up_cap) {
    if (ctx->h_up) cudaFreeHost(ctx->h_up);
    ctx->h_up_cap = std::max(up + up / 4 + 4096, 2 * ctx->h_up_cap);
    if (cudaMallocHost(&ctx->h_up, ctx->h_up_cap) != cudaSuccess) {
      ctx->h_up = nullptr;
      ctx->h_up_cap = 0;
      return ctx_fail(ctx, BS_ERR_NOMEM, "pinned host allocation failed");
    }
  }
  if (down > ctx->h_down_cap) {
    if (ctx->h_down) cudaFreeHost(ctx->h_down);
    ctx->h_down_cap = std::max(down + down / 4 + 4096, 2 * ctx->h_down_cap);
    if (cudaMallocHost(&ctx->h_down, ctx->h_down_cap) != cudaSuccess) {
      ctx->h_down = nullptr;
      ctx->h_down_cap = 0;
      return ctx_fail(ctx, BS_ERR_NOMEM, "pinned host allocation failed");
    }
  }
  return 0;
}

extern "C" int bs_init(int device, size_t mem_budget, bs_ctx** out) {
  if (!out) return BS_ERR_ARG;
  *out = nullptr;
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev == 0) {
    cudaGetLastError();
    return BS_ERR_CUDA;
  }
  if (device < 0 || device >= ndev) return BS_ERR_ARG;
  if (cudaSetDevice(device) != cudaSuccess) return BS_ERR_CUDA;
  bs_ctx* ctx = new bs_ctx();
  ctx->device = device;
  cudaDeviceProp prop;
  cudaGetDeviceProperties(&prop, device);
  ctx->sms = prop.multiProcessorCount;
  ctx->smem_optin = (int)prop.sharedMemPerBlockOptin;
  size_t freeb = 0, totalb = 0;
  cudaMemGetInfo(&freeb, &totalb);
  ctx->budget = mem_budget ? mem_budget : (size_t)(freeb * 0.9);
  if (cudaStreamCreateWithFlags(&ctx->own_stream, cudaStreamNonBlocking) != cudaSuccess) {
    delete ctx;
    return BS_ERR_CUDA;
  }
  ctx->stream = ctx->own_stream;
  int rc = ctx->tabs->init(ctx->stream);
  if (rc) {
    bs_free(ctx);
    return rc;
  }
  if (cudaMalloc(&ctx->d_status, sizeof(int32_t) * 4) != cudaSuccess) {
    bs_free(ctx);
    return BS_ERR_CUDA;
  }
  cudaMemset(ctx->d_status, 0, sizeof(int32_t) * 4);
  for (int c = 0; c < kNumUniClasses; ++c)
    for (int t = 0; t < 3; ++t) ctx->occ[c][t] = uni_occupancy(c, kUniThreadChoices[t]);
  if (set_stage_smem_limits(ctx->smem_optin) != 0) {
    cudaGetLastError();
    bs_free(ctx);
    return BS_ERR_CUDA;
  }
  if (cudaDeviceSynchronize() != cudaSuccess) {
    bs_free(ctx);
    return BS_ERR_CUDA;
  }
  *out = ctx;
  return BS_OK;
}

extern "C" void bs_free(bs_ctx* ctx) {
  if (!ctx) return;
  if (ctx->server) bs_serve_stop(ctx);
  cudaSetDevice(ctx->device);
  if (ctx->own_stream) cudaStreamSynchronize(ctx->own_stream);
  if (ctx->stream && ctx->stream != ctx->own_stream) cudaStreamSynchronize(ctx->stream);
  if (ctx->aux_stream) cudaStreamSynchronize(ctx->aux_stream);
  ctx->own_tabs.release();  // serving slots borrow their parent's tables
  if (ctx->ws) cudaFree(ctx->ws);
  if (ctx->dev_ws) cudaFree(ctx->dev_ws);
  if (ctx->d_status) cudaFree(ctx->d_status);
  if (ctx->h_up) cudaFreeHost(ctx->h_up);
  if (ctx->h_down) cudaFreeHost(ctx->h_down);
  ctx_release_extra(ctx);
  if (ctx->own_stream) cudaStreamDestroy(ctx->own_stream);
  if (ctx->aux_stream) cudaStreamDestroy(ctx->aux_stream);
  delete ctx;
}

extern "C" int bs_set_stream(bs_ctx* ctx, void* stream) {
  if (!ctx) return BS_ERR_ARG;
  cudaStreamSynchronize(ctx->stream);
  ctx->stream = stream ? (cudaStream_t)stream : ctx->own_stream;
  return BS_OK;
}

extern "C" const char* bs_error_string(int status) {
  switch (status) {
    case BS_OK: return "ok";
    case BS_ERR_ARG: return "invalid argument";
    case BS_ERR_NOMEM: return "device memory budget exceeded";
    case BS_ERR_UNLUCKY: return "too many unlucky primes";
    case BS_ERR_TIMEOUT: return "bounded device wait expired";
    case BS_ERR_CUDA: return "CUDA runtime error";
    case BS_ERR_ZERO: return "square-free part of the zero polynomial";
    case BS_ERR_RANGE: return "problem exceeds the prime table or transform size";
    case BS_ERR_INTERNAL: return "device-side consistency check failed";
    case BS_ERR_CAPACITY: return "output capacity too small";
    default: return "unknown status";
  }
}

extern "C" const char* bs_last_error_detail(const bs_ctx* ctx) {
  return ctx ? ctx->err.c_str() : "no context";
}

extern "C" int bs_last_stats(const bs_ctx* ctx, bs_stats* out) {
  if (!ctx || !out) return BS_ERR_ARG;
  *out = ctx->stats;
  return BS_OK;
}

extern "C" int bs_prime_table(int count, uint32_t* primes) {
  const HostPrimes& H = host_primes();
  if (count < 0 || count > (int)H.p.size() || (!primes && count)) return BS_ERR_ARG;
  for (int i = 0; i < count; ++i) primes[i] = H.p[i];
  return BS_OK;
}

// ------------------------------------------------------------------------------------
// shared helpers
// ------------------------------------------------------------------------------------
static int check_bipoly(bs_ctx* ctx, const bs_bipoly* p, const char* name) {
  if (!p) return ctx_fail(ctx, BS_ERR_ARG, std::string(name) + " is null");
  if (p->deg_x < 0 || p->deg_y < 0 || p->limbs < 1 || p->limbs > kMaxLimbs || !p->c)
    return ctx_fail(ctx, BS_ERR_ARG, std::string(name) + ": bad extents, limbs or pointer");
  return 0;
}

static Grid grid_of(const bs_bipoly* p) { return Grid{p->c, p->deg_x, p->deg_y, p->limbs}; }

// upper bounds from extents and limb counts only
int bs::meta_bounds(const bs_bipoly* f, const bs_bipoly* g, int var, MetaBounds* mb) {
  const int fe = var ? f->deg_y : f->deg_x, fo = var ? f->deg_x : f->deg_y;
  const int ge = var ? g->deg_y : g->deg_x, go = var ? g->deg_x : g->deg_y;
  const int64_t d1 = (int64_t)(f->deg_x + f->deg_y) * (g->deg_x + g->deg_y);
  const int64_t d2 = (int64_t)ge * fo + (int64_t)fe * go;
  int64_t D = std::min(d1, d2);
  if (D < 0) D = 0;
  mb->D = (int32_t)D;
  if (D + 1 > kNMax) return BS_ERR_RANGE;
  int logN = 0;
  while ((1ll << logN) < D + 1) ++logN;
  mb->logN = logN;
  mb->rows = (fe + 1) + (ge + 1);
  mb->len = std::max(fe, ge) + 1;
  // coefficient magnitudes below 2^(32 L - 1)
  auto Sbound = [&](int rows, int cols, int L) {
    UF c = uf_make(1, 32 * L - 1, false);
    UF l1 = uf_mul(uf_make((uint64_t)cols, 0, false), c);
    return uf_mul(uf_make((uint64_t)rows, 0, false), uf_mul(l1, l1));
  };
  const UF Sf = Sbound(fe + 1, fo + 1, f->limbs);
  const UF Sg = Sbound(ge + 1, go + 1, g->limbs);
  const HostPrimes& H = host_primes();
  Plan P = finish_plan(Sf, fe, f->deg_x + f->deg_y, fo, 32 * f->limbs, Sg, ge, g->deg_x + g->deg_y,
                       go, 32 * g->limbs, H.lg_prefix.data(), (int)H.p.size());
  if (P.status) return P.status;
  mb->k_total = std::max(P.k_total, 1);
  mb->k_need = std::max(P.k_need, 1);
  mb->out_limbs = P.out_limbs;
  return 0;
}

extern "C" int bs_plan(const bs_bipoly* f, const bs_bipoly* g, int var, bs_plan_info* out) {
  if (!out || (var != 0 && var != 1)) return BS_ERR_ARG;
  if (check_bipoly(nullptr, f, "f") || check_bipoly(nullptr, g, "g")) return BS_ERR_ARG;
  const HostPrimes& H = host_primes();
  const Plan P = plan_host(grid_of(f), grid_of(g), var, H.lg_prefix.data(), (int)H.p.size(),
                          H.p.data());
  out->trivial = P.trivial;
  out->m_e = P.me;
  out->n_e = P.ne;
  out->D = P.trivial == 1 ? -1 : P.D;
  out->N = P.N;
  out->k_need = P.k_need;
  out->k_total = P.k_total;
  out->out_limbs = P.out_limbs;
  out->log2B_q16 = P.log2B_q16;
  return P.status;
}

extern "C" int bs_resultant_bounds(const bs_bipoly* f, const bs_bipoly* g, int var,
                                   int32_t* deg_cap, int32_t* limbs_cap) {
  if (!f || !g || !deg_cap || !limbs_cap || (var != 0 && var != 1)) return BS_ERR_ARG;
  if (f->deg_x < 0 || f->deg_y < 0 || g->deg_x < 0 || g->deg_y < 0 || f->limbs < 1 ||
      g->limbs < 1 || f->limbs > kMaxLimbs || g->limbs > kMaxLimbs)
    return BS_ERR_ARG;
  MetaBounds mb;
  int rc = meta_bounds(f, g, var, &mb);
  if (rc) return rc;
  *deg_cap = mb.D;
  *limbs_cap = mb.out_limbs;
  return BS_OK;
}

// copy one result coefficient block (rows of src_limbs two's complement limbs) into a
// caller buffer of dst_limbs, checking that each value fits
static bool copy_coeffs(const uint32_t* src, int src_limbs, int ncoef, uint32_t* dst, int dst_limbs) {
  if (src_limbs == dst_limbs) {  // same width: one copy
    std::memcpy(dst, src, sizeof(uint32_t) * (size_t)ncoef * src_limbs);
    return true;
  }
  for (int i = 0; i < ncoef; ++i) {
    const uint32_t* s = src + (size_t)i * src_limbs;
    uint32_t* d = dst + (size_t)i * dst_limbs;
    const uint32_t ext = (s[src_limbs - 1] >> 31) ? 0xffffffffu : 0u;
    for (int l = 0; l < dst_limbs; ++l) d[l] = l < src_limbs ? s[l] : ext;
    // the dropped limbs must be pure sign extension of the kept ones
    const uint32_t kept_ext = (d[dst_limbs - 1] >> 31) ? 0xffffffffu : 0u;
    for (int l = dst_limbs; l < src_limbs; ++l)
      if (s[l] != kept_ext) return false;
  }
  return true;
}

static bool coeff_is_zero(const uint32_t* s, int limbs) {
  for (int l = 0; l < limbs; ++l)
    if (s[l]) return false;
  return true;
}

// ------------------------------------------------------------------------------------
// batch of host-resident jobs (also serves bs_resultant with n = 1)
// ------------------------------------------------------------------------------------
namespace bs {

int batch_plan(bs_ctx* ctx, int n, const bs_bipoly* f, const bs_bipoly* g, int var, HostBatch* hb) {
  HostBatch& B = *hb;
  B = HostBatch{};
  B.n = n;
  B.var = var;
  const HostPrimes& H = host_primes();
  const int T = (int)H.p.size();
  B.plans.resize(n);
  for (int i = 0; i < n; ++i) {
    int rc = check_bipoly(ctx, f + i, "f");
    if (rc) return rc;
    rc = check_bipoly(ctx, g + i, "g");
    if (rc) return rc;
  }
  // plans are independent: large batches plan on several host threads
  parallel_for(n, 256, [&](int i) {
    B.plans[i] = plan_host(grid_of(f + i), grid_of(g + i), var, H.lg_prefix.data(), T, H.p.data());
  });
  for (int i = 0; i < n; ++i)
    if (B.plans[i].status)
      return ctx_fail(ctx, B.plans[i].status, "planning failed for job " + std::to_string(i));
  B.big.assign(n, 0);
  for (int i = 0; i < n; ++i) {
    const Plan& P = B.plans[i];
    if (P.trivial) continue;
    B.needT = std::max(B.needT, P.k_total);
    B.needLog = std::max(B.needLog, P.logN);
    if (P.k_need > kCrtWarpMaxK) {  // weighted sums of many primes, Garner for rejections
      B.big[i] = 1;
      B.kmax_big = std::max(B.kmax_big, P.k_need);
      B.lmax_big = std::max(B.lmax_big, P.out_limbs + 1);
    } else {
      B.kmax = std::max(B.kmax, P.k_need);
      B.lmax = std::max(B.lmax, P.out_limbs + 1);
    }
    B.maxN = std::max(B.maxN, P.N);
    const int c = uni_class_of(std::max(P.me, P.ne) + 1);
    if (c < 0) return ctx_fail(ctx, BS_ERR_RANGE, "degree in the eliminated variable above 64");
    ++B.cls_count[c];
    if (P.logN <= kWarpLogNMax) ++B.ecls_count[eval_class_of(P.logN)];
  }
  {  // the block Garner kernel serves jobs of many primes with rejected primes
    const size_t need = ((size_t)B.kmax_big * kCrtTile + 3 * (size_t)B.kmax_big + 3 * (size_t)B.lmax_big) *
                        sizeof(uint32_t);
    if (need + 64 > (size_t)ctx->smem_optin)
      return ctx_fail(ctx, BS_ERR_RANGE, "too many primes for the reconstruction stage");
  }
  B.in_f.resize(n);
  B.in_g.resize(n);
  size_t in_words = 0, pstat_words = 0;
  for (int i = 0; i < n; ++i) {
    B.in_f[i] = (int64_t)(f[i].deg_y + 1) * (f[i].deg_x + 1) * f[i].limbs;
    B.in_g[i] = (int64_t)(g[i].deg_y + 1) * (g[i].deg_x + 1) * g[i].limbs;
    in_words += B.in_f[i] + B.in_g[i];
    if (!B.plans[i].trivial) pstat_words += B.plans[i].k_total;
  }
  Layout up;
  B.o_jobs = up.take(sizeof(Job) * n);
  B.o_eoff = up.take(sizeof(int64_t) * (n + 1));
  B.o_ioff = up.take(sizeof(int64_t) * (n + 1));
  B.o_iwoff = up.take(sizeof(int64_t) * (n + 1));
  B.o_coff = up.take(sizeof(int64_t) * (n + 1));
  B.o_cbt = up.take(sizeof(int64_t) * (n + 1));
  B.o_cbg = up.take(sizeof(int64_t) * (n + 1));
  B.o_cbc = up.take(sizeof(int64_t) * (n + 1));
  B.o_cbf = up.take(sizeof(int64_t) * (n + 1));
  for (int c = 0; c < kNumUniClasses; ++c) {
    B.o_cids[c] = up.take(sizeof(int32_t) * std::max(B.cls_count[c], 1));
    B.o_coffs[c] = up.take(sizeof(int64_t) * (B.cls_count[c] + 1));
  }
  for (int c = 0; c < kNumEvalClasses; ++c) {
    B.o_eids[c] = up.take(sizeof(int32_t) * std::max(B.ecls_count[c], 1));
    B.o_eoffs[c] = up.take(sizeof(int64_t) * (B.ecls_count[c] + 1));
  }
  B.o_status = up.take(sizeof(int32_t) * 4);
  B.o_pstat = up.take(sizeof(int32_t) * std::max<size_t>(pstat_words, 1));
  B.o_in = up.take(sizeof(uint32_t) * std::max<size_t>(in_words, 1));
  B.up_bytes = up.used;
  Layout cmp;
  cmp.used = B.up_bytes;
  B.o_ev.assign(n, 0);
  B.o_vals.assign(n, 0);
  B.o_rmod.assign(n, 0);
  B.o_sel.assign(n, 0);
  B.o_wsM.assign(n, 0);
  B.o_wsY.assign(n, 0);
  B.o_wsS.assign(n, 0);
  for (int i = 0; i < n; ++i) {
    const Plan& P = B.plans[i];
    if (P.trivial) continue;
    const int rows = (P.me + 1) + (P.ne + 1);
    B.o_ev[i] = cmp.take(sizeof(uint32_t) * (size_t)P.k_total * rows * P.N);
    B.o_vals[i] = cmp.take(sizeof(uint32_t) * (size_t)P.k_total * P.N);
    B.o_rmod[i] = cmp.take(sizeof(uint32_t) * (size_t)P.k_need * (P.D + 1));
    B.o_sel[i] = cmp.take(sizeof(int32_t) * P.k_need);
    if (B.big[i]) {
      const size_t wl = (size_t)big_ws_len(P.k_need);
      B.o_wsM[i] = cmp.take(sizeof(uint32_t) * (size_t)P.k_need * wl);
      B.o_wsY[i] = cmp.take(sizeof(uint32_t) * (size_t)P.k_need);
      B.o_wsS[i] = cmp.take(sizeof(uint32_t) * 3 * (size_t)(std::max(P.D, 0) + 1) * wl);
    }
  }
  Layout dn;
  dn.used = cmp.used;
  B.dn_start = dn.take(0);
  B.o_out.assign(n, 0);
  for (int i = 0; i < n; ++i) {
    const Plan& P = B.plans[i];
    const int cap_deg = std::max(P.D, 0);
    B.o_out[i] = dn.take(sizeof(uint32_t) * (size_t)(cap_deg + 1) * P.out_limbs);
  }
  B.o_status_dn = dn.take(sizeof(int32_t) * 4);
  B.total = dn.used;
  B.dn_bytes = B.total - B.dn_start;
  return 0;
}

int batch_launch(bs_ctx* ctx, HostBatch& B, const bs_bipoly* f, const bs_bipoly* g, char* base,
                 char* hu, char* hd, bool use_graph) {
  const int n = B.n;
  std::memset(hu, 0, B.up_bytes);
  {  // staged inputs
    uint32_t* dst = (uint32_t*)(hu + B.o_in);
    for (int i = 0; i < n; ++i) {
      std::memcpy(dst, f[i].c, sizeof(uint32_t) * B.in_f[i]);
      dst += B.in_f[i];
      std::memcpy(dst, g[i].c, sizeof(uint32_t) * B.in_g[i]);
      dst += B.in_g[i];
    }
  }
  Job* hj = (Job*)(hu + B.o_jobs);
  int64_t* eoff = (int64_t*)(hu + B.o_eoff);
  int64_t* ioff = (int64_t*)(hu + B.o_ioff);
  int64_t* iwoff = (int64_t*)(hu + B.o_iwoff);
  int64_t* coff = (int64_t*)(hu + B.o_coff);
  int64_t* cbt = (int64_t*)(hu + B.o_cbt);
  int64_t* cbg = (int64_t*)(hu + B.o_cbg);
  int64_t* cbc = (int64_t*)(hu + B.o_cbc);
  int64_t* cbf = (int64_t*)(hu + B.o_cbf);
  cbt[0] = cbg[0] = cbc[0] = cbf[0] = 0;
  int32_t* cids[kNumUniClasses];
  int64_t* coffs[kNumUniClasses];
  int cfill[kNumUniClasses] = {0};
  for (int c = 0; c < kNumUniClasses; ++c) {
    cids[c] = (int32_t*)(hu + B.o_cids[c]);
    coffs[c] = (int64_t*)(hu + B.o_coffs[c]);
    coffs[c][0] = 0;
  }
  int32_t* eids[kNumEvalClasses];
  int64_t* eoffs[kNumEvalClasses];
  int efill[kNumEvalClasses] = {0};
  for (int c = 0; c < kNumEvalClasses; ++c) {
    eids[c] = (int32_t*)(hu + B.o_eids[c]);
    eoffs[c] = (int64_t*)(hu + B.o_eoffs[c]);
    eoffs[c][0] = 0;
  }
  eoff[0] = ioff[0] = iwoff[0] = coff[0] = 0;
  size_t in_pos = 0, ps_pos = 0;
  const int crt_tile = crt_warp_kernel(ctx, B.kmax, B.lmax) ? ctx->tune.crt_tile : kCrtTile;
  B.instances = B.mulmods = B.k_need_sum = B.k_total_sum = 0;
  B.maxpts = B.maxprimes = 0;
  for (int i = 0; i < n; ++i) {
    const Plan& P = B.plans[i];
    Job J;
    std::memset(&J, 0, sizeof(J));
    J.f = Grid{(const uint32_t*)(base + B.o_in) + in_pos, f[i].deg_x, f[i].deg_y, f[i].limbs};
    in_pos += B.in_f[i];
    J.g = Grid{(const uint32_t*)(base + B.o_in) + in_pos, g[i].deg_x, g[i].deg_y, g[i].limbs};
    in_pos += B.in_g[i];
    J.var = B.var;
    J.plan = P;
    J.cap_deg = std::max(P.D, 0);
    J.cap_limbs = P.out_limbs;
    J.out = (uint32_t*)(base + B.o_out[i]);
    J.status = (int32_t*)(base + B.o_status);
    J.rejected = (int32_t*)(base + B.o_status) + 1;
    int64_t ne = 0, ni = 0, niw = 0, nu = 0;
    if (!P.trivial) {
      J.rows = (P.me + 1) + (P.ne + 1);
      J.ev = (uint32_t*)(base + B.o_ev[i]);
      J.vals = (uint32_t*)(base + B.o_vals[i]);
      J.den_in_ev = P.logN <= kWarpInttLogNMax;  // interpolated one warp per prime
      J.rmod = (uint32_t*)(base + B.o_rmod[i]);
      J.sel = (int32_t*)(base + B.o_sel[i]);
      J.pstat = (int32_t*)(base + B.o_pstat) + ps_pos;
      ps_pos += P.k_total;
      if (P.logN <= kWarpLogNMax) {
        const int ec = eval_class_of(P.logN);
        eids[ec][efill[ec]] = i;
        const int ew = ctx->tune.eval_independent ? 1 : ctx->tune.eval_warps;  // rows per item
        eoffs[ec][efill[ec] + 1] = eoffs[ec][efill[ec]] + (int64_t)P.k_total * ((J.rows + ew - 1) / ew);
        ++efill[ec];
      } else {
        ne = (int64_t)P.k_total * J.rows;
      }
      // interpolation: one warp per prime up to 2^kWarpLogNMax points, else one block
      if (P.logN <= kWarpInttLogNMax)
        niw = P.k_total;
      else
        ni = P.k_total;
      nu = (int64_t)P.k_total << P.logN;  // instances
      const int c = uni_class_of(std::max(P.me, P.ne) + 1);
      cids[c][cfill[c]] = i;
      coffs[c][cfill[c] + 1] = coffs[c][cfill[c]] + nu;
      ++cfill[c];
      B.instances += (int64_t)P.k_total << P.logN;
      B.mulmods += ((int64_t)P.k_total << P.logN) * (int64_t)P.me * P.ne;
      B.k_need_sum += P.k_need;
      B.k_total_sum += P.k_total;
      B.maxpts = std::max(B.maxpts, P.N);
      B.maxprimes = std::max(B.maxprimes, P.k_total);
    }
    hj[i] = J;
    eoff[i + 1] = eoff[i] + ne;
    ioff[i + 1] = ioff[i] + ni;
    iwoff[i + 1] = iwoff[i] + niw;
    int64_t nbt = 0, nbg = 0, nbc = 0, nbf = 0;
    if (B.big[i]) {
      const int wl = big_ws_len(P.k_need);
      J.wsM = (uint32_t*)(base + B.o_wsM[i]);
      J.wsY = (uint32_t*)(base + B.o_wsY[i]);
      J.wsS = (uint32_t*)(base + B.o_wsS[i]);
      J.wsL = wl;
      nbt = (P.k_need + kBigTabThreads - 1) / kBigTabThreads;
      nbg = (int64_t)((J.cap_deg + kBigGI) / kBigGI) * ((wl + kBigGL - 1) / kBigGL);
      nbc = (J.cap_deg + kBigCarryWarps) / kBigCarryWarps;
      nbf = (J.cap_deg + kCrtTile) / kCrtTile;
      hj[i] = J;
    }
    cbt[i + 1] = cbt[i] + nbt;
    cbg[i + 1] = cbg[i] + nbg;
    cbc[i + 1] = cbc[i] + nbc;
    cbf[i + 1] = cbf[i] + nbf;
    coff[i + 1] = coff[i] + (B.big[i] ? 0 : (J.cap_deg + crt_tile) / crt_tile);
  }
  cudaStream_t s = ctx->stream;
  int rc = ctx_cuda(ctx, cudaMemcpyAsync(base, hu, B.up_bytes, cudaMemcpyHostToDevice, s), "upload");
  if (rc) return rc;
  // ---- device stages
  const Tables Tv = ctx->tabs->view();
  StageLaunch L;
  L.jobs = (const Job*)(base + B.o_jobs);
  L.eval = WorkList{nullptr, (const int64_t*)(base + B.o_eoff), n};
  L.intt = WorkList{nullptr, (const int64_t*)(base + B.o_ioff), n};
  L.intt_w = WorkList{nullptr, (const int64_t*)(base + B.o_iwoff), n};
  L.crt = WorkList{nullptr, (const int64_t*)(base + B.o_coff), n};
  L.crt_big_tab = WorkList{nullptr, (const int64_t*)(base + B.o_cbt), n};
  L.crt_big_gemm = WorkList{nullptr, (const int64_t*)(base + B.o_cbg), n};
  L.crt_big_carry = WorkList{nullptr, (const int64_t*)(base + B.o_cbc), n};
  L.crt_big_fb = WorkList{nullptr, (const int64_t*)(base + B.o_cbf), n};
  L.crt_big_items[0] = cbt[n];
  L.crt_big_items[1] = cbg[n];
  L.crt_big_items[2] = cbc[n];
  L.crt_big_items[3] = cbf[n];
  L.kmax_big = B.kmax_big;
  L.lmax_big = B.lmax_big;
  for (int c = 0; c < kNumUniClasses; ++c) {
    L.uni[c] = WorkList{(const int32_t*)(base + B.o_cids[c]), (const int64_t*)(base + B.o_coffs[c]),
                        B.cls_count[c]};
    L.uni_items[c] = B.cls_count[c] ? coffs[c][B.cls_count[c]] : 0;
  }
  for (int c = 0; c < kNumEvalClasses; ++c) {
    L.evw[c] = WorkList{(const int32_t*)(base + B.o_eids[c]), (const int64_t*)(base + B.o_eoffs[c]),
                        B.ecls_count[c]};
    L.evw_items[c] = B.ecls_count[c] ? eoffs[c][B.ecls_count[c]] : 0;
  }
  L.evw_any_items = 0;
  L.eval_items = eoff[n];
  L.intt_items = ioff[n];
  L.intt_w_items = iwoff[n];
  L.crt_items = coff[n];
  L.maxN = B.maxN;
  L.kmax = B.kmax;
  L.lmax = B.lmax;
  L.kt_max = B.needT;
  L.logN_max = B.needLog;
  L.eval_warps = ctx->tune.eval_warps;
  L.eval_blocks_per_sm = ctx->tune.eval_blocks_per_sm;
  L.eval_independent = ctx->tune.eval_independent != 0;
  L.crt_tile = crt_tile;
  L.crt_blocks_per_sm = ctx->tune.crt_blocks_per_sm;
  for (int c = 0; c < kNumUniClasses; ++c) L.uni_threads[c] = ctx->tune.uni_threads[c];
  L.pdl = true;
  rc = launch_stages(ctx, L, Tv, use_graph);
  if (rc) return rc;
  rc = ctx_cuda(ctx, cudaMemcpyAsync(base + B.o_status_dn, base + B.o_status, sizeof(int32_t) * 4,
                                     cudaMemcpyDeviceToDevice, s),
                "status copy");
  if (rc) return rc;
  return ctx_cuda(ctx, cudaMemcpyAsync(hd, base + B.dn_start, B.dn_bytes, cudaMemcpyDeviceToHost, s),
                  "download");
}

int batch_finish(bs_ctx* ctx, const HostBatch& B, const char* hd, bs_upoly* out) {
  const int32_t* st = (const int32_t*)(hd + (B.o_status_dn - B.dn_start));
  ctx->stats = bs_stats{};
  ctx->stats.jobs = B.n;
  ctx->stats.primes_needed = B.k_need_sum;
  ctx->stats.primes_evaluated = B.k_total_sum;
  ctx->stats.primes_rejected = st[1];
  ctx->stats.instances = B.instances;
  ctx->stats.mulmods_alg = B.mulmods;
  ctx->stats.max_points = B.maxpts;
  ctx->stats.max_primes = B.maxprimes;
  if (st[0]) return ctx_fail(ctx, st[0], device_failure_detail(st));
  // results are independent: large batches are formatted on several host threads
  std::vector<int> err(B.n, 0);
  parallel_for(B.n, 256, [&](int i) {
    const Plan& P = B.plans[i];
    const uint32_t* src = (const uint32_t*)(hd + (B.o_out[i] - B.dn_start));
    const int ncoef = std::max(P.D, 0) + 1;
    int deg = -1;
    for (int c = ncoef - 1; c >= 0; --c)
      if (!coeff_is_zero(src + (size_t)c * P.out_limbs, P.out_limbs)) {
        deg = c;
        break;
      }
    if (deg > out[i].deg) {
      err[i] = 1;
      return;
    }
    const int cap = out[i].deg;
    if (deg >= 0 && !copy_coeffs(src, P.out_limbs, deg + 1, out[i].c, out[i].limbs)) {
      err[i] = 2;
      return;
    }
    for (int c = deg + 1; c <= cap; ++c)
      std::memset(out[i].c + (size_t)c * out[i].limbs, 0, sizeof(uint32_t) * out[i].limbs);
    out[i].deg = deg;
  });
  for (int i = 0; i < B.n; ++i) {
    if (err[i] == 1) return ctx_fail(ctx, BS_ERR_CAPACITY, "output degree capacity too small");
    if (err[i] == 2) return ctx_fail(ctx, BS_ERR_CAPACITY, "output limb capacity too small");
  }
  return BS_OK;
}

}  // namespace bs

int run_host_batch(bs_ctx* ctx, int n, const bs_bipoly* f, const bs_bipoly* g, int var,
                   bs_upoly* out, bool use_graph) {
  if (!ctx || n < 0 || !out || (n && (!f || !g)) || (var != 0 && var != 1))
    return ctx_fail(ctx, BS_ERR_ARG, "bad arguments");
  if (n == 0) return BS_OK;
  if (ctx->server) return ctx_fail(ctx, BS_ERR_ARG, "the context runs a serving loop");
  cudaSetDevice(ctx->device);
  HostBatch B;
  int rc = batch_plan(ctx, n, f, g, var, &B);
  if (rc) return rc;
  bool query = false;
  for (int i = 0; i < n; ++i)
    if (!out[i].c) query = true;
  if (query) {
    for (int i = 0; i < n; ++i) {
      const Plan& P = B.plans[i];
      out[i].deg = P.trivial == 1 ? -1 : P.D;
      out[i].limbs = P.out_limbs;
    }
    return BS_OK;
  }
  for (int i = 0; i < n; ++i)
    if (out[i].limbs < 1 || out[i].deg < -1)
      return ctx_fail(ctx, BS_ERR_ARG, "bad output capacity");
  rc = ctx->tabs->ensure(B.needT, B.needLog, ctx->stream);
  if (rc) return ctx_fail(ctx, rc, "table setup failed");
  rc = ensure_workspace(ctx, B.total);
  if (rc) return rc;
  rc = ensure_pinned(ctx, B.up_bytes, B.dn_bytes);
  if (rc) return rc;
  rc = batch_launch(ctx, B, f, g, (char*)ctx->ws, (char*)ctx->h_up, (char*)ctx->h_down, use_graph);
  if (rc) return rc;
  rc = ctx_cuda(ctx, cudaStreamSynchronize(ctx->stream), "stream");
  if (rc) return rc;
  return batch_finish(ctx, B, (const char*)ctx->h_down, out);
}

// ------------------------------------------------------------------------------------
// autotuning of the batched launch shapes
// ------------------------------------------------------------------------------------
extern "C" int bs_autotune_batch(bs_ctx* ctx, int n, const bs_bipoly* f, const bs_bipoly* g,
                                 int var, bs_tune_info* info) {
  if (!ctx || n < 1 || !f || !g || (var != 0 && var != 1)) return ctx_fail(ctx, BS_ERR_ARG, "bad arguments");
  if (ctx->server) return ctx_fail(ctx, BS_ERR_ARG, "the context runs a serving loop");
  cudaSetDevice(ctx->device);
  HostBatch B;
  int rc = batch_plan(ctx, n, f, g, var, &B);
  if (rc) return rc;
  rc = ctx->tabs->ensure(B.needT, B.needLog, ctx->stream);
  if (rc) return ctx_fail(ctx, rc, "table setup failed");
  rc = ensure_workspace(ctx, B.total);
  if (rc) return rc;
  rc = ensure_pinned(ctx, B.up_bytes, B.dn_bytes);
  if (rc) return rc;
  const bool was_profiling = ctx->profile;
  if (!ctx->prof_ev[0])
    for (int i = 0; i < kProfEvents; ++i) cudaEventCreate(&ctx->prof_ev[i]);
  ctx->profile = true;
  int trials = 0;
  // stage times (ms) of one run with the context's current shapes: [eval, unires, intt, crt]
  auto run = [&](float* st) -> int {
    float best[4] = {1e30f, 1e30f, 1e30f, 1e30f};
    for (int rep = 0; rep < 2; ++rep) {
      int r = batch_launch(ctx, B, f, g, (char*)ctx->ws, (char*)ctx->h_up, (char*)ctx->h_down, false);
      if (r) return r;
      r = ctx_cuda(ctx, cudaStreamSynchronize(ctx->stream), "stream");
      if (r) return r;
      for (int k = 0; k < 4; ++k) {
        float ms = 0.f;
        if (ctx->prof_rec[k + 1] && ctx->prof_rec[k + 2])
          cudaEventElapsedTime(&ms, ctx->prof_ev[k + 1], ctx->prof_ev[k + 2]);
        best[k] = std::min(best[k], ms);
      }
    }
    ++trials;
    for (int k = 0; k < 4; ++k) st[k] = best[k];
    return 0;
  };
  const Tune dflt;
  ctx->tune = dflt;
  float st[4];
  rc = run(st);
  if (rc) {
    ctx->profile = was_profiling;
    return rc;
  }
  const float ms_default = st[0] + st[1] + st[2] + st[3];
  Tune best = dflt;
  // evaluation: the variant (independent warps: grid cap; staged blocks: rows per block
  // and grid cap)
  {
    float bt = st[0];
    for (int v : {1, 0})
      for (int w : {2, 4, 8})
        for (int b : {4, 8, 16}) {
          if (v == 1 && w != dflt.eval_warps) continue;  // rows per block unused there
          if (v == dflt.eval_independent && w == dflt.eval_warps && b == dflt.eval_blocks_per_sm) continue;
          ctx->tune = best;
          ctx->tune.eval_independent = v;
          ctx->tune.eval_warps = w;
          ctx->tune.eval_blocks_per_sm = b;
          if ((rc = run(st))) break;
          if (st[0] < bt) {
            bt = st[0];
            best.eval_independent = v;
            best.eval_warps = w;
            best.eval_blocks_per_sm = b;
          }
        }
  }
  // univariate resultants: threads per block, one degree class at a time
  for (int c = 0; c < kNumUniClasses && !rc; ++c) {
    if (!B.cls_count[c]) continue;
    ctx->tune = best;
    if ((rc = run(st))) break;
    float bt = st[1];
    const int cur = best.uni_threads[c];
    for (int th : kUniThreadChoices) {
      if (th == cur) continue;
      ctx->tune = best;
      ctx->tune.uni_threads[c] = th;
      if ((rc = run(st))) break;
      if (st[1] < bt) {
        bt = st[1];
        best.uni_threads[c] = th;
      }
    }
  }
  // reconstruction: coefficients per block and grid cap (warp kernel only)
  if (!rc && crt_warp_kernel(ctx, B.kmax, B.lmax)) {
    ctx->tune = best;
    rc = run(st);
    float bt = st[3];
    for (int t : {2, 4, 8})
      for (int b : {2, 4, 8}) {
        if (rc || (t == best.crt_tile && b == best.crt_blocks_per_sm)) continue;
        ctx->tune = best;
        ctx->tune.crt_tile = t;
        ctx->tune.crt_blocks_per_sm = b;
        if ((rc = run(st))) break;
        if (st[3] < bt) {
          bt = st[3];
          best.crt_tile = t;
          best.crt_blocks_per_sm = b;
        }
      }
  }
  ctx->tune = best;
  float ms_tuned = 0.f;
  if (!rc) {
    rc = run(st);
    ms_tuned = st[0] + st[1] + st[2] + st[3];
  }
  ctx->profile = was_profiling;
  if (rc) {
    ctx->tune = dflt;
    return rc;
  }
  if (info) {
    info->eval_warps = best.eval_warps;
    info->eval_blocks_per_sm = best.eval_blocks_per_sm;
    for (int c = 0; c < kNumUniClasses; ++c) info->uni_threads[c] = best.uni_threads[c];
    info->crt_tile = best.crt_tile;
    info->crt_blocks_per_sm = best.crt_blocks_per_sm;
    info->eval_independent = best.eval_independent;
    info->ms_default = ms_default;
    info->ms_tuned = ms_tuned;
    info->trials = trials;
  }
  return BS_OK;
}

extern "C" int bs_set_tune(bs_ctx* ctx, const bs_tune_info* t) {
  if (!ctx) return BS_ERR_ARG;
  if (!t) {
    ctx->tune = Tune{};
    return BS_OK;
  }
  Tune u;
  if (t->eval_warps < 1 || t->eval_warps > kEvalThreads / 32 || t->eval_blocks_per_sm < 1 ||
      t->eval_blocks_per_sm > 64 || (t->crt_tile != 1 && t->crt_tile != 2 && t->crt_tile != 4 &&
                                     t->crt_tile != 8) ||
      t->crt_blocks_per_sm < 1 || t->crt_blocks_per_sm > 64 ||
      (t->eval_independent != 0 && t->eval_independent != 1))
    return ctx_fail(ctx, BS_ERR_ARG, "launch shape out of range");
  for (int c = 0; c < kNumUniClasses; ++c) {
    if (t->uni_threads[c] != 64 && t->uni_threads[c] != 128 && t->uni_threads[c] != 256)
      return ctx_fail(ctx, BS_ERR_ARG, "univariate block size must be 64, 128 or 256");
    u.uni_threads[c] = t->uni_threads[c];
  }
  u.eval_warps = t->eval_warps;
  u.eval_blocks_per_sm = t->eval_blocks_per_sm;
  u.crt_tile = t->crt_tile;
  u.crt_blocks_per_sm = t->crt_blocks_per_sm;
  u.eval_independent = t->eval_independent;
  ctx->tune = u;
  return BS_OK;
}

extern "C" int bs_resultant(bs_ctx* ctx, const bs_bipoly* f, const bs_bipoly* g, int var,
                            bs_upoly* out) {
  if (!ctx) return BS_ERR_ARG;
  NvtxScope nv("bs_resultant");
  return run_host_batch(ctx, 1, f, g, var, out, false);
}

extern "C" int bs_resultant_batch(bs_ctx* ctx, int n, const bs_bipoly* f, const bs_bipoly* g,
                                  int var, bs_upoly* out) {
  if (!ctx) return BS_ERR_ARG;
  NvtxScope nv("bs_resultant_batch");
  return run_host_batch(ctx, n, f, g, var, out, true);
}

// ------------------------------------------------------------------------------------
// device-resident single job
// ------------------------------------------------------------------------------------
extern "C" int bs_resultant_device(bs_ctx* ctx, const bs_bipoly* f, const bs_bipoly* g, int var,
                                   bs_upoly* out) {
  if (!ctx) return BS_ERR_ARG;
  if (!out || !out->c || (var != 0 && var != 1)) return ctx_fail(ctx, BS_ERR_ARG, "bad arguments");
  if (ctx->server) return ctx_fail(ctx, BS_ERR_ARG, "the context runs a serving loop");
  NvtxScope nv("bs_resultant_device");
  int rc = check_bipoly(ctx, f, "f");
  if (rc) return rc;
  rc = check_bipoly(ctx, g, "g");
  if (rc) return rc;
  cudaSetDevice(ctx->device);
  MetaBounds mb;
  rc = meta_bounds(f, g, var, &mb);
  if (rc) return ctx_fail(ctx, rc, "problem exceeds the supported range");
  if (out->deg < mb.D || out->limbs < mb.out_limbs)
    return ctx_fail(ctx, BS_ERR_CAPACITY, "output capacity below bs_resultant_bounds()");
  const int cls = uni_class_of(mb.len);
  if (cls < 0) return ctx_fail(ctx, BS_ERR_RANGE, "degree in the eliminated variable above 64");
  rc = ctx->tabs->ensure(mb.k_total, mb.logN, ctx->stream);
  if (rc) return ctx_fail(ctx, rc, "table setup failed");
  const int N = 1 << mb.logN;
  Layout lay;
  const size_t o_job = lay.take(sizeof(Job));
  const size_t o_offs = lay.take(sizeof(int64_t) * kNumOffs);
  const size_t o_pstat = lay.take(sizeof(int32_t) * mb.k_total);
  const size_t o_ev = lay.take(sizeof(uint32_t) * (size_t)mb.k_total * mb.rows * N);
  const size_t o_vals = lay.take(sizeof(uint32_t) * (size_t)mb.k_total * N);
  const size_t o_rmod = lay.take(sizeof(uint32_t) * (size_t)mb.k_need * (mb.D + 1));
  const size_t o_sel = lay.take(sizeof(int32_t) * mb.k_need);
  if (lay.used > ctx->dev_ws_cap) {
    if (lay.used > ctx->budget) return ctx_fail(ctx, BS_ERR_NOMEM, "workspace exceeds the memory budget");
    if (ctx->dev_ws) {
      cudaStreamSynchronize(ctx->stream);
      cudaFree(ctx->dev_ws);
    }
    ctx->dev_ws = nullptr;
    ctx->dev_ws_cap = 0;
    if (cudaMalloc(&ctx->dev_ws, lay.used) != cudaSuccess) {
      cudaGetLastError();
      return ctx_fail(ctx, BS_ERR_NOMEM, "cudaMalloc of the workspace failed");
    }
    ctx->dev_ws_cap = lay.used;
  }
  char* base = (char*)ctx->dev_ws;
  Job J;
  std::memset(&J, 0, sizeof(J));
  J.f = grid_of(f);
  J.g = grid_of(g);
  J.var = var;
  J.ev = (uint32_t*)(base + o_ev);
  J.vals = (uint32_t*)(base + o_vals);
  J.rmod = (uint32_t*)(base + o_rmod);
  J.pstat = (int32_t*)(base + o_pstat);
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
  cudaStream_t s = ctx->stream;
  // the job descriptor travels as a kernel argument into device memory (no host copy
  // in flight that could be overwritten by the next call)
  rc = launch_device_job(ctx, J, (Job*)(base + o_job), (int64_t*)(base + o_offs), mb, cls);
  if (rc) return rc;
  ctx->stats = bs_stats{};
  ctx->stats.jobs = 1;
  (void)s;
  return BS_OK;
}

extern "C" int bs_device_status(bs_ctx* ctx) {
  if (!ctx) return BS_ERR_ARG;
  int32_t st[4] = {0, 0, 0, 0};
  if (cudaMemcpyAsync(st, ctx->d_status, sizeof(st), cudaMemcpyDeviceToHost, ctx->stream) !=
          cudaSuccess ||
      cudaStreamSynchronize(ctx->stream) != cudaSuccess)
    return ctx_fail(ctx, BS_ERR_CUDA, "status read failed");
  cudaMemsetAsync(ctx->d_status, 0, sizeof(st), ctx->stream);
  ctx->stats.primes_rejected = st[1];
  if (st[0]) return ctx_fail(ctx, st[0], device_failure_detail(st));
  return BS_OK;
}

// ------------------------------------------------------------------------------------
// univariate resultants of given images
// ------------------------------------------------------------------------------------
extern "C" int bs_uni_resultant_modp(bs_ctx* ctx, int n, const uint32_t* p, const uint32_t* a,
                                     int da, int lda, const uint32_t* b, int db, int ldb,
                                     uint32_t* res) {
  if (!ctx) return BS_ERR_ARG;
  if (n < 0 || da < 0 || db < 0 || lda < da + 1 || ldb < db + 1 || (n && (!p || !a || !b || !res)))
    return ctx_fail(ctx, BS_ERR_ARG, "bad arguments");
  if (n == 0) return BS_OK;
  const int cls = uni_class_of(std::max(da, db) + 1);
  if (cls < 0) return ctx_fail(ctx, BS_ERR_RANGE, "degree above 64");
  cudaSetDevice(ctx->device);
  std::vector<int32_t> idx(n);
  for (int i = 0; i < n; ++i) {
    idx[i] = table_index(p[i]);
    if (idx[i] < 0) return ctx_fail(ctx, BS_ERR_ARG, "not a table prime");
    for (int j = 0; j <= da; ++j)
      if (a[(size_t)i * lda + j] >= p[i]) return ctx_fail(ctx, BS_ERR_ARG, "input not reduced");
    for (int j = 0; j <= db; ++j)
      if (b[(size_t)i * ldb + j] >= p[i]) return ctx_fail(ctx, BS_ERR_ARG, "input not reduced");
  }
  Layout lay;
  const size_t o_idx = lay.take(sizeof(int32_t) * n);
  const size_t o_a = lay.take(sizeof(uint32_t) * (size_t)n * lda);
  const size_t o_b = lay.take(sizeof(uint32_t) * (size_t)n * ldb);
  const size_t o_r = lay.take(sizeof(uint32_t) * n);
  int rc = ensure_workspace(ctx, lay.used);
  if (rc) return rc;
  char* base = (char*)ctx->ws;
  cudaStream_t s = ctx->stream;
  rc |= ctx_cuda(ctx, cudaMemcpyAsync(base + o_idx, idx.data(), sizeof(int32_t) * n, cudaMemcpyHostToDevice, s), "h2d");
  rc |= ctx_cuda(ctx, cudaMemcpyAsync(base + o_a, a, sizeof(uint32_t) * (size_t)n * lda, cudaMemcpyHostToDevice, s), "h2d");
  rc |= ctx_cuda(ctx, cudaMemcpyAsync(base + o_b, b, sizeof(uint32_t) * (size_t)n * ldb, cudaMemcpyHostToDevice, s), "h2d");
  if (rc) return rc;
  const Tables Tv = ctx->tabs->view();
  launch_uni_direct(cls, n, s, (const int32_t*)(base + o_idx), (const uint32_t*)(base + o_a), da, lda,
                    (const uint32_t*)(base + o_b), db, ldb, (uint32_t*)(base + o_r), Tv);
  uint32_t* dR = (uint32_t*)(base + o_r);
  rc = ctx_cuda(ctx, cudaGetLastError(), "launch");
  if (rc) return rc;
  rc = ctx_cuda(ctx, cudaMemcpyAsync(res, dR, sizeof(uint32_t) * n, cudaMemcpyDeviceToHost, s), "d2h");
  if (rc) return rc;
  return ctx_cuda(ctx, cudaStreamSynchronize(s), "stream");
}
