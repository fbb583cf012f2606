// Principal subresultant coefficients sr_0, ..., sr_(q-1) of two bivariate polynomials
// with respect to one variable, exactly, by the modular route of the resultant (Sec. 3.3
// uses them to count the distinct points over the x-critical values; Sec. 5.1 gives the
// route): the same plan, reduction and evaluation, one psc sequence mod p per (prime,
// point) instead of one resultant, then one interpolation and one reconstruction per
// index i.
//
// Every sr_i is a minor of the Sylvester matrix built from a subset of its rows, so the
// resultant's coefficient bound (each row norm is at least 1) and degree bound hold for
// all of them, and the resultant's plan serves unchanged.  Primes are rejected by the same
// rule (a leading coefficient vanishing at a point of the prime's set), so all indices
// share one selection.
//
// One psc job is the primary job (evaluation and the psc stage) followed by q sub-jobs,
// one per index, which the interpolation and reconstruction kernels treat as resultant
// jobs whose values sit in slice i of the primary job's value array.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <string>
#include <vector>

#include "batch.cuh"
#include "ctx.cuh"
#include "modpoly.cuh"
#include "psc.cuh"

namespace bs {

// ---- the psc stage: one sequence per thread --------------------------------------------
template <int L>
__global__ void __launch_bounds__(kUniMaxThreads) k_psc(const Job* jobs, WorkList wl, Tables T) {
  const int64_t total = wl.off[wl.n];
  for (int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; g < total;
       g += (int64_t)gridDim.x * blockDim.x) {
    const int ji = find_item(wl.off, wl.n, g);
    const Job* J = jobs + (wl.ids ? wl.ids[ji] : ji);
    const int logN = J->plan.logN;
    const int64_t inst = g - wl.off[ji];
    const int N = 1 << logN;
    const int q = (int)(inst >> logN);
    const int t = (int)(inst & (N - 1));
    const int me = J->plan.me, ne = J->plan.ne;
    const int rows = J->rows;
    const PrimeConst pc = T.pc[q];
    const Mod M{pc.p, pc.pinv};
    // this instance's column of evaluations; read once, then reused as its scratch
    uint32_t* col = J->ev + (int64_t)q * rows * N + t;
    const uint32_t* bg = col + (int64_t)(me + 1) * N;
    uint32_t A[Arr<L>::N], B[Arr<L>::N];
#pragma unroll
    for (int s = 0; s < Arr<L>::N; ++s) {
      A[s] = (s <= me) ? col[(int64_t)(me - s) * N] : 0u;
      B[s] = (s <= ne) ? bg[(int64_t)(ne - s) * N] : 0u;
    }
    if (A[0] == 0 || B[0] == 0) J->pstat[q] = 1;  // unlucky: a leading coefficient vanishes
    psc_seq<L>(A, me + 1, B, ne + 1, M, pc.one_m, J->vals + inst, J->psc_stride, col, N);
  }
}

// ---- the subresultant stage: S_d(A, B) at one (prime, point) per thread ------------------
// The job's value slices j = 0..d receive the coefficient of y^j.  A point where a
// leading coefficient vanishes rejects its prime (the rule of the resultant).
template <int L>
__global__ void __launch_bounds__(kUniMaxThreads) k_sres(const Job* jobs, WorkList wl, Tables T, int d) {
  const int64_t total = wl.off[wl.n];
  for (int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; g < total;
       g += (int64_t)gridDim.x * blockDim.x) {
    const int ji = find_item(wl.off, wl.n, g);
    const Job* J = jobs + (wl.ids ? wl.ids[ji] : ji);
    const int logN = J->plan.logN;
    const int64_t inst = g - wl.off[ji];
    const int N = 1 << logN;
    const int q = (int)(inst >> logN);
    const int t = (int)(inst & (N - 1));
    const int me = J->plan.me, ne = J->plan.ne;
    const PrimeConst pc = T.pc[q];
    const Mod M{pc.p, pc.pinv};
    const uint32_t* bf = J->ev + (int64_t)q * J->rows * N + t;
    const uint32_t* bg = bf + (int64_t)(me + 1) * N;
    uint32_t A[Arr<L>::N], B[Arr<L>::N];
#pragma unroll
    for (int s = 0; s < Arr<L>::N; ++s) {
      A[s] = (s <= me) ? __ldg(bf + (int64_t)(me - s) * N) : 0u;
      B[s] = (s <= ne) ? __ldg(bg + (int64_t)(ne - s) * N) : 0u;
    }
    if (A[0] == 0 || B[0] == 0) J->pstat[q] = 1;  // unlucky: a leading coefficient vanishes
    if (!sres_seq<L>(A, me + 1, B, ne + 1, d, M, pc.one_m, J->vals + inst, J->psc_stride))
      set_status(J->status, kErrInternal);
  }
}

static void launch_sres(int cls, int grid, int threads, cudaStream_t s, const Job* jobs, WorkList wl,
                        Tables T, int d) {
  switch (cls) {
    case 0: k_sres<8><<<grid, threads, 0, s>>>(jobs, wl, T, d); break;
    case 1: k_sres<16><<<grid, threads, 0, s>>>(jobs, wl, T, d); break;
    case 2: k_sres<24><<<grid, threads, 0, s>>>(jobs, wl, T, d); break;
    case 3: k_sres<33><<<grid, threads, 0, s>>>(jobs, wl, T, d); break;
    case 4: k_sres<48><<<grid, threads, 0, s>>>(jobs, wl, T, d); break;
    default: k_sres<65><<<grid, threads, 0, s>>>(jobs, wl, T, d); break;
  }
}

static void launch_psc(int cls, int grid, int threads, cudaStream_t s, const Job* jobs, WorkList wl,
                       Tables T) {
  switch (cls) {
    case 0: k_psc<8><<<grid, threads, 0, s>>>(jobs, wl, T); break;
    case 1: k_psc<16><<<grid, threads, 0, s>>>(jobs, wl, T); break;
    case 2: k_psc<24><<<grid, threads, 0, s>>>(jobs, wl, T); break;
    case 3: k_psc<33><<<grid, threads, 0, s>>>(jobs, wl, T); break;
    case 4: k_psc<48><<<grid, threads, 0, s>>>(jobs, wl, T); break;
    default: k_psc<65><<<grid, threads, 0, s>>>(jobs, wl, T); break;
  }
}

// ---- host side ---------------------------------------------------------------------------
struct PscPlan {
  Plan P;
  bool modp = false;  // one good prime, residues only (no reconstruction)
  int sres_d = -1;    // >= 0: the coefficients of S_d instead of the psc sequence
  int q = 0, rows = 0;  // q: output polynomials (sr_0..sr_(q-1), or the d + 1 of S_d)
  size_t o_jobs = 0, o_ev_off = 0, o_psc_off = 0, o_ids = 0, o_intt_off = 0, o_crt_off = 0;
  size_t o_status = 0, o_pstat = 0, o_in = 0, up_bytes = 0;
  size_t o_ev = 0, o_vals = 0, o_rmod = 0, o_sel = 0;
  size_t dn_start = 0, o_out = 0, o_status_dn = 0, dn_bytes = 0, total = 0;
  int64_t in_f = 0, in_g = 0;
};

static int check_grid(bs_ctx* ctx, const bs_bipoly* p) {
  if (!p || p->deg_x < 0 || p->deg_y < 0 || p->limbs < 1 || p->limbs > kMaxLimbs || !p->c)
    return ctx_fail(ctx, BS_ERR_ARG, "bad bivariate polynomial");
  return 0;
}

static int psc_plan(bs_ctx* ctx, const bs_bipoly* f, const bs_bipoly* g, int var, bool modp, PscPlan* pp,
                    int sres_d = -1) {
  PscPlan& S = *pp;
  S.modp = modp;
  S.sres_d = sres_d;
  const HostPrimes& H = host_primes();
  const Grid gf{f->c, f->deg_x, f->deg_y, f->limbs}, gg{g->c, g->deg_x, g->deg_y, g->limbs};
  S.P = plan_host(gf, gg, var, H.lg_prefix.data(), (int)H.p.size(), H.p.data());
  if (S.P.status) return ctx_fail(ctx, S.P.status, "planning failed");
  if (modp && !S.P.trivial) {  // the first good prime only; the spares stay
    S.P.k_total = S.P.k_total - S.P.k_need + 1;
    S.P.k_need = 1;
  }
  S.q = S.P.trivial ? 0 : std::min(S.P.me, S.P.ne);
  if (S.q <= 0) {
    S.q = 0;
    return 0;
  }
  if (sres_d >= 0) {  // S_d is defined for d below the smaller degree
    if (sres_d >= S.q) return ctx_fail(ctx, BS_ERR_ARG, "subresultant index out of range");
    S.q = sres_d + 1;
  }
  const Plan& P = S.P;
  if (uni_class_of(std::max(P.me, P.ne) + 1) < 0)
    return ctx_fail(ctx, BS_ERR_RANGE, "degree in the eliminated variable above 64");
  if (kInttSmemWords * (size_t)P.N * sizeof(uint32_t) > (size_t)ctx->smem_optin)
    return ctx_fail(ctx, BS_ERR_RANGE, "transform size exceeds shared memory");
  S.rows = (P.me + 1) + (P.ne + 1);
  S.in_f = (int64_t)(f->deg_y + 1) * (f->deg_x + 1) * f->limbs;
  S.in_g = (int64_t)(g->deg_y + 1) * (g->deg_x + 1) * g->limbs;
  const int q = S.q;
  Layout up;
  S.o_jobs = up.take(sizeof(Job) * (q + 1));
  S.o_ev_off = up.take(sizeof(int64_t) * 2);
  S.o_psc_off = up.take(sizeof(int64_t) * 2);
  S.o_ids = up.take(sizeof(int32_t) * q);
  S.o_intt_off = up.take(sizeof(int64_t) * (q + 1));
  S.o_crt_off = up.take(sizeof(int64_t) * (q + 1));
  S.o_status = up.take(sizeof(int32_t) * 4);
  S.o_pstat = up.take(sizeof(int32_t) * P.k_total);
  S.o_in = up.take(sizeof(uint32_t) * (size_t)(S.in_f + S.in_g));
  S.up_bytes = up.used;
  Layout cmp;
  cmp.used = S.up_bytes;
  S.o_ev = cmp.take(sizeof(uint32_t) * (size_t)P.k_total * S.rows * P.N);
  S.o_vals = cmp.take(sizeof(uint32_t) * (size_t)q * P.k_total * P.N);
  if (!modp) {
    S.o_rmod = cmp.take(sizeof(uint32_t) * (size_t)q * P.k_need * (P.D + 1));
    S.o_sel = cmp.take(sizeof(int32_t) * (size_t)q * P.k_need);
  }
  Layout dn;
  dn.used = cmp.used;
  S.dn_start = dn.take(0);
  if (modp) {  // the residues and the selected prime are the result
    S.o_rmod = dn.take(sizeof(uint32_t) * (size_t)q * (P.D + 1));
    S.o_sel = dn.take(sizeof(int32_t) * (size_t)q);
  } else {
    S.o_out = dn.take(sizeof(uint32_t) * (size_t)q * (P.D + 1) * P.out_limbs);
  }
  S.o_status_dn = dn.take(sizeof(int32_t) * 4);
  S.total = dn.used;
  S.dn_bytes = S.total - S.dn_start;
  return 0;
}

static int psc_launch(bs_ctx* ctx, const PscPlan& S, const bs_bipoly* f, const bs_bipoly* g, int var,
                      char* base, char* hu, char* hd) {
  const Plan& P = S.P;
  const int q = S.q;
  std::memset(hu, 0, S.up_bytes);
  uint32_t* in = (uint32_t*)(hu + S.o_in);
  std::memcpy(in, f->c, sizeof(uint32_t) * S.in_f);
  std::memcpy(in + S.in_f, g->c, sizeof(uint32_t) * S.in_g);
  const uint32_t* din = (const uint32_t*)(base + S.o_in);
  Job* hj = (Job*)(hu + S.o_jobs);
  const int64_t stride = (int64_t)P.k_total * P.N;
  int32_t* status = (int32_t*)(base + S.o_status);
  {  // the primary job: evaluation and the psc stage
    Job& J = hj[0];
    J.f = Grid{din, f->deg_x, f->deg_y, f->limbs};
    J.g = Grid{din + S.in_f, g->deg_x, g->deg_y, g->limbs};
    J.var = var;
    J.plan = P;
    J.rows = S.rows;
    J.ev = (uint32_t*)(base + S.o_ev);
    J.vals = (uint32_t*)(base + S.o_vals);
    J.pstat = (int32_t*)(base + S.o_pstat);
    J.status = status;
    J.npsc = q;
    J.psc_stride = stride;
    J.cap_deg = P.D;
    J.cap_limbs = P.out_limbs;
  }
  int32_t* ids = (int32_t*)(hu + S.o_ids);
  int64_t* ioff = (int64_t*)(hu + S.o_intt_off);
  int64_t* coff = (int64_t*)(hu + S.o_crt_off);
  ioff[0] = coff[0] = 0;
  for (int i = 0; i < q; ++i) {  // sub-job i + 1: index i
    Job& J = hj[i + 1];
    J.plan = P;
    J.vals = (uint32_t*)(base + S.o_vals) + i * stride;
    J.rmod = (uint32_t*)(base + S.o_rmod) + (size_t)i * P.k_need * (P.D + 1);
    J.sel = (int32_t*)(base + S.o_sel) + (size_t)i * P.k_need;
    J.pstat = (int32_t*)(base + S.o_pstat);
    J.out = S.modp ? nullptr : (uint32_t*)(base + S.o_out) + (size_t)i * (P.D + 1) * P.out_limbs;
    J.cap_deg = P.D;
    J.cap_limbs = P.out_limbs;
    J.status = status;
    J.rejected = i == 0 ? status + 1 : nullptr;
    ids[i] = i + 1;
    ioff[i + 1] = ioff[i] + P.k_total;
    coff[i + 1] = coff[i] + (P.D + kCrtTile) / kCrtTile;
  }
  const int ew = ctx->tune.eval_warps;
  int64_t* eo = (int64_t*)(hu + S.o_ev_off);
  int64_t* po = (int64_t*)(hu + S.o_psc_off);
  const bool warp_eval = P.logN <= kWarpLogNMax;
  eo[0] = 0;
  eo[1] = warp_eval ? (int64_t)P.k_total * ((S.rows + ew - 1) / ew) : (int64_t)P.k_total * S.rows;
  po[0] = 0;
  po[1] = (int64_t)P.k_total << P.logN;
  cudaStream_t s = ctx->stream;
  int rc = ctx_cuda(ctx, cudaMemcpyAsync(base, hu, S.up_bytes, cudaMemcpyHostToDevice, s), "upload");
  if (rc) return rc;
  const Tables Tv = ctx->tabs->view();
  const Job* dj = (const Job*)(base + S.o_jobs);
  const int sms = ctx->sms;
  const WorkList wl_ev{nullptr, (const int64_t*)(base + S.o_ev_off), 1};
  if (warp_eval) {
    const int grid = (int)std::min<int64_t>(eo[1], (int64_t)sms * ctx->tune.eval_blocks_per_sm);
    launch_eval_w(eval_class_of(P.logN), grid, ew, s, dj, wl_ev, Tv, PfHint{P.k_total, P.N, P.k_need});
  } else {
    const int ecw = std::max(2, P.N >> 10);
    const int grid = (int)std::min<int64_t>(eo[1], (int64_t)sms * std::max(1, 16 / ecw));
    launch_eval(grid, ecw, s, dj, wl_ev, Tv);
  }
  {
    const int cls = uni_class_of(std::max(P.me, P.ne) + 1);
    const int th = 128;
    const int grid = (int)std::min<int64_t>((po[1] + th - 1) / th, (int64_t)sms * std::max(1, ctx->occ[cls][1]));
    const WorkList wl_p{nullptr, (const int64_t*)(base + S.o_psc_off), 1};
    if (S.sres_d >= 0)
      launch_sres(cls, grid, th, s, dj, wl_p, Tv, S.sres_d);
    else
      launch_psc(cls, grid, th, s, dj, wl_p, Tv);
  }
  const WorkList wl_i{(const int32_t*)(base + S.o_ids), (const int64_t*)(base + S.o_intt_off), q};
  if (P.logN <= kWarpInttLogNMax)
    launch_intt_w((int)std::min<int64_t>((ioff[q] + kInttWarps - 1) / kInttWarps, (int64_t)sms * 8), s, dj,
                  wl_i, Tv);
  else
    launch_intt((int)std::min<int64_t>(ioff[q], (int64_t)sms * 8), kInttSmemWords * sizeof(uint32_t) * (size_t)P.N, s, dj,
                wl_i, Tv);
  const WorkList wl_c{(const int32_t*)(base + S.o_ids), (const int64_t*)(base + S.o_crt_off), q};
  if (!S.modp) {  // the modular form stops at the residues
  const int crt_grid = (int)std::min<int64_t>(coff[q], (int64_t)sms * 4);
  const int kmax = P.k_need, lmax = P.out_limbs + 1;
  const size_t wsm = crt_warp_smem(kmax, lmax);
  if (kmax <= kCrtWarpMaxK && wsm <= (size_t)ctx->smem_optin - 64) {
    launch_crt_w(crt_grid, kCrtTile, wsm, s, dj, wl_c, Tv, kmax, lmax);
  } else {
    const size_t per = (size_t)3 * lmax * sizeof(uint32_t);
    const size_t fixed = ((size_t)kmax * kCrtTile + 3 * (size_t)kmax) * sizeof(uint32_t);
    if (fixed + per > (size_t)ctx->smem_optin - 64)
      return ctx_fail(ctx, BS_ERR_RANGE, "too many primes for the reconstruction stage");
    const int w = (int)std::min<size_t>(kCrtWarps, ((size_t)ctx->smem_optin - 64 - fixed) / per);
    launch_crt(crt_grid, w * 32, fixed + per * w, s, dj, wl_c, Tv, kmax, lmax, 0);
  }
  }
  rc = ctx_cuda(ctx, cudaGetLastError(), "launch");
  if (rc) return rc;
  rc = ctx_cuda(ctx, cudaMemcpyAsync(base + S.o_status_dn, status, sizeof(int32_t) * 4, cudaMemcpyDeviceToDevice, s),
                "status copy");
  if (rc) return rc;
  return ctx_cuda(ctx, cudaMemcpyAsync(hd, base + S.dn_start, S.dn_bytes, cudaMemcpyDeviceToHost, s),
                  "download");
}

static int psc_finish(bs_ctx* ctx, const PscPlan& S, const char* hd, bs_upoly* out) {
  const Plan& P = S.P;
  const int32_t* st = (const int32_t*)(hd + (S.o_status_dn - S.dn_start));
  if (st[0]) return ctx_fail(ctx, st[0], device_failure_detail(st));
  for (int i = 0; i < S.q; ++i) {
    const uint32_t* src = (const uint32_t*)(hd + (S.o_out - S.dn_start)) + (size_t)i * (P.D + 1) * P.out_limbs;
    int deg = P.D;
    while (deg >= 0 && limbs_zero(src + (size_t)deg * P.out_limbs, P.out_limbs)) --deg;
    if (deg < 0) {
      for (int c = 0; c <= out[i].deg; ++c)
        std::memset(out[i].c + (size_t)c * out[i].limbs, 0, sizeof(uint32_t) * out[i].limbs);
      out[i].deg = -1;
      continue;
    }
    const int rc = put_result(ctx, src, P.out_limbs, deg, out + i);
    if (rc) return rc;
  }
  return BS_OK;
}

static int run_psc(bs_ctx* ctx, const bs_bipoly* f, const bs_bipoly* g, int var, int cap_q, int32_t* q_out,
                   bs_upoly* out, int sres_d = -1) {
  if (ctx->server) return ctx_fail(ctx, BS_ERR_ARG, "the context runs a serving loop");
  int rc = check_grid(ctx, f);
  if (!rc) rc = check_grid(ctx, g);
  if (rc) return rc;
  cudaSetDevice(ctx->device);
  PscPlan S;
  rc = psc_plan(ctx, f, g, var, false, &S, sres_d);
  if (rc) return rc;
  *q_out = S.q;
  if (S.q == 0) {
    if (sres_d >= 0) return ctx_fail(ctx, BS_ERR_ARG, "subresultant index out of range");
    return BS_OK;
  }
  if (!out || !out[0].c) {  // size query
    for (int i = 0; out && i < std::min(cap_q, S.q); ++i) {
      out[i].deg = S.P.D;
      out[i].limbs = S.P.out_limbs;
    }
    return BS_OK;
  }
  if (cap_q < S.q) return ctx_fail(ctx, BS_ERR_CAPACITY, "fewer outputs than coefficients");
  for (int i = 0; i < S.q; ++i)
    if (!out[i].c || out[i].limbs < 1 || out[i].deg < -1) return ctx_fail(ctx, BS_ERR_ARG, "bad output capacity");
  rc = ctx->tabs->ensure(S.P.k_total, S.P.logN, ctx->stream);
  if (rc) return ctx_fail(ctx, rc, "table setup failed");
  rc = ensure_workspace(ctx, S.total);
  if (rc) return rc;
  rc = ensure_pinned(ctx, S.up_bytes, S.dn_bytes);
  if (rc) return rc;
  rc = psc_launch(ctx, S, f, g, var, (char*)ctx->ws, (char*)ctx->h_up, (char*)ctx->h_down);
  if (rc) return rc;
  rc = ctx_cuda(ctx, cudaStreamSynchronize(ctx->stream), "stream");
  if (rc) return rc;
  return psc_finish(ctx, S, (const char*)ctx->h_down, out);
}

static int run_psc_modp(bs_ctx* ctx, const bs_bipoly* f, const bs_bipoly* g, int var, int32_t* q_out,
                        int32_t* dmax, int32_t* deg, uint32_t* coef, uint32_t* p_out) {
  if (ctx->server) return ctx_fail(ctx, BS_ERR_ARG, "the context runs a serving loop");
  int rc = check_grid(ctx, f);
  if (!rc) rc = check_grid(ctx, g);
  if (rc) return rc;
  cudaSetDevice(ctx->device);
  PscPlan S;
  rc = psc_plan(ctx, f, g, var, true, &S);
  if (rc) return rc;
  *q_out = S.q;
  if (S.q == 0) return BS_OK;
  if (!coef) {  // size query
    *dmax = S.P.D;
    return BS_OK;
  }
  if (!deg || *dmax < S.P.D) return ctx_fail(ctx, BS_ERR_CAPACITY, "residue capacity too small");
  const int cap = *dmax + 1;
  rc = ctx->tabs->ensure(S.P.k_total, S.P.logN, ctx->stream);
  if (rc) return ctx_fail(ctx, rc, "table setup failed");
  rc = ensure_workspace(ctx, S.total);
  if (rc) return rc;
  rc = ensure_pinned(ctx, S.up_bytes, S.dn_bytes);
  if (rc) return rc;
  rc = psc_launch(ctx, S, f, g, var, (char*)ctx->ws, (char*)ctx->h_up, (char*)ctx->h_down);
  if (rc) return rc;
  rc = ctx_cuda(ctx, cudaStreamSynchronize(ctx->stream), "stream");
  if (rc) return rc;
  const char* hd = (const char*)ctx->h_down;
  const int32_t* st = (const int32_t*)(hd + (S.o_status_dn - S.dn_start));
  if (st[0]) return ctx_fail(ctx, st[0], device_failure_detail(st));
  const int32_t* sel = (const int32_t*)(hd + (S.o_sel - S.dn_start));
  *p_out = host_primes().p[sel[0]];
  const int D = S.P.D;
  for (int i = 0; i < S.q; ++i) {
    const uint32_t* src = (const uint32_t*)(hd + (S.o_rmod - S.dn_start)) + (size_t)i * (D + 1);
    int d = D;
    while (d >= 0 && src[d] == 0u) --d;
    deg[i] = d;
    std::memcpy(coef + (size_t)i * cap, src, sizeof(uint32_t) * (D + 1));
    std::memset(coef + (size_t)i * cap + D + 1, 0, sizeof(uint32_t) * (cap - D - 1));
  }
  return BS_OK;
}

}  // namespace bs

using namespace bs;

extern "C" int bs_psc_modp(bs_ctx* ctx, const bs_bipoly* f, const bs_bipoly* g, int var, int32_t* q,
                           int32_t* dmax, int32_t* deg, uint32_t* coef, uint32_t* p) {
  if (!ctx) return BS_ERR_ARG;
  if (!f || !g || !q || !dmax || !p || (var != 0 && var != 1)) return ctx_fail(ctx, BS_ERR_ARG, "bad arguments");
  return run_psc_modp(ctx, f, g, var, q, dmax, deg, coef, p);
}

extern "C" int bs_subresultant(bs_ctx* ctx, const bs_bipoly* f, const bs_bipoly* g, int var, int d,
                               int cap, int32_t* n, bs_upoly* out) {
  if (!ctx) return BS_ERR_ARG;
  if (!f || !g || !n || (var != 0 && var != 1) || d < 0 || cap < 0)
    return ctx_fail(ctx, BS_ERR_ARG, "bad arguments");
  return run_psc(ctx, f, g, var, cap, n, out, d);
}

extern "C" int bs_psc(bs_ctx* ctx, const bs_bipoly* f, const bs_bipoly* g, int var, int cap_q, int32_t* q,
                      bs_upoly* out) {
  if (!ctx) return BS_ERR_ARG;
  if (!f || !g || !q || (var != 0 && var != 1) || cap_q < 0) return ctx_fail(ctx, BS_ERR_ARG, "bad arguments");
  return run_psc(ctx, f, g, var, cap_q, q, out);
}
