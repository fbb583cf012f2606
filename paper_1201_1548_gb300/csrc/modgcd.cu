// Modular gcds in Z[x]: the gcd of two polynomials and the square-free part of one, for
// a batch of jobs in one pass of launches (Sec. 5.1, "Computing gcds in Z[x]": the gcd is
// computed modulo many primes and lifted by Chinese remaindering; Sec. 2.1, BiProject:
// the square-free factorisation of the projection starts from gcd(R, R')).
//
// For a job on a (and b), with lc(a) as scale:
//   gcd:              H = (lc(a) / lc(G)) G,   G = the primitive gcd of a and b;
//   square-free part: H = a / gcd(a, a') over Q, which has integer coefficients and
//                     leading coefficient lc(a).
// Mignotte's bound for a factor of a gives ||H||_inf <= 2^deg(H) ||a||_2 in both cases.
// For every prime not dividing a leading coefficient, the image of H is lc(a) times the
// monic gcd (respectively (a mod p) divided by the monic gcd of a and a') whenever the
// gcd mod p has the minimal degree over the primes tried; larger degrees mark unlucky
// primes (Brown's rule).  H is rebuilt by Chinese remaindering, its content c removed
// with the sign of lc(a), and the final polynomial rebuilt from the images of
// H (s c)^-1 m, where m = gcd(cont a, cont b) for the gcd and 1 for the square-free part.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <string>
#include <vector>

#include "batch.cuh"
#include "ctx.cuh"
#include "modpoly.cuh"
#include "wbig.cuh"

namespace bs {

enum : int32_t { kMgGcd = 0, kMgSqf = 1, kMgDiv = 2 };

struct MgJob {
  const uint32_t* A;  // [(da + 1) * La] limbs of a
  const uint32_t* B;  // [(db + 1) * Lb] limbs of b (gcd jobs)
  int32_t da, db, La, Lb;
  int32_t kind;
  int32_t k_total, k_need;
  int32_t cap;        // degree bound of H
  int32_t Lc;         // limbs of the reconstructed values
  uint32_t* Qp;       // [k_total][cap + 1] images of H (standard form)
  int32_t* dg;        // [k_total] gcd degree mod p; -2: the prime divides a leading coefficient
  int32_t* sel;       // [k_need] selected table indices
  uint32_t* rmod;     // [k_need][deg H + 1] residues handed to the reconstruction
  int32_t* info;      // [0] deg H, [1] good primes, [2] minimal gcd degree, [3] status
  uint32_t* content;  // [Lc] content of H
  uint32_t* cmul;     // [Lc] final multiplier m
  uint32_t* cinv;     // [k_need] m (s c)^-1 mod p (Montgomery form)
  Job* crt;           // [2] reconstructions of H and of the result
};


__global__ void k_mg_images(const MgJob* jobs, WorkList wl, Tables T) {
  extern __shared__ uint32_t sm[];
  __shared__ int s_top, s_la, s_lb;
  const int64_t total = wl.off[wl.n];
  for (int64_t item = blockIdx.x; item < total; item += gridDim.x) {
    const int ji = find_item(wl.off, wl.n, item);
    const MgJob& J = jobs[ji];
    const int q = (int)(item - wl.off[ji]);
    const PrimeConst pc = T.pc[q];
    const Mod M{pc.p, pc.pinv};
    const uint32_t* pw = T.pw + (int64_t)q * (kMaxLimbs + 1);
    const uint32_t* mpw = T.mpw + (int64_t)q * (kMaxLimbs + 1);
    const int da = J.da;
    uint32_t* sA = sm;
    uint32_t* sB = sA + da + 1;
    const int nb = (J.kind != kMgSqf) ? J.db + 1 : da;  // a' has degree < da
    uint32_t* sR = sB + (nb > 0 ? nb : 1);              // square-free part: a kept for the division
    for (int i = threadIdx.x; i <= da; i += blockDim.x) {
      const uint32_t v = reduce_coef(J.A + (int64_t)i * J.La, J.La, pw, mpw, pc);
      sA[i] = v;
      if (J.kind == kMgSqf) sR[i] = v;
    }
    if (J.kind != kMgSqf)
      for (int i = threadIdx.x; i <= J.db; i += blockDim.x)
        sB[i] = reduce_coef(J.B + (int64_t)i * J.Lb, J.Lb, pw, mpw, pc);
    __syncthreads();
    if (J.kind == kMgSqf)  // a'_i = (i + 1) a_{i+1}; (i + 1) in Montgomery form is (i + 1) R
      for (int i = threadIdx.x; i < da; i += blockDim.x)
        sB[i] = mmul(sA[i + 1], redc((uint64_t)(uint32_t)(i + 1) * pc.r2, M.p, M.pinv), M);
    __syncthreads();
    const uint32_t lca = sA[da];
    const int lbd = (J.kind != kMgSqf) ? J.db : da - 1;
    if (threadIdx.x == 0) {
      int lb = lbd;
      while (lb >= 0 && sB[lb] == 0) --lb;
      s_la = da;
      s_lb = lb;
    }
    __syncthreads();
    // a prime dividing lc(a) or lc(b) is skipped (for a' the leading coefficient is
    // da lc(a), and p > da)
    const bool bad = (J.kind == kMgDiv) ? (s_lb != J.db)
                                        : (lca == 0u) || (J.kind == kMgGcd && s_lb != J.db);
    uint32_t* Qo = J.Qp + (int64_t)q * (J.cap + 1);
    if (bad) {
      if (threadIdx.x == 0) J.dg[q] = -2;
      __syncthreads();
      continue;
    }
    if (J.kind == kMgDiv) {  // a / b mod p, one quotient coefficient per step; -3: a remainder
      const int db = J.db, dq = da - db;
      const uint32_t ilb = minv(sB[db], pc.one_m, M);
      for (int s = dq; s >= 0; --s) {
        const uint32_t qc = mmul(sA[s + db], ilb, M);
        __syncthreads();
        for (int i = threadIdx.x; i < db; i += blockDim.x) sA[s + i] = msub(sA[s + i], mmul(qc, sB[i], M), M.p);
        if (threadIdx.x == 0) Qo[s] = redc((uint64_t)qc, M.p, M.pinv);
        __syncthreads();
      }
      bool rem = false;
      for (int i = threadIdx.x; i < db; i += blockDim.x) rem = rem || (sA[i] != 0u);
      rem = __syncthreads_or(rem);
      for (int i = dq + 1 + threadIdx.x; i <= J.cap; i += blockDim.x) Qo[i] = 0u;
      if (threadIdx.x == 0) J.dg[q] = rem ? -3 : 0;
      __syncthreads();
      continue;
    }
    int dgq;
    uint32_t* X = smem_euclid(sA, s_la, sB, s_lb, M, &dgq, &s_top);
    if (J.kind == kMgSqf && dgq < 0) dgq = 0;  // cannot happen for a != 0; kept total
    const uint32_t ilc = minv(X[dgq], pc.one_m, M);
    if (J.kind == kMgGcd) {
      // image of H = lc(a) * monic gcd, in standard form
      const uint32_t scale = mmul(ilc, lca, M);
      for (int i = threadIdx.x; i <= J.cap; i += blockDim.x)
        Qo[i] = (i <= dgq) ? redc((uint64_t)mmul(X[i], scale, M), M.p, M.pinv) : 0u;
    } else {
      for (int i = threadIdx.x; i <= dgq; i += blockDim.x) X[i] = mmul(X[i], ilc, M);
      __syncthreads();
      // H = a / gcd by long division (gcd monic), one quotient coefficient per step
      const int dq = da - dgq;
      for (int s = dq; s >= 0; --s) {
        const uint32_t qc = sR[s + dgq];
        __syncthreads();
        for (int i = threadIdx.x; i < dgq; i += blockDim.x)
          sR[s + i] = msub(sR[s + i], mmul(qc, X[i], M), M.p);
        if (threadIdx.x == 0) Qo[s] = redc((uint64_t)qc, M.p, M.pinv);
        __syncthreads();
      }
      for (int i = dq + 1 + threadIdx.x; i <= J.cap; i += blockDim.x) Qo[i] = 0u;
    }
    if (threadIdx.x == 0) J.dg[q] = dgq;
    __syncthreads();
  }
}

// ---- selection: one thread per job ------------------------------------------------------
__global__ void k_mg_select(const MgJob* jobs, int n) {
  const int ji = blockIdx.x * blockDim.x + threadIdx.x;
  if (ji >= n) return;
  const MgJob& J = jobs[ji];
  int mind = 1 << 30;
  for (int q = 0; q < J.k_total; ++q)
    if (J.dg[q] >= 0 && J.dg[q] < mind) mind = J.dg[q];
  int r = 0;
  for (int q = 0; q < J.k_total && r < J.k_need; ++q)
    if (J.dg[q] == mind) J.sel[r++] = q;
  const int degH = (r == 0) ? -1 : (J.kind == kMgGcd ? mind : J.kind == kMgDiv ? J.da - J.db : J.da - mind);
  J.info[0] = degH;
  J.info[1] = r;
  J.info[2] = (r == 0) ? -1 : mind;
  bool inexact = false;  // a remainder modulo some prime: b does not divide a
  for (int q = 0; q < J.k_total; ++q) inexact = inexact || J.dg[q] == -3;
  const bool ok = r == J.k_need && !inexact;
  J.info[3] = inexact ? kErrArg : ok ? 0 : kErrUnlucky;  // the job's status word (the reconstructions may add to it)
  for (int t = 0; t < 2; ++t) {
    J.crt[t].plan.D = ok ? degH : 0;
    J.crt[t].plan.status = J.info[3];
  }
}

// ---- residues for a reconstruction: blocks over jobs and their selected primes ----------
// second = 0: images of H; second = 1: images of H times cinv
// blockIdx.x strides over the jobs, blockIdx.y over a job's selected primes (rows)
__global__ void k_mg_gather(const MgJob* jobs, int n, Tables T, int second) {
  for (int ji = blockIdx.x; ji < n; ji += gridDim.x) {
    const MgJob& J = jobs[ji];
    if (J.info[3] != 0) continue;
    const int dh = J.info[0];
    for (int r = blockIdx.y; r < J.k_need; r += gridDim.y) {
      const int q = J.sel[r];
      const uint32_t* src = J.Qp + (int64_t)q * (J.cap + 1);
      uint32_t* dst = J.rmod + (int64_t)r * (dh + 1);
      if (second) {  // standard form times Montgomery form gives standard form
        const PrimeConst pc = T.pc[q];
        const uint32_t ci = J.cinv[r];
        for (int i = threadIdx.x; i <= dh; i += blockDim.x) dst[i] = redc((uint64_t)src[i] * ci, pc.p, pc.pinv);
      } else {
        for (int i = threadIdx.x; i <= dh; i += blockDim.x) dst[i] = src[i];
      }
    }
  }
}

// ---- contents: one block per job, its warps splitting the coefficients -----------------
template <int K>
__device__ void mg_content_job(const MgJob& J, uint32_t* part) {
  if (J.info[3] != 0) return;
  if (J.kind == kMgDiv) {  // the quotient is the result as it is
    for (int l = threadIdx.x; l < J.Lc; l += blockDim.x) J.content[l] = J.cmul[l] = (l == 0) ? 1u : 0u;
    return;
  }
  const int dh = J.info[0];
  block_content<K>(J.crt[0].out, dh + 1, J.Lc, nullptr, 0, 1, part, J.Lc, J.content, J.Lc);
  if (J.kind == kMgGcd) {  // gcd(cont a, cont b) = cont gcd(a, b): it fits the output's limbs
    const int Lp = std::max(std::max(J.La, J.Lb), J.Lc);
    block_content<K>(J.A, J.da + 1, J.La, J.B, J.db + 1, J.Lb, part, Lp, J.cmul, J.Lc);
  } else {
    for (int l = threadIdx.x; l < J.Lc; l += blockDim.x) J.cmul[l] = (l == 0) ? 1u : 0u;
  }
}

// dynamic shared memory: (blockDim.x / 32) * max(Lc, La, Lb) words for the partial gcds
__global__ void __launch_bounds__(256) k_mg_content(const MgJob* jobs, int n, int K) {
  extern __shared__ uint32_t mg_part[];
  for (int ji = blockIdx.x; ji < n; ji += gridDim.x) {
    if (K <= 1)
      mg_content_job<1>(jobs[ji], mg_part);
    else if (K <= 2)
      mg_content_job<2>(jobs[ji], mg_part);
    else if (K <= 4)
      mg_content_job<4>(jobs[ji], mg_part);
    else
      mg_content_job<8>(jobs[ji], mg_part);
  }
}

// ---- per selected prime: m (s c)^-1 mod p, s the sign of lc(a) -------------------------
__global__ void k_mg_cinv(const MgJob* jobs, int n, Tables T) {
  for (int ji = blockIdx.x; ji < n; ji += gridDim.x) {
    const MgJob& J = jobs[ji];
    if (J.info[3] != 0) continue;
    const bool neg = J.kind != kMgDiv && (J.A[(int64_t)J.da * J.La + J.La - 1] >> 31) != 0;
    for (int r = threadIdx.x; r < J.k_need; r += blockDim.x) {
      const int q = J.sel[r];
      const PrimeConst pc = T.pc[q];
      const Mod M{pc.p, pc.pinv};
      uint32_t c = mag_mod(J.content, J.Lc, pc.p);
      if (neg) c = mneg(c, pc.p);
      const uint32_t m = mag_mod(J.cmul, J.Lc, pc.p);
      const uint32_t c_m = redc((uint64_t)c * pc.r2, M.p, M.pinv);
      const uint32_t m_m = redc((uint64_t)m * pc.r2, M.p, M.pinv);
      J.cinv[r] = mmul(minv(c_m, pc.one_m, M), m_m, M);
    }
  }
}

// ---- host side ---------------------------------------------------------------------------
// result = sign(lc) * u (positive leading coefficient), written as L limbs per coefficient
static void normalised_copy(const bs_upoly& u, int d, std::vector<uint32_t>* out, int* L) {
  *L = u.limbs + 1;  // negating the most negative value needs one more limb
  out->assign((size_t)(d + 1) * (*L), 0u);
  const bool neg = (u.c[(size_t)d * u.limbs + u.limbs - 1] >> 31) != 0;
  for (int i = 0; i <= d; ++i) {
    const uint32_t* s = u.c + (size_t)i * u.limbs;
    uint32_t* t = out->data() + (size_t)i * (*L);
    const uint32_t ext = (s[u.limbs - 1] >> 31) ? 0xffffffffu : 0u;
    uint64_t carry = 1;
    for (int l = 0; l < *L; ++l) {
      const uint32_t v = l < u.limbs ? s[l] : ext;
      if (neg) {
        const uint64_t x = (uint64_t)(uint32_t)~v + carry;
        t[l] = (uint32_t)x;
        carry = x >> 32;
      } else {
        t[l] = v;
      }
    }
  }
}

int mg_plan(bs_ctx* ctx, int n, const int* kind, const bs_upoly* a, const bs_upoly* b, MgBatch* mbp) {
  MgBatch& B = *mbp;
  B = MgBatch{};
  B.n = n;
  const HostPrimes& H = host_primes();
  const int T = (int)H.p.size();
  B.kind.assign(kind, kind + n);
  B.k_need.assign(n, 0);
  B.k_total.assign(n, 0);
  B.cap.assign(n, 0);
  B.out_limbs.assign(n, 1);
  B.da.assign(n, -1);
  B.db.assign(n, -1);
  B.special.assign(n, 0);
  B.special_out.assign(n, {});
  B.special_deg.assign(n, -1);
  B.swap.assign(n, 0);
  std::vector<int> sL(n, 1);
  size_t in_words = 0;
  int maxdeg = 0;
  for (int j = 0; j < n; ++j) {
    const int kd = kind[j];
    if (kd != kMgGcd && kd != kMgSqf && kd != kMgDiv) return ctx_fail(ctx, BS_ERR_ARG, "unknown job kind");
    const bs_upoly* pa = a + j;
    const bs_upoly* pb = b ? b + j : nullptr;
    auto bad = [](const bs_upoly* u) {
      return !u || u->deg < -1 || u->limbs < 1 || u->limbs > kMaxUniLimbs || (u->deg >= 0 && !u->c);
    };
    if (bad(pa) || (kd != kMgSqf && bad(pb))) return ctx_fail(ctx, BS_ERR_ARG, "bad polynomial");
    int da = trimmed_degree(*pa);
    int db = kd != kMgSqf ? trimmed_degree(*pb) : -1;
    if (kd == kMgDiv) {
      if (db < 0) return ctx_fail(ctx, BS_ERR_ARG, "division by the zero polynomial");
      if (da >= 0 && da < db) return ctx_fail(ctx, BS_ERR_ARG, "the division is not exact");
      if (da < 0) {  // 0 / b = 0
        B.special[j] = 1;
        B.special_deg[j] = -1;
        continue;
      }
    } else if (kd == kMgSqf) {
      if (da < 0) return ctx_fail(ctx, BS_ERR_ZERO, "square-free part of the zero polynomial");
      if (da == 0) {
        B.special[j] = 1;
        B.special_out[j] = {1u};
        B.special_deg[j] = 0;
        sL[j] = 1;
        continue;
      }
    } else {
      if (da < 0 && db < 0) {
        B.special[j] = 1;
        B.special_deg[j] = -1;
        continue;
      }
      if (da < 0 || db < 0) {  // gcd(0, u) = u with a positive leading coefficient
        const bs_upoly& u = da < 0 ? *pb : *pa;
        const int du = da < 0 ? db : da;
        B.special[j] = 1;
        B.special_deg[j] = du;
        normalised_copy(u, du, &B.special_out[j], &sL[j]);
        continue;
      }
    }
    int64_t l2a = log2_norm2_q16(*pa, da);
    if (kd == kMgGcd) {
      // the scale carrier is the input with the smaller norm
      const int64_t l2b = log2_norm2_q16(*pb, db);
      if (l2b < l2a) {
        B.swap[j] = 1;
        std::swap(da, db);
        l2a = l2b;
      }
    }
    const bs_upoly& A = B.swap[j] ? *pb : *pa;
    const bs_upoly* Bp = B.swap[j] ? pa : pb;
    const int cap = kd == kMgGcd ? std::min(da, db) : kd == kMgDiv ? da - db : da;
    const int64_t bits = (int64_t)cap + (l2a + 65535) / 65536 + 1;  // |H| < 2^bits
    const int64_t need = (bits + 2) * 65536;
    if (H.lg_prefix[T] < need) return ctx_fail(ctx, BS_ERR_RANGE, "bound exceeds the prime table");
    const int k = std::max(1, prime_count_host(H.lg_prefix.data(), T, need));
    const int lcb = (kd == kMgDiv ? 0 : lc_bits(A, da)) + (kd != kMgSqf ? lc_bits(*Bp, db) : 0);
    const int kt = std::min(T, k + 4 + k / 8 + lcb / 30);
    if ((bits + 2 + 31) / 32 > 256) return ctx_fail(ctx, BS_ERR_RANGE, "coefficients above 8192 bits");
    B.da[j] = da;
    B.db[j] = db;
    B.k_need[j] = k;
    B.k_total[j] = kt;
    B.cap[j] = cap;
    B.out_limbs[j] = (int)((bits + 2 + 31) / 32);
    B.kmax = std::max(B.kmax, k);
    B.lmax = std::max(B.lmax, B.out_limbs[j] + 1);
    B.needT = std::max(B.needT, kt);
    const size_t words = kd != kMgSqf ? (size_t)(da + 1) + (db + 1) + 1 : (size_t)3 * (da + 1);
    B.smem = std::max(B.smem, words * sizeof(uint32_t));
    maxdeg = std::max(maxdeg, std::max(da, db));
    in_words += (size_t)(da + 1) * A.limbs + (kd != kMgSqf ? (size_t)(db + 1) * Bp->limbs : 0);
    B.in_limbs = std::max(B.in_limbs, std::max(A.limbs, kd != kMgSqf ? Bp->limbs : 1));
    B.items += kt;
  }
  if (B.smem > (size_t)ctx->smem_optin - 64)
    return ctx_fail(ctx, BS_ERR_RANGE, "degree too large for one block's shared memory");
  B.threads = std::min(256, std::max(32, (maxdeg + 1 + 31) / 32 * 32));
  // layout: [upload: inputs, jobs, item offsets, reconstruction jobs, tile offsets, ids |
  //          compute: images, selections, residues, contents | download: results, info]
  Layout up;
  B.o_jobs = up.take(sizeof(MgJob) * std::max(n, 1));
  B.o_items = up.take(sizeof(int64_t) * (n + 1));
  B.o_crt = up.take(sizeof(Job) * 2 * std::max(n, 1));
  B.o_toff = up.take(sizeof(int64_t) * (n + 1));
  B.o_ids1 = up.take(sizeof(int32_t) * std::max(n, 1));
  B.o_ids2 = up.take(sizeof(int32_t) * std::max(n, 1));
  B.o_in = up.take(sizeof(uint32_t) * std::max<size_t>(in_words, 1));
  B.up_bytes = up.used;
  Layout cmp;
  cmp.used = B.up_bytes;
  B.o_qp.assign(n, 0);
  B.o_dg.assign(n, 0);
  B.o_sel.assign(n, 0);
  B.o_rmod.assign(n, 0);
  B.o_cont.assign(n, 0);
  B.o_cmul.assign(n, 0);
  B.o_cinv.assign(n, 0);
  B.o_h.assign(n, 0);
  for (int j = 0; j < n; ++j) {
    if (B.special[j]) continue;
    const size_t c1 = (size_t)B.cap[j] + 1;
    B.o_qp[j] = cmp.take(sizeof(uint32_t) * (size_t)B.k_total[j] * c1);
    B.o_dg[j] = cmp.take(sizeof(int32_t) * B.k_total[j]);
    B.o_sel[j] = cmp.take(sizeof(int32_t) * B.k_need[j]);
    B.o_rmod[j] = cmp.take(sizeof(uint32_t) * (size_t)B.k_need[j] * c1);
    B.o_cont[j] = cmp.take(sizeof(uint32_t) * B.out_limbs[j]);
    B.o_cmul[j] = cmp.take(sizeof(uint32_t) * B.out_limbs[j]);
    B.o_cinv[j] = cmp.take(sizeof(uint32_t) * B.k_need[j]);
    B.o_h[j] = cmp.take(sizeof(uint32_t) * c1 * B.out_limbs[j]);
  }
  Layout dn;
  dn.used = cmp.used;
  B.dn_start = dn.take(0);
  B.o_out.assign(n, 0);
  B.o_info.assign(n, 0);
  for (int j = 0; j < n; ++j) {
    if (B.special[j]) continue;
    B.o_info[j] = dn.take(sizeof(int32_t) * 4);
    B.o_out[j] = dn.take(sizeof(uint32_t) * ((size_t)B.cap[j] + 1) * B.out_limbs[j]);
  }
  B.total = dn.used;
  B.dn_bytes = B.total - B.dn_start;
  B.special_limbs = sL;
  return 0;
}

int mg_launch(bs_ctx* ctx, MgBatch& B, const bs_upoly* a, const bs_upoly* b, char* base, char* hu,
              char* hd) {
  (void)hd;
  const int n = B.n;
  std::memset(hu, 0, B.up_bytes);
  MgJob* hj = (MgJob*)(hu + B.o_jobs);
  int64_t* items = (int64_t*)(hu + B.o_items);
  Job* hc = (Job*)(hu + B.o_crt);
  int64_t* toff = (int64_t*)(hu + B.o_toff);
  int32_t* ids1 = (int32_t*)(hu + B.o_ids1);
  int32_t* ids2 = (int32_t*)(hu + B.o_ids2);
  uint32_t* in = (uint32_t*)(hu + B.o_in);
  const uint32_t* din = (const uint32_t*)(base + B.o_in);
  size_t pos = 0;
  items[0] = 0;
  toff[0] = 0;
  int m = 0;  // general jobs, compacted
  B.gen.clear();
  for (int j = 0; j < n; ++j) {
    if (B.special[j]) continue;
    const bs_upoly& A = B.swap[j] ? b[j] : a[j];
    const bs_upoly* Bp = B.kind[j] != kMgSqf ? (B.swap[j] ? a + j : b + j) : nullptr;
    MgJob J;
    std::memset(&J, 0, sizeof(J));
    std::memcpy(in + pos, A.c, sizeof(uint32_t) * (size_t)(B.da[j] + 1) * A.limbs);
    J.A = din + pos;
    pos += (size_t)(B.da[j] + 1) * A.limbs;
    J.La = A.limbs;
    J.da = B.da[j];
    if (Bp) {
      std::memcpy(in + pos, Bp->c, sizeof(uint32_t) * (size_t)(B.db[j] + 1) * Bp->limbs);
      J.B = din + pos;
      pos += (size_t)(B.db[j] + 1) * Bp->limbs;
      J.Lb = Bp->limbs;
      J.db = B.db[j];
    } else {
      J.B = nullptr;
      J.Lb = 1;
      J.db = -1;
    }
    J.kind = B.kind[j];
    J.k_total = B.k_total[j];
    J.k_need = B.k_need[j];
    J.cap = B.cap[j];
    J.Lc = B.out_limbs[j];
    J.Qp = (uint32_t*)(base + B.o_qp[j]);
    J.dg = (int32_t*)(base + B.o_dg[j]);
    J.sel = (int32_t*)(base + B.o_sel[j]);
    J.rmod = (uint32_t*)(base + B.o_rmod[j]);
    J.info = (int32_t*)(base + B.o_info[j]);
    J.content = (uint32_t*)(base + B.o_cont[j]);
    J.cmul = (uint32_t*)(base + B.o_cmul[j]);
    J.cinv = (uint32_t*)(base + B.o_cinv[j]);
    J.crt = (Job*)(base + B.o_crt) + 2 * m;
    for (int t = 0; t < 2; ++t) {
      Job& C = hc[2 * m + t];
      std::memset(&C, 0, sizeof(C));
      C.plan.k_need = J.k_need;
      C.plan.k_total = J.k_total;
      C.plan.D = J.cap;  // lowered by the selection kernel
      C.plan.out_limbs = J.Lc;
      C.cap_deg = J.cap;
      C.cap_limbs = J.Lc;
      C.sel = J.sel;
      C.rmod = J.rmod;
      C.out = (uint32_t*)(base + (t == 0 ? B.o_h[j] : B.o_out[j]));
      C.status = J.info + 3;
    }
    hj[m] = J;
    items[m + 1] = items[m] + J.k_total;
    toff[m + 1] = toff[m] + (J.cap + kCrtTile) / kCrtTile;
    ids1[m] = 2 * m;
    ids2[m] = 2 * m + 1;
    B.gen.push_back(j);
    ++m;
  }
  cudaStream_t s = ctx->stream;
  int rc = ctx_cuda(ctx, cudaMemcpyAsync(base, hu, B.up_bytes, cudaMemcpyHostToDevice, s), "upload");
  if (rc) return rc;
  if (m == 0) return 0;
  const Tables Tv = ctx->tabs->view();
  const MgJob* dj = (const MgJob*)(base + B.o_jobs);
  const Job* dc = (const Job*)(base + B.o_crt);
  const WorkList wl_items{nullptr, (const int64_t*)(base + B.o_items), m};
  const WorkList wl1{(const int32_t*)(base + B.o_ids1), (const int64_t*)(base + B.o_toff), m};
  const WorkList wl2{(const int32_t*)(base + B.o_ids2), (const int64_t*)(base + B.o_toff), m};
  const int64_t tiles = toff[m];
  if (B.smem > 48 * 1024 && set_dyn_smem_limit((const void*)k_mg_images, ctx->smem_optin) != 0)
    return ctx_fail(ctx, BS_ERR_CUDA, "shared memory limit");
  const int img_grid = (int)std::min<int64_t>(items[m], (int64_t)8 * ctx->sms);
  k_mg_images<<<img_grid, B.threads, B.smem, s>>>(dj, wl_items, Tv);
  k_mg_select<<<(m + 127) / 128, 128, 0, s>>>(dj, m);
  const int gblocks = std::min(m, 4 * ctx->sms);
  // the gathers: a few jobs still fill the GPU by spreading their rows over blockIdx.y
  const dim3 ggrid(gblocks, std::max(1, std::min(B.kmax, (4 * ctx->sms + gblocks - 1) / gblocks)));
  k_mg_gather<<<ggrid, 256, 0, s>>>(dj, m, Tv, 0);
  const int crt_grid = (int)std::min<int64_t>(tiles, (int64_t)4 * ctx->sms);
  const size_t wsm = crt_warp_smem(B.kmax, B.lmax);
  auto crt = [&](const WorkList& wl) -> int {
    if (B.kmax <= kCrtWarpMaxK && wsm <= (size_t)ctx->smem_optin - 64) {
      launch_crt_w(crt_grid, kCrtTile, wsm, s, dc, wl, Tv, B.kmax, B.lmax);
      return 0;
    }
    const size_t per = (size_t)3 * B.lmax * sizeof(uint32_t);
    const size_t fixed = ((size_t)B.kmax * kCrtTile + 3 * (size_t)B.kmax) * sizeof(uint32_t);
    if (fixed + per > (size_t)ctx->smem_optin - 64) return BS_ERR_RANGE;
    const int w = (int)std::min<size_t>(kCrtWarps, ((size_t)ctx->smem_optin - 64 - fixed) / per);
    launch_crt(crt_grid, w * 32, fixed + per * w, s, dc, wl, Tv, B.kmax, B.lmax, 0);
    return 0;
  };
  if (crt(wl1)) return ctx_fail(ctx, BS_ERR_RANGE, "too many primes for the reconstruction stage");
  const int K = (std::max(B.lmax - 1, B.in_limbs) + 31) / 32;  // <= 8: 256 limbs at most
  {  // one block per job, one warp per 64 coefficients of the longest job (8 at most)
    int maxc = 1;
    for (int j : B.gen) maxc = std::max(maxc, std::max(B.da[j], B.db[j]) + 1);
    const int W = std::min(8, std::max(1, (maxc + 63) / 64));
    const size_t part_words = (size_t)W * std::max(B.lmax, B.in_limbs);
    k_mg_content<<<m, W * 32, part_words * sizeof(uint32_t), s>>>(dj, m, K);
  }
  k_mg_cinv<<<gblocks, 128, 0, s>>>(dj, m, Tv);
  k_mg_gather<<<ggrid, 256, 0, s>>>(dj, m, Tv, 1);
  if (crt(wl2)) return ctx_fail(ctx, BS_ERR_RANGE, "too many primes for the reconstruction stage");
  rc = ctx_cuda(ctx, cudaGetLastError(), "launch");
  if (rc) return rc;
  return ctx_cuda(ctx, cudaMemcpyAsync(hd, base + B.dn_start, B.dn_bytes, cudaMemcpyDeviceToHost, s),
                  "download");
}

int mg_finish(bs_ctx* ctx, const MgBatch& B, const char* hd, bs_upoly* out, int* job_status) {
  int first = 0;
  for (int j = 0; j < B.n; ++j) {
    int st = 0;
    if (B.special[j]) {
      if (B.special_deg[j] < 0) {
        for (int i = 0; i <= out[j].deg; ++i)
          std::memset(out[j].c + (size_t)i * out[j].limbs, 0, sizeof(uint32_t) * out[j].limbs);
        out[j].deg = -1;
      } else {
        st = put_result(ctx, B.special_out[j].data(), B.special_limbs[j], B.special_deg[j], out + j);
      }
    } else {
      const int32_t* info = (const int32_t*)(hd + (B.o_info[j] - B.dn_start));
      st = info[3];
      if (st) {
        ctx_fail(ctx, st, "too few primes agree on the minimal gcd degree");
      } else {
        const uint32_t* src = (const uint32_t*)(hd + (B.o_out[j] - B.dn_start));
        st = put_result(ctx, src, B.out_limbs[j], info[0], out + j);
      }
    }
    if (job_status) job_status[j] = st;
    if (st && !first) first = st;
  }
  return first;
}

// upper bounds of the result shape of job j (for size queries and the serving loop)
void mg_result_shape(const MgBatch& B, int j, int* deg, int* limbs) {
  if (B.special[j]) {
    *deg = B.special_deg[j];
    *limbs = B.special_limbs[j];
  } else {
    *deg = B.cap[j];
    *limbs = B.out_limbs[j];
  }
}

int run_mg(bs_ctx* ctx, int n, const int* kind, const bs_upoly* a, const bs_upoly* b, bs_upoly* out) {
  if (ctx->server) return ctx_fail(ctx, BS_ERR_ARG, "the context runs a serving loop");
  cudaSetDevice(ctx->device);
  MgBatch B;
  int rc = mg_plan(ctx, n, kind, a, b, &B);
  if (rc) return rc;
  bool query = false;
  for (int j = 0; j < n; ++j)
    if (!out[j].c) query = true;
  if (query) {
    for (int j = 0; j < n; ++j) mg_result_shape(B, j, &out[j].deg, &out[j].limbs);
    return BS_OK;
  }
  for (int j = 0; j < n; ++j)
    if (out[j].limbs < 1 || out[j].deg < -1) return ctx_fail(ctx, BS_ERR_ARG, "bad output capacity");
  rc = ctx->tabs->ensure(B.needT, 0, ctx->stream);
  if (rc) return ctx_fail(ctx, rc, "table setup failed");
  rc = ensure_workspace(ctx, B.total);
  if (rc) return rc;
  rc = ensure_pinned(ctx, B.up_bytes, B.dn_bytes);
  if (rc) return rc;
  rc = mg_launch(ctx, B, a, b, (char*)ctx->ws, (char*)ctx->h_up, (char*)ctx->h_down);
  if (rc) return rc;
  rc = ctx_cuda(ctx, cudaStreamSynchronize(ctx->stream), "stream");
  if (rc) return rc;
  return mg_finish(ctx, B, (const char*)ctx->h_down, out, nullptr);
}

}  // namespace bs

using namespace bs;

extern "C" int bs_squarefree_part(bs_ctx* ctx, const bs_upoly* r, bs_upoly* out) {
  if (!ctx) return BS_ERR_ARG;
  if (!r || !out) return ctx_fail(ctx, BS_ERR_ARG, "bad arguments");
  const int kind = kMgSqf;
  return run_mg(ctx, 1, &kind, r, nullptr, out);
}

extern "C" int bs_gcd_z(bs_ctx* ctx, const bs_upoly* a, const bs_upoly* b, bs_upoly* out) {
  if (!ctx) return BS_ERR_ARG;
  if (!a || !b || !out) return ctx_fail(ctx, BS_ERR_ARG, "bad arguments");
  const int kind = kMgGcd;
  return run_mg(ctx, 1, &kind, a, b, out);
}

extern "C" int bs_modgcd_batch(bs_ctx* ctx, int n, const int* kind, const bs_upoly* a,
                               const bs_upoly* b, bs_upoly* out) {
  if (!ctx) return BS_ERR_ARG;
  if (n < 0 || (n && (!kind || !a || !out))) return ctx_fail(ctx, BS_ERR_ARG, "bad arguments");
  if (n == 0) return BS_OK;
  return run_mg(ctx, n, kind, a, b, out);
}
