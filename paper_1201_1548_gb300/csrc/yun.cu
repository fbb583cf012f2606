// Square-free factorisation in Z[x] by Yun's algorithm (Sec. 2.1, BiProject: the
// projected resultant is split into square-free, pairwise coprime factors r_i with
// R = c prod r_i^i), computed modulo many primes and lifted by Chinese remaindering
// (Sec. 5.1, "Computing gcds in Z[x]").
//
// For a prime p with p > deg R and p not dividing lc(R), R mod p has at most as many
// distinct roots as R, with equality exactly when every r_i mod p stays square-free and
// the r_i mod p stay pairwise coprime.  Since deg gcd(R, R') = deg R - (number of distinct
// roots), the primes attaining the minimal deg gcd(R mod p, R' mod p) are those where
// Yun's algorithm over Z_p returns the monic images of the r_i, with the same degree
// sequence (Brown's rule).
//
// Every factor image is scaled to H_i = lc(R) monic(r_i) = (lc(R) / lc(r_i)) r_i, an
// integer polynomial with ||H_i||_inf <= 2^deg(r_i) ||R||_2 (Mignotte's bound for a factor
// of R).  All factors of a job are concatenated and lifted in one reconstruction; the
// content c_i of each H_i is computed on the device (one warp per factor, or the block's
// warps together on each factor when a job has few factors), and a second reconstruction of the
// images H_i (s c_i)^-1, s the sign of lc(R), yields the primitive r_i with positive
// leading coefficients.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <vector>

#include "batch.cuh"
#include "ctx.cuh"
#include "modpoly.cuh"
#include "wbig.cuh"

namespace bs {

struct YunJob {
  const uint32_t* A;  // [(da + 1) * La] limbs of R
  int32_t da, La;
  int32_t k_total, k_need;
  int32_t cap;        // coefficient capacity of the concatenated factors (2 da)
  int32_t Lc;         // limbs of the reconstructed values
  uint32_t* Qp;       // [k_total][cap] images of H_1, H_2, ... (standard form)
  int32_t* dg;        // [k_total] deg gcd(R, R') mod p; -2: p divides lc(R)
  int32_t* ns;        // [k_total] number of factors mod p
  int32_t* sig;       // [k_total][da] factor degrees mod p
  int32_t* sel;       // [k_need] selected table indices
  uint32_t* rmod;     // [k_need][cap] residues handed to the reconstruction
  int32_t* info;      // [0] coefficients - 1, [1] good primes, [2] factors, [3] status
  int32_t* fdeg;      // [da] factor degrees
  int32_t* foff;      // [da + 1] first coefficient of each factor
  uint32_t* content;  // [da][Lc] content of H_i
  uint32_t* cinv;     // [da][k_need] (s c_i)^-1 mod p (Montgomery form)
  Job* crt;           // [2] reconstructions of the H_i and of the r_i
};

// ---- images: one block per (job, prime) -----------------------------------------------
// Shared memory: F, D, X, Y of deg R + 1 words each.  F holds R and then the running b,
// D holds R' and then the running c and d (both at the offset of the divisors removed so
// far: the in-place quotient of a division by a degree-e divisor starts at index e), X and
// Y are the gcd's working copies.
__global__ void k_yun_images(const YunJob* jobs, WorkList wl, Tables T) {
  extern __shared__ uint32_t sm[];
  __shared__ int s_top;
  const int64_t total = wl.off[wl.n];
  for (int64_t item = blockIdx.x; item < total; item += gridDim.x) {
    const int ji = find_item(wl.off, wl.n, item);
    const YunJob& J = jobs[ji];
    const int q = (int)(item - wl.off[ji]);
    const PrimeConst pc = T.pc[q];
    const Mod M{pc.p, pc.pinv};
    const uint32_t* pw = T.pw + (int64_t)q * (kMaxLimbs + 1);
    const uint32_t* mpw = T.mpw + (int64_t)q * (kMaxLimbs + 1);
    const int n = J.da;
    uint32_t* F = sm;
    uint32_t* D = F + (n + 1);
    uint32_t* X = D + (n + 1);
    uint32_t* Y = X + (n + 1);
    for (int i = threadIdx.x; i <= n; i += blockDim.x) {
      const uint32_t v = reduce_coef(J.A + (int64_t)i * J.La, J.La, pw, mpw, pc);
      F[i] = v;
      X[i] = v;
    }
    __syncthreads();
    const uint32_t lcR = F[n];
    if (lcR == 0u) {  // the prime divides lc(R)
      if (threadIdx.x == 0) {
        J.dg[q] = -2;
        J.ns[q] = 0;
      }
      __syncthreads();
      continue;
    }
    // R'_i = (i + 1) R_{i+1}; its degree is n - 1 because p > n
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
      const uint32_t v = mmul(F[i + 1], redc((uint64_t)(uint32_t)(i + 1) * pc.r2, M.p, M.pinv), M);
      D[i] = v;
      Y[i] = v;
    }
    __syncthreads();
    int e0;
    uint32_t* G = smem_euclid(X, n, Y, n - 1, M, &e0, &s_top);
    {
      const uint32_t ilc = minv(G[e0], pc.one_m, M);
      for (int i = threadIdx.x; i <= e0; i += blockDim.x) G[i] = mmul(G[i], ilc, M);
      __syncthreads();
    }
    // b = R / G, c = R' / G
    smem_div2(F, n, D, n - 1, G, e0, M);
    uint32_t* b = F + e0;
    int nb = n - e0;
    uint32_t* d = D + e0;
    // d = c - b' (c has degree nb - 1)
    for (int i = threadIdx.x; i < nb; i += blockDim.x)
      d[i] = msub(d[i], mmul(b[i + 1], redc((uint64_t)(uint32_t)(i + 1) * pc.r2, M.p, M.pinv), M), M.p);
    __syncthreads();
    if (threadIdx.x == 0) {
      int l = nb - 1;
      while (l >= 0 && d[l] == 0u) --l;
      s_top = l;
    }
    __syncthreads();
    int nd = s_top;
    __syncthreads();
    uint32_t* Qo = J.Qp + (int64_t)q * J.cap;
    int32_t* sg = J.sig + (int64_t)q * n;
    int pos = 0, s = 0;
    // b loses at least one degree every step once only factors of multiplicity > s are
    // left; Yun's sequence ends after at most n steps over a field of characteristic > n
    while (nb > 0 && s < n) {
      for (int i = threadIdx.x; i <= nb; i += blockDim.x) X[i] = b[i];
      for (int i = threadIdx.x; i <= nd; i += blockDim.x) Y[i] = d[i];
      __syncthreads();
      int ea;
      uint32_t* A = smem_euclid(X, nb, Y, nd, M, &ea, &s_top);  // gcd(b, 0) = b
      if (pos + ea + 1 > J.cap) break;  // sum (deg a_i + 1) <= 2 deg R; kept as a guard
      const uint32_t ilc = minv(A[ea], pc.one_m, M);
      const uint32_t scale = mmul(ilc, lcR, M);
      for (int i = threadIdx.x; i <= ea; i += blockDim.x) {
        const uint32_t v = A[i];
        Qo[pos + i] = redc((uint64_t)mmul(v, scale, M), M.p, M.pinv);
        A[i] = mmul(v, ilc, M);
      }
      if (threadIdx.x == 0) sg[s] = ea;
      __syncthreads();
      pos += ea + 1;
      ++s;
      // b = b / a, c = d / a (d = 0 gives c = 0)
      smem_div2(b, nb, d, nd, A, ea, M);
      b += ea;
      nb -= ea;
      const int nc = nd >= ea ? nd - ea : -1;
      d += ea;
      // d = c - b'
      for (int i = threadIdx.x; i < nb; i += blockDim.x) {
        const uint32_t ci = (i <= nc) ? d[i] : 0u;
        d[i] = msub(ci, mmul(b[i + 1], redc((uint64_t)(uint32_t)(i + 1) * pc.r2, M.p, M.pinv), M), M.p);
      }
      __syncthreads();
      if (threadIdx.x == 0) {
        int l = nb - 1;
        while (l >= 0 && d[l] == 0u) --l;
        s_top = l;
      }
      __syncthreads();
      nd = s_top;
      __syncthreads();
    }
    if (threadIdx.x == 0) {
      J.dg[q] = (nb > 0) ? -3 : e0;  // -3: the sequence did not end (not for p > n)
      J.ns[q] = s;
    }
    __syncthreads();
  }
}

// ---- selection: one thread per job ------------------------------------------------------
__global__ void k_yun_select(const YunJob* jobs, int n) {
  const int ji = blockIdx.x * blockDim.x + threadIdx.x;
  if (ji >= n) return;
  const YunJob& J = jobs[ji];
  int mind = 1 << 30;
  for (int q = 0; q < J.k_total; ++q)
    if (J.dg[q] >= 0 && J.dg[q] < mind) mind = J.dg[q];
  int r = 0;
  for (int q = 0; q < J.k_total && r < J.k_need; ++q)
    if (J.dg[q] == mind) J.sel[r++] = q;
  int status = (r == J.k_need) ? 0 : kErrUnlucky;
  int s = 0, tot = 0;
  if (status == 0) {
    const int q0 = J.sel[0];
    s = J.ns[q0];
    const int32_t* sg0 = J.sig + (int64_t)q0 * J.da;
    // primes with the minimal gcd degree share the degree sequence of the true factors
    for (int t = 1; t < r && status == 0; ++t) {
      const int qt = J.sel[t];
      if (J.ns[qt] != s) status = kErrUnlucky;
      const int32_t* sgt = J.sig + (int64_t)qt * J.da;
      for (int i = 0; i < s && status == 0; ++i)
        if (sgt[i] != sg0[i]) status = kErrUnlucky;
    }
    for (int i = 0; i < s; ++i) {
      J.fdeg[i] = sg0[i];
      J.foff[i] = tot;
      tot += sg0[i] + 1;
    }
    J.foff[s] = tot;
  }
  if (status) {
    s = 0;
    tot = 0;
  }
  J.info[0] = tot - 1;
  J.info[1] = r;
  J.info[2] = s;
  J.info[3] = status;
  for (int t = 0; t < 2; ++t) {
    J.crt[t].plan.D = status ? 0 : tot - 1;
    J.crt[t].plan.status = status;
  }
}

__device__ __forceinline__ int factor_of(const int32_t* foff, int s, int i) {
  int lo = 0, hi = s - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (foff[mid] <= i)
      lo = mid;
    else
      hi = mid - 1;
  }
  return lo;
}

// ---- residues for a reconstruction: blocks over jobs and their selected primes ----------
// second = 0: images of the H_i; second = 1: images of H_i (s c_i)^-1
// blockIdx.x strides over the jobs, blockIdx.y over a job's selected primes (rows)
__global__ void k_yun_gather(const YunJob* jobs, int n, Tables T, int second) {
  for (int ji = blockIdx.x; ji < n; ji += gridDim.x) {
    const YunJob& J = jobs[ji];
    if (J.info[3] != 0) continue;
    const int cnt1 = J.info[0] + 1;
    const int s = J.info[2];
    for (int r = blockIdx.y; r < J.k_need; r += gridDim.y) {
      const int q = J.sel[r];
      const uint32_t* src = J.Qp + (int64_t)q * J.cap;
      uint32_t* dst = J.rmod + (int64_t)r * cnt1;
      if (second) {  // standard form times Montgomery form gives standard form
        const PrimeConst pc = T.pc[q];
        for (int i = threadIdx.x; i < cnt1; i += blockDim.x) {
          const int f = factor_of(J.foff, s, i);
          dst[i] = redc((uint64_t)src[i] * J.cinv[(int64_t)f * J.k_need + r], pc.p, pc.pinv);
        }
      } else {
        for (int i = threadIdx.x; i < cnt1; i += blockDim.x) dst[i] = src[i];
      }
    }
  }
}

// ---- contents: block per job, one warp per factor or all warps on each factor -----------
template <int K>
__device__ void yun_content_factor(const YunJob& J, int f) {
  ContentAcc<K> h;
  h.fold(J.crt[0].out + (int64_t)J.foff[f] * J.Lc, J.fdeg[f] + 1, J.Lc);
  h.store(J.content + (int64_t)f * J.Lc, J.Lc);
}

// one warp per factor when the job has at least as many factors as the block has warps;
// otherwise the factors one after the other, each by all warps (block_content)
template <int K>
__device__ void yun_content_job(const YunJob& J, uint32_t* part) {
  const int s = J.info[2], warps = blockDim.x >> 5;
  if (s >= warps) {
    for (int f = threadIdx.x >> 5; f < s; f += warps) yun_content_factor<K>(J, f);
    return;
  }
  for (int f = 0; f < s; ++f)
    block_content<K>(J.crt[0].out + (int64_t)J.foff[f] * J.Lc, J.fdeg[f] + 1, J.Lc, nullptr, 0, 1, part, J.Lc,
                     J.content + (int64_t)f * J.Lc, J.Lc);
}

// dynamic shared memory: (blockDim.x / 32) * Lc words for the partial gcds
__global__ void __launch_bounds__(256) k_yun_content(const YunJob* jobs, int n, int K) {
  extern __shared__ uint32_t yun_part[];
  for (int ji = blockIdx.x; ji < n; ji += gridDim.x) {
    const YunJob& J = jobs[ji];
    if (J.info[3] != 0) continue;
    if (K <= 1)
      yun_content_job<1>(J, yun_part);
    else if (K <= 2)
      yun_content_job<2>(J, yun_part);
    else if (K <= 4)
      yun_content_job<4>(J, yun_part);
    else
      yun_content_job<8>(J, yun_part);
  }
}

// ---- per (factor, selected prime): (s c_i)^-1 mod p -------------------------------------
__global__ void k_yun_cinv(const YunJob* jobs, int n, Tables T) {
  for (int ji = blockIdx.x; ji < n; ji += gridDim.x) {
    const YunJob& J = jobs[ji];
    if (J.info[3] != 0) continue;
    const bool neg = (J.A[(int64_t)J.da * J.La + J.La - 1] >> 31) != 0;
    const int cnt = J.info[2] * J.k_need;
    for (int t = threadIdx.x; t < cnt; t += blockDim.x) {
      const int f = t / J.k_need;
      const int r = t - f * J.k_need;
      const PrimeConst pc = T.pc[J.sel[r]];
      const Mod M{pc.p, pc.pinv};
      uint32_t c = mag_mod(J.content + (int64_t)f * J.Lc, J.Lc, pc.p);
      if (neg) c = mneg(c, pc.p);
      const uint32_t c_m = redc((uint64_t)c * pc.r2, M.p, M.pinv);
      J.cinv[t] = minv(c_m, pc.one_m, M);
    }
  }
}

// ---- host side ---------------------------------------------------------------------------
struct YunBatch {
  int n = 0;
  std::vector<int> da, k_need, k_total, cap, out_limbs;
  int kmax = 1, lmax = 1, needT = 1;
  int64_t items = 0;
  size_t smem = 0;
  int threads = 32;
  size_t o_jobs = 0, o_items = 0, o_crt = 0, o_toff = 0, o_ids1 = 0, o_ids2 = 0, o_in = 0;
  size_t up_bytes = 0;
  std::vector<size_t> o_qp, o_dg, o_ns, o_sig, o_sel, o_rmod, o_foff, o_cont, o_cinv, o_h;
  std::vector<size_t> o_info, o_fdeg, o_out;
  size_t dn_start = 0, dn_bytes = 0, total = 0;
};

static int yun_plan(bs_ctx* ctx, int n, const bs_upoly* r, YunBatch* ybp) {
  YunBatch& B = *ybp;
  B = YunBatch{};
  B.n = n;
  const HostPrimes& H = host_primes();
  const int T = (int)H.p.size();
  B.da.assign(n, -1);
  B.k_need.assign(n, 0);
  B.k_total.assign(n, 0);
  B.cap.assign(n, 0);
  B.out_limbs.assign(n, 1);
  int maxdeg = 0;
  size_t in_words = 0;
  for (int j = 0; j < n; ++j) {
    const bs_upoly& u = r[j];
    if (u.deg < -1 || u.limbs < 1 || u.limbs > kMaxUniLimbs || (u.deg >= 0 && !u.c))
      return ctx_fail(ctx, BS_ERR_ARG, "bad polynomial");
    const int da = trimmed_degree(u);
    if (da < 0) return ctx_fail(ctx, BS_ERR_ZERO, "square-free factorisation of the zero polynomial");
    B.da[j] = da;
    if (da == 0) continue;  // a constant: no factors
    const int64_t l2 = log2_norm2_q16(u, da);
    const int64_t bits = (int64_t)da + (l2 + 65535) / 65536 + 1;  // |H_i| < 2^bits
    const int64_t need = (bits + 2) * 65536;
    if (H.lg_prefix[T] < need) return ctx_fail(ctx, BS_ERR_RANGE, "bound exceeds the prime table");
    if ((bits + 2 + 31) / 32 > 256) return ctx_fail(ctx, BS_ERR_RANGE, "coefficients above 8192 bits");
    const int k = std::max(1, prime_count_host(H.lg_prefix.data(), T, need));
    const int kt = std::min(T, k + 4 + k / 8 + lc_bits(u, da) / 30);
    B.k_need[j] = k;
    B.k_total[j] = kt;
    B.cap[j] = 2 * da;
    B.out_limbs[j] = (int)((bits + 2 + 31) / 32);
    B.kmax = std::max(B.kmax, k);
    B.lmax = std::max(B.lmax, B.out_limbs[j] + 1);
    B.needT = std::max(B.needT, kt);
    B.smem = std::max(B.smem, (size_t)4 * (da + 1) * sizeof(uint32_t));
    maxdeg = std::max(maxdeg, da);
    in_words += (size_t)(da + 1) * u.limbs;
    B.items += kt;
  }
  if (B.smem > (size_t)ctx->smem_optin - 64)
    return ctx_fail(ctx, BS_ERR_RANGE, "degree too large for one block's shared memory");
  B.threads = std::min(256, std::max(32, (maxdeg + 1 + 31) / 32 * 32));
  // layout: [upload: jobs, item offsets, reconstruction jobs, tile offsets, ids, inputs |
  //          compute: images, selections, residues, contents | download: info, degrees, results]
  Layout up;
  B.o_jobs = up.take(sizeof(YunJob) * std::max(n, 1));
  B.o_items = up.take(sizeof(int64_t) * (n + 1));
  B.o_crt = up.take(sizeof(Job) * 2 * std::max(n, 1));
  B.o_toff = up.take(sizeof(int64_t) * (n + 1));
  B.o_ids1 = up.take(sizeof(int32_t) * std::max(n, 1));
  B.o_ids2 = up.take(sizeof(int32_t) * std::max(n, 1));
  B.o_in = up.take(sizeof(uint32_t) * std::max<size_t>(in_words, 1));
  B.up_bytes = up.used;
  Layout cmp;
  cmp.used = B.up_bytes;
  for (auto* v : {&B.o_qp, &B.o_dg, &B.o_ns, &B.o_sig, &B.o_sel, &B.o_rmod, &B.o_foff, &B.o_cont,
                  &B.o_cinv, &B.o_h, &B.o_info, &B.o_fdeg, &B.o_out})
    v->assign(n, 0);
  for (int j = 0; j < n; ++j) {
    if (B.da[j] < 1) continue;
    const size_t cap = (size_t)B.cap[j], da = (size_t)B.da[j], kt = (size_t)B.k_total[j];
    const size_t kn = (size_t)B.k_need[j], L = (size_t)B.out_limbs[j];
    B.o_qp[j] = cmp.take(sizeof(uint32_t) * kt * cap);
    B.o_dg[j] = cmp.take(sizeof(int32_t) * kt);
    B.o_ns[j] = cmp.take(sizeof(int32_t) * kt);
    B.o_sig[j] = cmp.take(sizeof(int32_t) * kt * da);
    B.o_sel[j] = cmp.take(sizeof(int32_t) * kn);
    B.o_rmod[j] = cmp.take(sizeof(uint32_t) * kn * cap);
    B.o_foff[j] = cmp.take(sizeof(int32_t) * (da + 1));
    B.o_cont[j] = cmp.take(sizeof(uint32_t) * da * L);
    B.o_cinv[j] = cmp.take(sizeof(uint32_t) * da * kn);
    B.o_h[j] = cmp.take(sizeof(uint32_t) * cap * L);
  }
  Layout dn;
  dn.used = cmp.used;
  B.dn_start = dn.take(0);
  for (int j = 0; j < n; ++j) {
    if (B.da[j] < 1) continue;
    B.o_info[j] = dn.take(sizeof(int32_t) * 4);
    B.o_fdeg[j] = dn.take(sizeof(int32_t) * B.da[j]);
    B.o_out[j] = dn.take(sizeof(uint32_t) * (size_t)B.cap[j] * B.out_limbs[j]);
  }
  B.total = dn.used;
  B.dn_bytes = B.total - B.dn_start;
  return 0;
}

static int yun_launch(bs_ctx* ctx, YunBatch& B, const bs_upoly* r, char* base, char* hu) {
  const int n = B.n;
  std::memset(hu, 0, B.up_bytes);
  YunJob* hj = (YunJob*)(hu + B.o_jobs);
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
  int m = 0;  // jobs that run on the device, compacted
  for (int j = 0; j < n; ++j) {
    if (B.da[j] < 1) continue;
    const bs_upoly& u = r[j];
    YunJob J;
    std::memset(&J, 0, sizeof(J));
    std::memcpy(in + pos, u.c, sizeof(uint32_t) * (size_t)(B.da[j] + 1) * u.limbs);
    J.A = din + pos;
    pos += (size_t)(B.da[j] + 1) * u.limbs;
    J.da = B.da[j];
    J.La = u.limbs;
    J.k_total = B.k_total[j];
    J.k_need = B.k_need[j];
    J.cap = B.cap[j];
    J.Lc = B.out_limbs[j];
    J.Qp = (uint32_t*)(base + B.o_qp[j]);
    J.dg = (int32_t*)(base + B.o_dg[j]);
    J.ns = (int32_t*)(base + B.o_ns[j]);
    J.sig = (int32_t*)(base + B.o_sig[j]);
    J.sel = (int32_t*)(base + B.o_sel[j]);
    J.rmod = (uint32_t*)(base + B.o_rmod[j]);
    J.info = (int32_t*)(base + B.o_info[j]);
    J.fdeg = (int32_t*)(base + B.o_fdeg[j]);
    J.foff = (int32_t*)(base + B.o_foff[j]);
    J.content = (uint32_t*)(base + B.o_cont[j]);
    J.cinv = (uint32_t*)(base + B.o_cinv[j]);
    J.crt = (Job*)(base + B.o_crt) + 2 * m;
    for (int t = 0; t < 2; ++t) {
      Job& C = hc[2 * m + t];
      std::memset(&C, 0, sizeof(C));
      C.plan.k_need = J.k_need;
      C.plan.k_total = J.k_total;
      C.plan.D = J.cap - 1;  // lowered by the selection kernel
      C.plan.out_limbs = J.Lc;
      C.cap_deg = J.cap - 1;
      C.cap_limbs = J.Lc;
      C.sel = J.sel;
      C.rmod = J.rmod;
      C.out = (uint32_t*)(base + (t == 0 ? B.o_h[j] : B.o_out[j]));
      C.status = J.info + 3;
    }
    hj[m] = J;
    items[m + 1] = items[m] + J.k_total;
    toff[m + 1] = toff[m] + (J.cap - 1 + kCrtTile) / kCrtTile;
    ids1[m] = 2 * m;
    ids2[m] = 2 * m + 1;
    ++m;
  }
  cudaStream_t s = ctx->stream;
  int rc = ctx_cuda(ctx, cudaMemcpyAsync(base, hu, B.up_bytes, cudaMemcpyHostToDevice, s), "upload");
  if (rc || m == 0) return rc;
  const Tables Tv = ctx->tabs->view();
  const YunJob* dj = (const YunJob*)(base + B.o_jobs);
  const Job* dc = (const Job*)(base + B.o_crt);
  const WorkList wl_items{nullptr, (const int64_t*)(base + B.o_items), m};
  const WorkList wl1{(const int32_t*)(base + B.o_ids1), (const int64_t*)(base + B.o_toff), m};
  const WorkList wl2{(const int32_t*)(base + B.o_ids2), (const int64_t*)(base + B.o_toff), m};
  if (B.smem > 48 * 1024 && set_dyn_smem_limit((const void*)k_yun_images, ctx->smem_optin) != 0)
    return ctx_fail(ctx, BS_ERR_CUDA, "shared memory limit");
  const int img_grid = (int)std::min<int64_t>(items[m], (int64_t)8 * ctx->sms);
  k_yun_images<<<img_grid, B.threads, B.smem, s>>>(dj, wl_items, Tv);
  k_yun_select<<<(m + 127) / 128, 128, 0, s>>>(dj, m);
  const int gblocks = std::min(m, 4 * ctx->sms);
  // the gathers: a few jobs still fill the GPU by spreading their rows over blockIdx.y
  const dim3 ggrid(gblocks, std::max(1, std::min(B.kmax, (4 * ctx->sms + gblocks - 1) / gblocks)));
  k_yun_gather<<<ggrid, 256, 0, s>>>(dj, m, Tv, 0);
  const int crt_grid = (int)std::min<int64_t>(toff[m], (int64_t)4 * ctx->sms);
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
  const int K = (B.lmax - 1 + 31) / 32;  // <= 8: out_limbs <= 256
  k_yun_content<<<gblocks, 256, (size_t)8 * B.lmax * sizeof(uint32_t), s>>>(dj, m, K);
  k_yun_cinv<<<gblocks, 128, 0, s>>>(dj, m, Tv);
  k_yun_gather<<<ggrid, 256, 0, s>>>(dj, m, Tv, 1);
  if (crt(wl2)) return ctx_fail(ctx, BS_ERR_RANGE, "too many primes for the reconstruction stage");
  rc = ctx_cuda(ctx, cudaGetLastError(), "launch");
  if (rc) return rc;
  return ctx_cuda(ctx, cudaMemcpyAsync(ctx->h_down, base + B.dn_start, B.dn_bytes, cudaMemcpyDeviceToHost, s),
                  "download");
}

static int yun_finish(bs_ctx* ctx, const YunBatch& B, const char* hd, int cap_factors, int32_t* fdeg,
                      int32_t* nfac, bs_upoly* out) {
  int first = 0;
  for (int j = 0; j < B.n; ++j) {
    int st = 0;
    int32_t* fd = fdeg + (size_t)j * cap_factors;
    nfac[j] = 0;
    if (B.da[j] == 0) {  // a constant has no factors
      for (int i = 0; i <= out[j].deg; ++i)
        std::memset(out[j].c + (size_t)i * out[j].limbs, 0, sizeof(uint32_t) * out[j].limbs);
      out[j].deg = -1;
    } else {
      const int32_t* info = (const int32_t*)(hd + (B.o_info[j] - B.dn_start));
      st = info[3];
      if (st) {
        ctx_fail(ctx, st, "too few primes agree on the minimal gcd degree");
      } else if (info[2] > cap_factors) {
        st = ctx_fail(ctx, BS_ERR_CAPACITY, "factor capacity too small");
      } else {
        const int32_t* dsrc = (const int32_t*)(hd + (B.o_fdeg[j] - B.dn_start));
        const uint32_t* src = (const uint32_t*)(hd + (B.o_out[j] - B.dn_start));
        st = put_result(ctx, src, B.out_limbs[j], info[0], out + j);
        if (!st) {
          nfac[j] = info[2];
          std::memcpy(fd, dsrc, sizeof(int32_t) * info[2]);
        }
      }
    }
    if (st && !first) first = st;
  }
  return first;
}

static int run_yun(bs_ctx* ctx, int n, const bs_upoly* r, int cap_factors, int32_t* fdeg, int32_t* nfac,
                   bs_upoly* out) {
  if (ctx->server) return ctx_fail(ctx, BS_ERR_ARG, "the context runs a serving loop");
  cudaSetDevice(ctx->device);
  YunBatch B;
  int rc = yun_plan(ctx, n, r, &B);
  if (rc) return rc;
  bool query = false;
  for (int j = 0; j < n; ++j)
    if (!out[j].c) query = true;
  if (query) {  // upper bounds: deg R factors, 2 deg R coefficients
    for (int j = 0; j < n; ++j) {
      out[j].deg = B.da[j] < 1 ? -1 : B.cap[j] - 1;
      out[j].limbs = B.out_limbs[j];
      nfac[j] = std::max(B.da[j], 0);
    }
    return BS_OK;
  }
  if (cap_factors < 0 || (cap_factors > 0 && !fdeg)) return ctx_fail(ctx, BS_ERR_ARG, "bad factor capacity");
  for (int j = 0; j < n; ++j)
    if (out[j].limbs < 1 || out[j].deg < -1) return ctx_fail(ctx, BS_ERR_ARG, "bad output capacity");
  rc = ctx->tabs->ensure(B.needT, 0, ctx->stream);
  if (rc) return ctx_fail(ctx, rc, "table setup failed");
  rc = ensure_workspace(ctx, B.total);
  if (rc) return rc;
  rc = ensure_pinned(ctx, B.up_bytes, B.dn_bytes);
  if (rc) return rc;
  rc = yun_launch(ctx, B, r, (char*)ctx->ws, (char*)ctx->h_up);
  if (rc) return rc;
  rc = ctx_cuda(ctx, cudaStreamSynchronize(ctx->stream), "stream");
  if (rc) return rc;
  return yun_finish(ctx, B, (const char*)ctx->h_down, cap_factors, fdeg, nfac, out);
}

}  // namespace bs

using namespace bs;

extern "C" int bs_squarefree_factorization(bs_ctx* ctx, const bs_upoly* r, int cap_factors, int32_t* fdeg,
                                           int32_t* nfac, bs_upoly* out) {
  if (!ctx) return BS_ERR_ARG;
  if (!r || !out || !nfac) return ctx_fail(ctx, BS_ERR_ARG, "bad arguments");
  return run_yun(ctx, 1, r, cap_factors, fdeg, nfac, out);
}

extern "C" int bs_squarefree_factorization_batch(bs_ctx* ctx, int n, const bs_upoly* r, int cap_factors,
                                                 int32_t* fdeg, int32_t* nfac, bs_upoly* out) {
  if (!ctx) return BS_ERR_ARG;
  if (n < 0 || (n && (!r || !out || !nfac))) return ctx_fail(ctx, BS_ERR_ARG, "bad arguments");
  if (n == 0) return BS_OK;
  return run_yun(ctx, n, r, cap_factors, fdeg, nfac, out);
}
