// Weighted-sum reconstruction for many primes (step (e) of Sec. 5.1, for k_need above
// what one warp per coefficient stages in shared memory).
//
// With P = p_0 ... p_{k-1} (the first k table primes), M_j = P / p_j, y_j = M_j^-1 mod p_j
// and t_j = r_j y_j mod p_j for the residues r_j of a coefficient c,
//   c = sum_j t_j M_j - q P,   q = round(sum_j t_j / p_j),
// exactly (|c| < P / 4).  Three kernels per batch:
//   k_bigcrt_tables  one thread per prime: M_j by long division of P, y_j
//   k_bigcrt_gemm    C[i][l] = sum_j t_ij M_j[l] as 96-bit column sums, tiles of
//                    32 coefficients x 64 limbs stepping through the primes 32 at a time
//                    (t computed from the residues while staging)
//   k_bigcrt_carry   one warp per coefficient: q from sum_j t_j floor(2^62 / p_j), the
//                    carries of the column sums and the subtraction of q P, in limbs
// Jobs whose selected primes are not the first k of the table (a prime was rejected) are
// left to the block Garner kernel.
#include <cuda_runtime.h>

#include "ballot.cuh"
#include "common.cuh"
#include "resultant_kernels.cuh"

namespace bs {

__device__ __forceinline__ bool table_ordered(const Job* J, int k) { return J->sel[k - 1] == k - 1; }

// ---- tables: M_j = P / p_j (wsL limbs) and y_j -----------------------------------------
__global__ void __launch_bounds__(kBigTabThreads) k_bigcrt_tables(const Job* jobs, WorkList wl,
                                                                   Tables T) {
  pdl_wait();
  const int64_t total = wl.off[wl.n];
  for (int64_t item = blockIdx.x; item < total; item += gridDim.x) {
    const int ji = find_item(wl.off, wl.n, item);
    const Job* J = jobs + (wl.ids ? wl.ids[ji] : ji);
    const Plan& P = J->plan;
    const int k = P.k_need;
    if (P.status != 0 || P.trivial != 0 || !table_ordered(J, k)) continue;
    const int j = (int)(item - wl.off[ji]) * kBigTabThreads + threadIdx.x;
    if (j >= k) continue;
    const int L = J->wsL;
    const uint32_t* Pk = T.pp + (int64_t)k * T.LPP;
    const uint32_t p = T.pc[j].p;
    uint32_t* Mj = J->wsM + (int64_t)j * L;
    uint64_t rem = 0;
    for (int l = L - 1; l >= 0; --l) {  // exact long division, most significant limb first
      const uint64_t cur = (rem << 32) | (l < T.LPP ? Pk[l] : 0u);
      Mj[l] = (uint32_t)(cur / p);
      rem = cur % p;
    }
    // y_j = (prod_{i != j} p_i)^-1 mod p_j, Montgomery form
    const PrimeConst pc = T.pc[j];
    const Mod M{pc.p, pc.pinv};
    uint32_t prod = pc.one_m;
    for (int i = 0; i < k; ++i) {
      if (i == j) continue;
      const uint32_t pi = T.pc[i].p % p;
      prod = mmul(prod, redc((uint64_t)pi * pc.r2, p, pc.pinv), M);
    }
    J->wsY[j] = minv(prod, pc.one_m, M);
  }
  pdl_trigger();
}

// ---- C[i][l] = sum_j t_ij M_j[l] ------------------------------------------------------------
__global__ void __launch_bounds__(256) k_bigcrt_gemm(const Job* jobs, WorkList wl, Tables T) {
  pdl_wait();
  __shared__ uint32_t sT[kBigGJ][kBigGI];
  __shared__ uint32_t sM[kBigGJ][kBigGL];
  const int tid = threadIdx.x;
  const int r = tid >> 4;   // coefficients r, r + 16 of the tile
  const int c = tid & 15;   // limbs c, c + 16, c + 32, c + 48 of the tile
  const int64_t total = wl.off[wl.n];
  for (int64_t item = blockIdx.x; item < total; item += gridDim.x) {
    const int ji = find_item(wl.off, wl.n, item);
    const Job* J = jobs + (wl.ids ? wl.ids[ji] : ji);
    const Plan& P = J->plan;
    const int k = P.k_need;
    if (P.status != 0 || P.trivial != 0 || !table_ordered(J, k)) continue;  // uniform
    const int L = J->wsL, D = P.D;
    const int nlb = (L + kBigGL - 1) / kBigGL;
    const int local = (int)(item - wl.off[ji]);
    const int i0 = (local / nlb) * kBigGI, l0 = (local % nlb) * kBigGL;
    if (i0 > D) continue;  // above the degree: nothing to sum (uniform)
    uint64_t lo[2][4] = {};
    uint32_t hi[2][4] = {};
    for (int j0 = 0; j0 < k; j0 += kBigGJ) {
      __syncthreads();
      for (int e = tid; e < kBigGJ * kBigGI; e += blockDim.x) {
        const int jj = e / kBigGI, ii = e % kBigGI;
        const int j = j0 + jj, i = i0 + ii;
        uint32_t t = 0;
        if (j < k && i <= D) {
          const PrimeConst pc = T.pc[j];
          const Mod M{pc.p, pc.pinv};
          // standard form times Montgomery form: standard form
          t = mmul(J->rmod[(int64_t)j * (D + 1) + i], J->wsY[j], M);
        }
        sT[jj][ii] = t;
      }
      for (int e = tid; e < kBigGJ * kBigGL; e += blockDim.x) {
        const int jj = e / kBigGL, ll = e % kBigGL;
        const int j = j0 + jj, l = l0 + ll;
        sM[jj][ll] = (j < k && l < L) ? J->wsM[(int64_t)j * L + l] : 0u;
      }
      __syncthreads();
#pragma unroll 4
      for (int jj = 0; jj < kBigGJ; ++jj) {
        const uint32_t a0 = sT[jj][r], a1 = sT[jj][r + 16];
#pragma unroll
        for (int m = 0; m < 4; ++m) {
          const uint32_t b = sM[jj][c + 16 * m];
          const uint64_t p0 = (uint64_t)a0 * b, p1 = (uint64_t)a1 * b;
          const uint64_t s0 = lo[0][m] + p0, s1 = lo[1][m] + p1;
          hi[0][m] += (s0 < p0) ? 1u : 0u;
          hi[1][m] += (s1 < p1) ? 1u : 0u;
          lo[0][m] = s0;
          lo[1][m] = s1;
        }
      }
    }
    const int64_t plane = (int64_t)(J->cap_deg + 1) * L;
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int i = i0 + r + 16 * h;
      if (i > D) continue;
#pragma unroll
      for (int m = 0; m < 4; ++m) {
        const int l = l0 + c + 16 * m;
        if (l >= L) continue;
        uint32_t* S = J->wsS + (int64_t)i * L + l;
        S[0] = (uint32_t)lo[h][m];
        S[plane] = (uint32_t)(lo[h][m] >> 32);
        S[2 * plane] = hi[h][m];
      }
    }
  }
  pdl_trigger();
}

// ---- carries, q P, two's complement: one warp per coefficient ----------------------------
__global__ void __launch_bounds__(kBigCarryWarps * 32) k_bigcrt_carry(const Job* jobs, WorkList wl,
                                                                       Tables T) {
  pdl_wait();
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t total = wl.off[wl.n];
  for (int64_t item = blockIdx.x; item < total; item += gridDim.x) {
    const int ji = find_item(wl.off, wl.n, item);
    const Job* J = jobs + (wl.ids ? wl.ids[ji] : ji);
    const Plan& P = J->plan;
    const int k = P.k_need;
    const int cap = J->cap_limbs;
    const int i = (int)(item - wl.off[ji]) * kBigCarryWarps + warp;
    if (i > J->cap_deg) continue;
    uint32_t* out = J->out + (int64_t)i * cap;
    if (P.status != 0 || P.trivial != 0 || i > P.D) {
      for (int l = lane; l < cap; l += 32)
        out[l] = (P.status == 0 && P.trivial == 2 && i == 0 && l == 0) ? 1u : 0u;
      continue;
    }
    if (!table_ordered(J, k)) continue;  // the block Garner kernel writes this job
    const int L = J->wsL, D = P.D;
    // q = round(sum_j t_j floor(2^62 / p_j) / 2^62)
    uint64_t flo = 0;
    uint32_t fhi = 0;
    for (int j = lane; j < k; j += 32) {
      const PrimeConst pc = T.pc[j];
      const Mod M{pc.p, pc.pinv};
      const uint32_t t = mmul(J->rmod[(int64_t)j * (D + 1) + i], J->wsY[j], M);
      const uint64_t prod = (uint64_t)t * T.q62[j];
      flo += prod;
      fhi += (flo < prod) ? 1u : 0u;
    }
#pragma unroll
    for (int x = 16; x > 0; x >>= 1) {
      const uint64_t olo = __shfl_xor_sync(0xffffffffu, flo, x);
      const uint32_t ohi = __shfl_xor_sync(0xffffffffu, fhi, x);
      const uint64_t nlo = flo + olo;
      fhi = fhi + ohi + (nlo < flo ? 1u : 0u);
      flo = nlo;
    }
    const uint64_t rlo = flo + (1ull << 61);
    const uint32_t rhi = fhi + (rlo < flo ? 1u : 0u);
    const uint32_t qr = (rhi << 2) | (uint32_t)(rlo >> 62);
    const uint32_t* Pk = T.pp + (int64_t)k * T.LPP;
    const int64_t plane = (int64_t)(J->cap_deg + 1) * L;
    const uint32_t* S = J->wsS + (int64_t)i * L;
    uint32_t cin1 = 0, cin2 = 0, cq = 0, bsub = 0;
    uint32_t bprev = 0, cprev1 = 0, cprev2 = 0, qhprev = 0;
    for (int b0 = 0; b0 < cap; b0 += 32) {
      const int l = b0 + lane;
      const uint32_t a = l < L ? S[l] : 0u, bw = l < L ? S[plane + l] : 0u,
                     cw = l < L ? S[2 * plane + l] : 0u;
      // sum of the column words a_l + b_l 2^32 + c_l 2^64 at limb l
      uint32_t bin = __shfl_up_sync(0xffffffffu, bw, 1);
      uint32_t cin_w = __shfl_up_sync(0xffffffffu, cw, 2);
      const uint32_t c31 = __shfl_sync(0xffffffffu, cw, 31), c30 = __shfl_sync(0xffffffffu, cw, 30);
      const uint32_t b31 = __shfl_sync(0xffffffffu, bw, 31);
      if (lane == 0) {
        bin = bprev;
        cin_w = cprev2;
      }
      if (lane == 1) cin_w = cprev1;
      uint32_t rr = ballot_add(a, bin, cin1, lane);
      rr = ballot_add(rr, cin_w, cin2, lane);
      bprev = b31;
      cprev2 = c30;
      cprev1 = c31;
      // q P: limb l = lo(q P_l) + hi(q P_{l-1}) + carry
      const uint64_t qp = (uint64_t)qr * ((l < L && l < T.LPP) ? Pk[l] : 0u);
      uint32_t qh = __shfl_up_sync(0xffffffffu, (uint32_t)(qp >> 32), 1);
      const uint32_t qh31 = __shfl_sync(0xffffffffu, (uint32_t)(qp >> 32), 31);
      if (lane == 0) qh = qhprev;
      qhprev = qh31;
      const uint32_t qpl = ballot_add((uint32_t)qp, qh, cq, lane);
      const uint32_t res = ballot_sub(rr, qpl, bsub, lane);
      if (l < cap) out[l] = res;
    }
  }
  pdl_trigger();
}

void launch_bigcrt(int g_tab, int g_gemm, int g_carry, cudaStream_t s, const Job* jobs, WorkList tab,
                   WorkList gemm, WorkList carry, Tables T) {
  if (g_tab) k_bigcrt_tables<<<g_tab, kBigTabThreads, 0, s>>>(jobs, tab, T);
  if (g_gemm) k_bigcrt_gemm<<<g_gemm, 256, 0, s>>>(jobs, gemm, T);
  if (g_carry) k_bigcrt_carry<<<g_carry, kBigCarryWarps * 32, 0, s>>>(jobs, carry, T);
}

}  // namespace bs
