// Device stages of the modular resultant (Sec. 5.1, steps (a)-(e)):
//
//   k_plan_single   plan of one device-resident job (degrees, bound, primes)
//   k_eval          (a)+(b): reduce a coefficient row mod p, scale by g^i and evaluate it
//                   on the coset g * <omega> with a forward transform in shared memory
//   k_unires<L>     (c): one univariate resultant mod p per thread, formal degrees,
//                   detection of points where a leading coefficient vanishes
//   k_intt          prime selection + (d): inverse transform, unscaling, degree check
//   k_crt           (e): Garner mixed-radix digits, sign decision and conversion to
//                   two's complement limbs, one warp per coefficient
//
// All stage kernels are persistent: the grid is a multiple of the SM count and blocks
// stride over a flat work index whose extent is read from device memory, so the same
// launches serve host- and device-planned jobs and whole batches.
#include <cuda_runtime.h>
#include <stdint.h>

#include "common.cuh"
#include "resultant_kernels.cuh"
#include "unires.cuh"

namespace bs {

// ------------------------------------------------------------------------------------
// plan of a single device-resident job (one block)
// ------------------------------------------------------------------------------------
struct PolySummary {
  UF S;
  int m, td, dego, lcb;
};

__device__ void summarise_block(const Grid& h, int var, PolySummary* out, UF* sh_uf,
                                int* sh_int) {
  // per-thread partials over rows e = tid, tid + blockDim, ...
  UF S{0u, 0};
  int m = -1, td = -1, dego = -1;
  int ee = ext_e(h, var);
  for (int e = threadIdx.x; e <= ee; e += blockDim.x) {
    RowStat rs = row_stat(h, var, e);
    if (rs.max_o < 0) continue;
    S = uf_add(S, uf_mul(rs.l1, rs.l1));
    m = max(m, e);
    td = max(td, e + rs.max_o);
    dego = max(dego, rs.max_o);
  }
  // block reduction (upper floats added in any order stay upper bounds)
  sh_uf[threadIdx.x] = S;
  sh_int[3 * threadIdx.x + 0] = m;
  sh_int[3 * threadIdx.x + 1] = td;
  sh_int[3 * threadIdx.x + 2] = dego;
  __syncthreads();
  for (int s = blockDim.x / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s) {
      sh_uf[threadIdx.x] = uf_add(sh_uf[threadIdx.x], sh_uf[threadIdx.x + s]);
      for (int k = 0; k < 3; ++k)
        sh_int[3 * threadIdx.x + k] = max(sh_int[3 * threadIdx.x + k], sh_int[3 * (threadIdx.x + s) + k]);
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    out->S = sh_uf[0];
    out->m = sh_int[0];
    out->td = sh_int[1];
    out->dego = sh_int[2];
    out->lcb = 0;
    if (out->m >= 0) out->lcb = row_stat(h, var, out->m).min_bits;
  }
  __syncthreads();
}

__global__ void k_plan_single(Job* job, int64_t* offs, Tables T) {
  __shared__ UF sh_uf[256];
  __shared__ int sh_int[3 * 256];
  __shared__ PolySummary sf, sg;
  Job& J = *job;
  summarise_block(J.f, J.var, &sf, sh_uf, sh_int);
  summarise_block(J.g, J.var, &sg, sh_uf, sh_int);
  if (threadIdx.x == 0) {
    Plan P = finish_plan(sf.S, sf.m, sf.td, sf.dego, sf.lcb, sg.S, sg.m, sg.td, sg.dego, sg.lcb,
                         T.lg_prefix, T.T);
    // capacity checks against what the host sized from the grid extents
    if (P.status == 0 && P.trivial == 0) {
      if (P.k_total > T.Tt || P.k_need > T.Tg || P.N > T.NT) P.status = kErrInternal;
      if (P.D > J.cap_deg || P.out_limbs > J.cap_limbs) P.status = kErrInternal;
      if (P.k_total > J.cap_k_total || P.k_need > J.cap_k_need || P.logN > J.cap_logN ||
          P.D > J.cap_D || (P.me + 1) + (P.ne + 1) > J.cap_rows)
        P.status = kErrInternal;
    }
    if (P.status) set_status(J.status, P.status);
    J.plan = P;
    J.rows = (P.trivial || P.status) ? 0 : (P.me + 1) + (P.ne + 1);
    bool run = (P.status == 0 && P.trivial == 0);
    // offsets for the four stages (one job each): eval, unires tiles, intt, crt
    offs[0] = 0;
    offs[1] = run ? (int64_t)P.k_total * J.rows : 0;
    offs[2] = 0;
    offs[3] = run ? (((int64_t)P.k_total << P.logN) + kUniTile - 1) / kUniTile : 0;
    offs[4] = 0;
    offs[5] = run ? P.k_total : 0;
    offs[6] = 0;
    offs[7] = (int64_t)J.cap_deg + 1;
  }
}

// ------------------------------------------------------------------------------------
// (a) + (b): reduction, coset scaling, forward transform (decimation in frequency)
// ------------------------------------------------------------------------------------
__device__ __forceinline__ uint32_t residue_m(const uint32_t* c, int L, const uint32_t* pw,
                                              const uint32_t* mpw, uint32_t p, uint32_t pinv) {
  uint32_t acc = 0;
  for (int l = 0; l < L; ++l) acc = madd(acc, redc((uint64_t)c[l] * pw[l], p, pinv), p);
  if (c[L - 1] >> 31) acc = msub(acc, mpw[L], p);
  return acc;
}

// in-place forward transform of sm[0..N): output position u holds the value at
// g * omega^{bitreverse(u)}
__device__ __forceinline__ void dif_ntt(uint32_t* sm, int logN, const uint32_t* tw, int logNT,
                                        const Mod M) {
  const int N = 1 << logN;
  for (int lg = logN - 1; lg >= 0; --lg) {
    const int len = 1 << lg;
    const int stride_sh = logNT - (lg + 1);
    for (int bf = threadIdx.x; bf < (N >> 1); bf += blockDim.x) {
      const int j = bf & (len - 1);
      const int i0 = ((bf >> lg) << (lg + 1)) + j;
      const int i1 = i0 + len;
      const uint32_t u = sm[i0], v = sm[i1];
      sm[i0] = madd(u, v, M.p);
      sm[i1] = mmul(msub(u, v, M.p), tw[j << stride_sh], M);
    }
    __syncthreads();
  }
}

// in-place inverse transform (decimation in time) of bit-reversed input; output natural
// order, scaled by N
__device__ __forceinline__ void dit_intt(uint32_t* sm, int logN, const uint32_t* itw, int logNT,
                                         const Mod M) {
  const int N = 1 << logN;
  for (int lg = 0; lg < logN; ++lg) {
    const int len = 1 << lg;
    const int stride_sh = logNT - (lg + 1);
    for (int bf = threadIdx.x; bf < (N >> 1); bf += blockDim.x) {
      const int j = bf & (len - 1);
      const int i0 = ((bf >> lg) << (lg + 1)) + j;
      const int i1 = i0 + len;
      const uint32_t u = sm[i0];
      const uint32_t v = mmul(sm[i1], itw[j << stride_sh], M);
      sm[i0] = madd(u, v, M.p);
      sm[i1] = msub(u, v, M.p);
    }
    __syncthreads();
  }
}

__global__ void __launch_bounds__(kEvalThreads) k_eval(const Job* jobs, WorkList wl, Tables T) {
  extern __shared__ uint32_t sm[];
  const int64_t total = wl.off[wl.n];
  for (int64_t item = blockIdx.x; item < total; item += gridDim.x) {
    const int ji = find_item(wl.off, wl.n, item);
    const Job* J = jobs + (wl.ids ? wl.ids[ji] : ji);
    const int64_t local = item - wl.off[ji];
    const int rows = J->rows;
    const int q = (int)(local / rows);
    const int row = (int)(local - (int64_t)q * rows);
    const int me = J->plan.me;
    const int logN = J->plan.logN;
    const int N = 1 << logN;
    const bool isf = row <= me;
    const int e = isf ? row : row - me - 1;
    const Grid G = isf ? J->f : J->g;
    const int var = J->var;
    const PrimeConst pc = T.pc[q];
    const Mod M{pc.p, pc.pinv};
    const uint32_t* pw = T.pw + (int64_t)q * (kMaxLimbs + 1);
    const uint32_t* mpw = T.mpw + (int64_t)q * (kMaxLimbs + 1);
    const uint32_t* cp = T.cp + (int64_t)q * T.NT;
    const int eo = ext_o(G, var);
    for (int t = threadIdx.x; t < N; t += blockDim.x) {
      uint32_t acc = 0;
      for (int o = t; o <= eo; o += N) {
        const uint32_t r = residue_m(coef_ptr(G, var, e, o), G.L, pw, mpw, M.p, M.pinv);
        const uint32_t s = (o < T.NT) ? cp[o] : mpow(pc.g_m, (uint32_t)o, pc.one_m, M);
        acc = madd(acc, mmul(r, s, M), M.p);
      }
      sm[t] = acc;
    }
    __syncthreads();
    dif_ntt(sm, logN, T.tw + (int64_t)q * (T.NT >> 1), T.logNT, M);
    uint32_t* dst = J->ev + ((int64_t)q * rows + row) * N;
    for (int t = threadIdx.x; t < N; t += blockDim.x) dst[t] = sm[t];
    __syncthreads();
  }
}

// ------------------------------------------------------------------------------------
// (c): univariate resultants, one per thread
// ------------------------------------------------------------------------------------
template <int L>
__global__ void __launch_bounds__(kUniTile) k_unires(const Job* jobs, WorkList wl, Tables T) {
  const int64_t total = wl.off[wl.n];
  for (int64_t tile = blockIdx.x; tile < total; tile += gridDim.x) {
    const int ji = find_item(wl.off, wl.n, tile);
    const Job* J = jobs + (wl.ids ? wl.ids[ji] : ji);
    const int logN = J->plan.logN;
    const int64_t ninst = (int64_t)J->plan.k_total << logN;
    const int64_t inst = (tile - wl.off[ji]) * kUniTile + threadIdx.x;
    if (inst >= ninst) continue;
    const int N = 1 << logN;
    const int q = (int)(inst >> logN);
    const int t = (int)(inst & (N - 1));
    const int me = J->plan.me, ne = J->plan.ne;
    const int rows = J->rows;
    const PrimeConst pc = T.pc[q];
    const Mod M{pc.p, pc.pinv};
    const uint32_t* bf = J->ev + (int64_t)q * rows * N + t;
    const uint32_t* bg = bf + (int64_t)(me + 1) * N;
    uint32_t A[Arr<L>::N], B[Arr<L>::N];
#pragma unroll
    for (int s = 0; s < Arr<L>::N; ++s) {
      A[s] = (s <= me) ? __ldg(bf + (int64_t)(me - s) * N) : 0u;
      B[s] = (s <= ne) ? __ldg(bg + (int64_t)(ne - s) * N) : 0u;
    }
    if (A[0] == 0 || B[0] == 0) J->pstat[q] = 1;  // unlucky: a leading coefficient vanishes
    uint32_t den;
    uint32_t num = unires_numden<L>(A, me + 1, B, ne + 1, M, pc.one_m, &den);
    J->vals[inst] = mmul(num, minv(den, pc.one_m, M), M);
  }
}

// ------------------------------------------------------------------------------------
// prime selection + (d): inverse transform, unscaling, degree check
// ------------------------------------------------------------------------------------
__global__ void __launch_bounds__(kEvalThreads) k_intt(const Job* jobs, WorkList wl, Tables T) {
  extern __shared__ uint32_t sm[];
  const int64_t total = wl.off[wl.n];
  for (int64_t item = blockIdx.x; item < total; item += gridDim.x) {
    const int ji = find_item(wl.off, wl.n, item);
    const Job* J = jobs + (wl.ids ? wl.ids[ji] : ji);
    const int q = (int)(item - wl.off[ji]);
    const int k_need = J->plan.k_need, k_total = J->plan.k_total;
    // rank of prime q among the good primes; the block of prime 0 also checks that
    // enough good primes exist
    __shared__ int s_rank, s_good;
    if (threadIdx.x == 0) {
      s_rank = 0;
      s_good = 0;
    }
    __syncthreads();
    int cnt = 0;
    for (int j = threadIdx.x; j < q; j += blockDim.x) cnt += (J->pstat[j] == 0);
    if (cnt) atomicAdd(&s_rank, cnt);
    if (q == 0) {
      int g = 0;
      for (int j = threadIdx.x; j < k_total; j += blockDim.x) g += (J->pstat[j] == 0);
      if (g) atomicAdd(&s_good, g);
    }
    __syncthreads();
    const int r = s_rank;
    if (q == 0 && threadIdx.x == 0) {
      if (s_good < k_need) set_status(J->status, kErrUnlucky);
      if (J->rejected) atomicAdd(J->rejected, k_total - s_good);
    }
    const bool good = J->pstat[q] == 0;
    __syncthreads();
    if (!good || r >= k_need) continue;
    const int logN = J->plan.logN;
    const int N = 1 << logN;
    const int D = J->plan.D;
    const PrimeConst pc = T.pc[q];
    const Mod M{pc.p, pc.pinv};
    const uint32_t* src = J->vals + ((int64_t)q << logN);
    for (int t = threadIdx.x; t < N; t += blockDim.x) sm[t] = src[t];
    __syncthreads();
    dit_intt(sm, logN, T.itw + (int64_t)q * (T.NT >> 1), T.logNT, M);
    const uint32_t* icp = T.icp + (int64_t)q * T.NT;
    const uint32_t ni = T.ninv[q * (kLogNMax + 1) + logN];
    uint32_t* dst = J->rmod + (int64_t)r * (D + 1);
    bool bad = false;
    for (int i = threadIdx.x; i < N; i += blockDim.x) {
      const uint32_t v = mmul(mmul(sm[i], icp[i], M), ni, M);
      if (i <= D)
        dst[i] = v;
      else if (v != 0)
        bad = true;
    }
    if (bad) set_status(J->status, kErrInternal);
    if (threadIdx.x == 0) J->sel[r] = q;
    __syncthreads();
  }
}

// ------------------------------------------------------------------------------------
// (e): mixed-radix reconstruction, one warp per coefficient
// ------------------------------------------------------------------------------------
__global__ void __launch_bounds__(kCrtWarps * 32) k_crt(const Job* jobs, WorkList wl, Tables T,
                                                        int kmax, int lmax) {
  extern __shared__ uint32_t smc[];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int nwarps = blockDim.x >> 5;
  uint32_t* x = smc + (size_t)warp * (4 * kmax + lmax);
  uint32_t* pq = x + kmax;
  uint32_t* pinvq = pq + kmax;
  uint32_t* selq = pinvq + kmax;
  uint32_t* limb = selq + kmax;
  const int64_t total = wl.off[wl.n];
  for (int64_t item = (int64_t)blockIdx.x * nwarps + warp; item < total;
       item += (int64_t)gridDim.x * nwarps) {
    const int ji = find_item(wl.off, wl.n, item);
    const Job* J = jobs + (wl.ids ? wl.ids[ji] : ji);
    const int i = (int)(item - wl.off[ji]);
    const int cap = J->cap_limbs;
    uint32_t* out = J->out + (int64_t)i * cap;
    const Plan& P = J->plan;
    if (P.status != 0 || P.trivial != 0 || i > P.D) {
      const uint32_t v0 = (P.status == 0 && P.trivial == 2 && i == 0) ? 1u : 0u;
      for (int l = lane; l < cap; l += 32) out[l] = (l == 0) ? v0 : 0u;
      continue;
    }
    const int k = P.k_need;
    const int D = P.D;
    const int Tg = T.Tg;
    // residues and constants of the selected primes
    for (int j = lane; j < k; j += 32) {
      const int s = J->sel[j];
      const PrimeConst pc = T.pc[s];
      x[j] = J->rmod[(int64_t)j * (D + 1) + i];
      pq[j] = pc.p;
      pinvq[j] = pc.pinv;
      selq[j] = (uint32_t)s;
    }
    __syncwarp();
    // Garner: x_q <- (x_q - d_j) * p_j^-1 mod p_q for q > j; x_j is then digit d_j
    for (int j = 0; j < k - 1; ++j) {
      const uint32_t d = x[j];
      const uint32_t* grow = T.ginv + (int64_t)selq[j] * Tg;
      for (int q = j + 1 + lane; q < k; q += 32) {
        const uint32_t p = pq[q];
        const uint32_t dd = d >= p ? d - p : d;
        const Mod M{p, pinvq[q]};
        x[q] = mmul(msub(x[q], dd, p), grow[selq[q]], M);
      }
      __syncwarp();
    }
    // sign: the value exceeds (P-1)/2 iff its digits exceed ((p_j - 1)/2)_j from the top
    int hi = -1;
    for (int j = lane; j < k; j += 32)
      if (x[j] != (pq[j] - 1) / 2) hi = j;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) hi = max(hi, __shfl_xor_sync(0xffffffffu, hi, o));
    const bool neg = hi >= 0 && x[hi] > (pq[hi] - 1) / 2;
    __syncwarp();
    // negative values: u = P - 1 - c has digits p_j - 1 - d_j, and c - P = ~u
    if (neg)
      for (int j = lane; j < k; j += 32) x[j] = pq[j] - 1 - x[j];
    for (int l = lane; l < cap; l += 32) limb[l] = 0;
    __syncwarp();
    // Horner from the top digit, c = c * p_j + d_j, limbs spread over the lanes; the
    // carries of a 32-limb chunk are resolved with two ballots (generate / propagate)
    int alen = 0;
    bool ovf = false;
    for (int j = k - 1; j >= 0; --j) {
      const uint32_t pj = pq[j];
      alen = alen + 1 < cap ? alen + 1 : cap;
      uint32_t cin = 0, hprev = x[j];
      for (int b = 0; b < alen; b += 32) {
        const int l = b + lane;
        const uint32_t v = l < alen ? limb[l] : 0u;
        const uint64_t prod = (uint64_t)v * pj;
        const uint32_t lo = (uint32_t)prod, hi32 = (uint32_t)(prod >> 32);
        uint32_t hin = __shfl_up_sync(0xffffffffu, hi32, 1);
        if (lane == 0) hin = hprev;
        const uint32_t s = lo + hin;
        const uint32_t G = __ballot_sync(0xffffffffu, s < lo);
        const uint32_t Pm = __ballot_sync(0xffffffffu, s == 0xffffffffu) & ~G;
        const uint32_t X = G | Pm;
        const uint64_t S = (uint64_t)X + G + cin;
        const uint32_t C = (uint32_t)S ^ X ^ G;
        const uint32_t res = s + ((C >> lane) & 1u);
        __syncwarp();
        if (l < alen)
          limb[l] = res;
        else if (l == alen && res != 0)
          ovf = true;
        cin = (uint32_t)(S >> 32);
        hprev = __shfl_sync(0xffffffffu, hi32, 31);
      }
      if ((alen & 31) == 0 && (cin != 0 || hprev != 0)) ovf = true;
      __syncwarp();
    }
    if (__any_sync(0xffffffffu, ovf) && lane == 0) set_status(J->status, kErrInternal);
    for (int l = lane; l < cap; l += 32) out[l] = neg ? ~limb[l] : limb[l];
    __syncwarp();
  }
}

// ------------------------------------------------------------------------------------
// univariate resultants of given images (bs_uni_resultant_modp)
// ------------------------------------------------------------------------------------
template <int L>
__global__ void __launch_bounds__(kUniTile) k_unires_direct(int n, const int32_t* pidx,
                                                            const uint32_t* a, int da, int lda,
                                                            const uint32_t* b, int db, int ldb,
                                                            uint32_t* res, Tables T) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const PrimeConst pc = T.pc[pidx[i]];
  const Mod M{pc.p, pc.pinv};
  uint32_t A[Arr<L>::N], B[Arr<L>::N];
#pragma unroll
  for (int s = 0; s < Arr<L>::N; ++s) {
    A[s] = (s <= da) ? redc((uint64_t)a[(int64_t)i * lda + da - s] * pc.r2, M.p, M.pinv) : 0u;
    B[s] = (s <= db) ? redc((uint64_t)b[(int64_t)i * ldb + db - s] * pc.r2, M.p, M.pinv) : 0u;
  }
  uint32_t den;
  const uint32_t num = unires_numden<L>(A, da + 1, B, db + 1, M, pc.one_m, &den);
  res[i] = redc((uint64_t)mmul(num, minv(den, pc.one_m, M), M), M.p, M.pinv);
}

template __global__ void k_unires_direct<8>(int, const int32_t*, const uint32_t*, int, int,
                                            const uint32_t*, int, int, uint32_t*, Tables);
template __global__ void k_unires_direct<16>(int, const int32_t*, const uint32_t*, int, int,
                                             const uint32_t*, int, int, uint32_t*, Tables);
template __global__ void k_unires_direct<24>(int, const int32_t*, const uint32_t*, int, int,
                                             const uint32_t*, int, int, uint32_t*, Tables);
template __global__ void k_unires_direct<33>(int, const int32_t*, const uint32_t*, int, int,
                                             const uint32_t*, int, int, uint32_t*, Tables);
template __global__ void k_unires_direct<48>(int, const int32_t*, const uint32_t*, int, int,
                                             const uint32_t*, int, int, uint32_t*, Tables);
template __global__ void k_unires_direct<65>(int, const int32_t*, const uint32_t*, int, int,
                                             const uint32_t*, int, int, uint32_t*, Tables);

template __global__ void k_unires<8>(const Job*, WorkList, Tables);
template __global__ void k_unires<16>(const Job*, WorkList, Tables);
template __global__ void k_unires<24>(const Job*, WorkList, Tables);
template __global__ void k_unires<33>(const Job*, WorkList, Tables);
template __global__ void k_unires<48>(const Job*, WorkList, Tables);
template __global__ void k_unires<65>(const Job*, WorkList, Tables);

// ------------------------------------------------------------------------------------
// launchers (kernels are launched from the translation unit that defines them)
// ------------------------------------------------------------------------------------
template <int L>
static int occ1() {
  int b = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_unires<L>, kUniTile, 0);
  return b > 0 ? b : 1;
}

int uni_occupancy(int cls) {
  switch (cls) {
    case 0: return occ1<8>();
    case 1: return occ1<16>();
    case 2: return occ1<24>();
    case 3: return occ1<33>();
    case 4: return occ1<48>();
    default: return occ1<65>();
  }
}

void launch_uni(int cls, int grid, cudaStream_t s, const Job* jobs, WorkList wl, Tables T) {
  switch (cls) {
    case 0: k_unires<8><<<grid, kUniTile, 0, s>>>(jobs, wl, T); break;
    case 1: k_unires<16><<<grid, kUniTile, 0, s>>>(jobs, wl, T); break;
    case 2: k_unires<24><<<grid, kUniTile, 0, s>>>(jobs, wl, T); break;
    case 3: k_unires<33><<<grid, kUniTile, 0, s>>>(jobs, wl, T); break;
    case 4: k_unires<48><<<grid, kUniTile, 0, s>>>(jobs, wl, T); break;
    default: k_unires<65><<<grid, kUniTile, 0, s>>>(jobs, wl, T); break;
  }
}

void launch_uni_direct(int cls, int n, cudaStream_t s, const int32_t* idx, const uint32_t* a, int da,
                       int lda, const uint32_t* b, int db, int ldb, uint32_t* res, Tables T) {
  const int grid = (n + kUniTile - 1) / kUniTile;
  switch (cls) {
    case 0: k_unires_direct<8><<<grid, kUniTile, 0, s>>>(n, idx, a, da, lda, b, db, ldb, res, T); break;
    case 1: k_unires_direct<16><<<grid, kUniTile, 0, s>>>(n, idx, a, da, lda, b, db, ldb, res, T); break;
    case 2: k_unires_direct<24><<<grid, kUniTile, 0, s>>>(n, idx, a, da, lda, b, db, ldb, res, T); break;
    case 3: k_unires_direct<33><<<grid, kUniTile, 0, s>>>(n, idx, a, da, lda, b, db, ldb, res, T); break;
    case 4: k_unires_direct<48><<<grid, kUniTile, 0, s>>>(n, idx, a, da, lda, b, db, ldb, res, T); break;
    default: k_unires_direct<65><<<grid, kUniTile, 0, s>>>(n, idx, a, da, lda, b, db, ldb, res, T); break;
  }
}

void launch_eval(int grid, size_t smem, cudaStream_t s, const Job* jobs, WorkList wl, Tables T) {
  k_eval<<<grid, kEvalThreads, smem, s>>>(jobs, wl, T);
}
void launch_intt(int grid, size_t smem, cudaStream_t s, const Job* jobs, WorkList wl, Tables T) {
  k_intt<<<grid, kEvalThreads, smem, s>>>(jobs, wl, T);
}
void launch_crt(int grid, int threads, size_t smem, cudaStream_t s, const Job* jobs, WorkList wl,
                Tables T, int kmax, int lmax) {
  k_crt<<<grid, threads, smem, s>>>(jobs, wl, T, kmax, lmax);
}
void launch_plan_single(cudaStream_t s, Job* job, int64_t* offs, Tables T) {
  k_plan_single<<<1, 256, 0, s>>>(job, offs, T);
}
int set_dyn_smem_limit(const void* func, int optin) {
  cudaFuncAttributes a;
  if (cudaFuncGetAttributes(&a, func) != cudaSuccess) return kErrCuda;
  const int lim = optin - (int)a.sharedSizeBytes;
  if (cudaFuncSetAttribute(func, cudaFuncAttributeMaxDynamicSharedMemorySize, lim) != cudaSuccess)
    return kErrCuda;
  return 0;
}

int set_stage_smem_limits(int optin) {
  int rc = 0;
  rc |= set_dyn_smem_limit((const void*)k_eval, optin);
  rc |= set_dyn_smem_limit((const void*)k_intt, optin);
  rc |= set_dyn_smem_limit((const void*)k_crt, optin);
  return rc;
}

}  // namespace bs
