// Device stages of the modular resultant (Sec. 5.1, steps (a)-(e)):
//
//   k_plan_single   plan of one device-resident job (degrees, bound, primes, spares)
//   k_eval_w<R>     (a)+(b): reduce a coefficient row mod p, scale by g^i and evaluate it
//                   on the coset g * <omega>: one warp per row, N = 32 R points in
//                   registers (R = 0: the size class is read per job)
//   k_eval          the same for N > 1024: one block of N / 1024 warps per row
//   k_unires<L>     (c): one univariate resultant mod p per thread, formal degrees,
//                   detection of points where a leading coefficient vanishes
//   k_intt          prime selection + (d): inverse transform, unscaling, degree check,
//                   one block per prime; k_intt_w: one warp per prime (N <= 512)
//   k_crt_w<TILE>   (e): weighted-sum or Garner reconstruction, one warp per coefficient
//   k_crt           (e): block Garner for many primes (see also bigcrt.cu)
//
// All stage kernels are persistent: the grid is a multiple of the SM count and blocks
// stride over a flat work index whose extent is read from device memory, so the same
// launches serve host- and device-planned jobs and whole batches.
#include <cuda_runtime.h>
#include <stdint.h>

#include "common.cuh"
#include "resultant_kernels.cuh"
#include "unires.cuh"
#include "ballot.cuh"
#include "warp_ntt.cuh"

namespace bs {

// ------------------------------------------------------------------------------------
// L2 prefetch of the table ranges a job will read (the step may start with a cold L2):
// one bulk prefetch per contiguous range, trimmed inward to 16-byte boundaries so that
// every prefetched byte lies inside its allocation
// ------------------------------------------------------------------------------------
__device__ __forceinline__ void l2_prefetch_range(const void* p, size_t bytes) {
  uintptr_t a = ((uintptr_t)p + 15) & ~(uintptr_t)15;
  const uintptr_t e = ((uintptr_t)p + bytes) & ~(uintptr_t)15;
  while (a < e) {
    const uint32_t n = (uint32_t)((e - a) < (uintptr_t)65536 ? (e - a) : (uintptr_t)65536);
    asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(a), "r"(n) : "memory");
    a += n;
  }
}

// Per-prime tables are stored row after row, so the rows of the first kt primes form one
// contiguous block per table.  A bulk prefetch holds its thread and uses its SM's path
// to L2, so the 64 KiB chunks are dealt out one per block over the first blocks of a
// grid: `rank` is the caller's index among `ranks` issuers.  These are the tables the
// stages after evaluation read (inverse transform, reconstruction).
struct PfRange {
  const void* p;
  size_t bytes;
};

__device__ void prefetch_late_tables(const Tables& T, int kt, int N, int kn, int rank, int ranks,
                                     int32_t* st) {
  kt = min(kt, T.Tt);
  kn = min(kn, T.Tg);
  const int K = min(kn, T.WK);
  int64_t mwords = 0;  // the M_k block of k = K
  if (K >= 1) mwords = (int64_t)K * ws_len(K);
  if (!dbg_ok(K < 1 || T.ws_moff[K] + mwords <= T.ws_m_words, st, kDbgEvalPf)) return;
  const PfRange R[6] = {
      {T.itwp, sizeof(uint32_t) * (size_t)kt * T.NT},
      {T.icp, sizeof(uint32_t) * (size_t)kt * T.NT},
      {T.ginv, sizeof(uint32_t) * (size_t)kt * T.Tg},
      {T.pp, sizeof(uint32_t) * (size_t)(kn + 1) * T.LPP},
      {T.ws_y, sizeof(uint32_t) * (size_t)K * (K + 1) / 2},
      {T.ws_m, sizeof(uint32_t) * (size_t)min(mwords, T.ws_m_words)},
  };
  (void)N;
  constexpr size_t kChunk = 65536;
  int base = 0;
  for (int r = 0; r < 6; ++r) {
    const size_t bytes = R[r].bytes;
    const char* p0 = (const char*)R[r].p;
    if (r == 5 && K >= 1) {  // the block of k = K starts at ws_moff[K]: read it once
      p0 = (const char*)(T.ws_m + T.ws_moff[K]);
    }
    const int nchunks = (int)((bytes + kChunk - 1) / kChunk);
    for (int c = rank - base; c < nchunks; c += ranks) {
      if (c < 0) continue;
      const size_t off = (size_t)c * kChunk;
      const size_t len = bytes - off < kChunk ? bytes - off : kChunk;
      l2_prefetch_range(p0 + off, len);
    }
    base = (base + nchunks) % ranks;
  }
}

// c mod p in Montgomery form for a two's complement coefficient of L limbs
__device__ __forceinline__ uint32_t residue_m(const uint32_t* c, int L, const uint32_t* pw,
                                              const uint32_t* mpw, uint32_t p, uint32_t pinv) {
  uint32_t acc = 0;
  for (int l = 0; l < L; ++l) acc = madd(acc, redc((uint64_t)c[l] * pw[l], p, pinv), p);
  if (c[L - 1] >> 31) acc = msub(acc, mpw[L], p);
  return acc;
}

// ------------------------------------------------------------------------------------
// plan of a single device-resident job (one block of kPlanThreads)
// ------------------------------------------------------------------------------------
constexpr int kSlotInts = 6;  // per row slot: m, td, dego, lcb, lcnt, lco

struct PolySummary {
  UF S;
  int m, td, dego, lcb;
  int lcnt, lco;  // leading row: nonzero coefficients, index of the smallest one
  int64_t l2S;    // log2 S (Q16, rounded up), 0 for S = 0
};

__device__ __forceinline__ UF shfl_uf(UF a, int src_lane_xor) {
  UF b;
  b.m = __shfl_xor_sync(0xffffffffu, a.m, src_lane_xor);
  b.e = __shfl_xor_sync(0xffffffffu, a.e, src_lane_xor);
  return b;
}

// One half of the plan block (kPlanThreads / 2 threads) summarises one polynomial:
// thread t takes row e = t / 8 (+ 32 per round) and the coefficients o = t % 8, +8, ...
// of that row, so the loads of all rows are in flight together; the eight threads of a
// row combine their partial sums with shuffles, and the rows are combined through
// shared memory.
__device__ void summarise_half(const Grid& h, int var, int tid, PolySummary* out, UF* sh_uf,
                               int* sh_int) {
  constexpr int kHalf = kPlanThreads / 2;
  const int sub = tid & 7;
  const int ee = ext_e(h, var), eo = ext_o(h, var);
  // issue every line this thread reads before the first use, so the loads of the loop
  // below overlap instead of waiting one after another
  for (int e0 = 0; e0 <= ee; e0 += kHalf / 8) {
    const int e = e0 + tid / 8;
    if (e > ee) break;
    for (int o = sub; o <= eo; o += 8) {
      const uint32_t* c = coef_ptr(h, var, e, o);
      asm volatile("prefetch.L1 [%0];" ::"l"(c));
      if (h.L > 1) asm volatile("prefetch.L1 [%0];" ::"l"(c + h.L - 1));
    }
  }
  UF S{0u, 0};
  int m = -1, td = -1, dego = -1, lcb = 0, lcnt = 0, lco = 0;
  for (int e0 = 0; e0 <= ee; e0 += kHalf / 8) {
    const int e = e0 + tid / 8;
    UF l1{0u, 0};
    int mo = -1, mb = 0, cnt = 0, mbo = 0;
    if (h.L <= 2) {
      // narrow coefficients: exact 128-bit sums of the magnitudes, one rounding per row
      uint64_t slo = 0, shi = 0;
      if (e <= ee) {
        for (int o = sub; o <= eo; o += 8) {
          const uint64_t mag = mag_narrow(coef_ptr(h, var, e, o), h.L);
          if (mag) {
            slo += mag;
            shi += (slo < mag) ? 1u : 0u;
            mo = o;
            ++cnt;
            const int bits = 64 - clz64(mag);
            if (mb == 0 || bits < mb) {
              mb = bits;
              mbo = o;
            }
          }
        }
      }
#pragma unroll
      for (int x = 4; x > 0; x >>= 1) {
        const uint64_t olo = __shfl_xor_sync(0xffffffffu, slo, x);
        const uint64_t ohi = __shfl_xor_sync(0xffffffffu, shi, x);
        const uint64_t nlo = slo + olo;
        shi = shi + ohi + ((nlo < slo) ? 1u : 0u);
        slo = nlo;
      }
      l1 = uf_from_u128(shi, slo);
    } else if (e <= ee) {
      for (int o = sub; o <= eo; o += 8) {
        bool nz;
        int bits;
        const UF u = mag_uf(coef_ptr(h, var, e, o), h.L, &nz, &bits);
        if (nz) {
          l1 = uf_add(l1, u);
          mo = o;
          ++cnt;
          if (mb == 0 || bits < mb) {
            mb = bits;
            mbo = o;
          }
        }
      }
    }
#pragma unroll
    for (int x = 4; x > 0; x >>= 1) {
      if (h.L > 2) l1 = uf_add(l1, shfl_uf(l1, x));
      mo = max(mo, __shfl_xor_sync(0xffffffffu, mo, x));
      cnt += __shfl_xor_sync(0xffffffffu, cnt, x);
      const int ob = __shfl_xor_sync(0xffffffffu, mb, x);
      const int obo = __shfl_xor_sync(0xffffffffu, mbo, x);
      if (ob != 0 && (mb == 0 || ob < mb || (ob == mb && obo < mbo))) {
        mb = ob;
        mbo = obo;
      }
    }
    if (sub == 0 && mo >= 0) {
      S = uf_add(S, uf_mul(l1, l1));
      if (e > m) {
        m = e;
        lcb = mb;
        lcnt = cnt;
        lco = mbo;
      }
      td = max(td, e + mo);
      dego = max(dego, mo);
    }
  }
  // combine the row leaders (sub == 0) through shared memory, then one warp reduces
  // the slots with shuffles
  const int slot = tid / 8;
  if (sub == 0) {
    sh_uf[slot] = S;
    sh_int[kSlotInts * slot + 0] = m;
    sh_int[kSlotInts * slot + 1] = td;
    sh_int[kSlotInts * slot + 2] = dego;
    sh_int[kSlotInts * slot + 3] = lcb;
    sh_int[kSlotInts * slot + 4] = lcnt;
    sh_int[kSlotInts * slot + 5] = lco;
  }
  __syncthreads();
  if (tid < 32) {
    UF s{0u, 0};
    int M = -1, TD = -1, DO = -1, LCB = 0, LCN = 0, LCO = 0;
    for (int w = tid; w < kHalf / 8; w += 32) {
      s = uf_add(s, sh_uf[w]);
      if (sh_int[kSlotInts * w] > M) {
        M = sh_int[kSlotInts * w];
        LCB = sh_int[kSlotInts * w + 3];
        LCN = sh_int[kSlotInts * w + 4];
        LCO = sh_int[kSlotInts * w + 5];
      }
      TD = max(TD, sh_int[kSlotInts * w + 1]);
      DO = max(DO, sh_int[kSlotInts * w + 2]);
    }
#pragma unroll
    for (int x = 16; x > 0; x >>= 1) {
      s = uf_add(s, shfl_uf(s, x));
      const int oM = __shfl_xor_sync(0xffffffffu, M, x);
      const int oL = __shfl_xor_sync(0xffffffffu, LCB, x);
      const int oN = __shfl_xor_sync(0xffffffffu, LCN, x);
      const int oO = __shfl_xor_sync(0xffffffffu, LCO, x);
      if (oM > M) {
        M = oM;
        LCB = oL;
        LCN = oN;
        LCO = oO;
      }
      TD = max(TD, __shfl_xor_sync(0xffffffffu, TD, x));
      DO = max(DO, __shfl_xor_sync(0xffffffffu, DO, x));
    }
    if (tid == 0) {
      out->S = s;
      out->m = M;
      out->td = TD;
      out->dego = DO;
      out->lcb = LCB;
      out->lcnt = LCN;
      out->lco = LCO;
      out->l2S = s.m ? uf_log2_q16_up(s) : 0;
    }
  }
  __syncthreads();
}

// smallest k with lg_prefix[k] >= need, by one warp: every table prime has
// 30 < log2 p < 31, so k lies in [need / 31, need / 30 + 1]; the window is scanned 32
// entries per round (one round for all but very large bounds)
__device__ int prime_count_warp(const int64_t* lg_prefix, int T, int64_t need) {
  const int lane = threadIdx.x & 31;
  int lo = (int)(need / (31ll * 65536));
  int hi = (int)(need / (30ll * 65536)) + 2;
  if (lo > T) lo = T;
  if (hi > T) hi = T;
  while (true) {
    const int k = lo + lane;
    const bool ok = (k <= hi) && lg_prefix[k] >= need;
    const unsigned b = __ballot_sync(0xffffffffu, ok);
    if (b) return lo + __ffs(b) - 1;
    if (lo + 32 > hi) return hi + 1;  // not reachable for valid tables
    lo += 32;
  }
}

// whether p divides c (c < 2^64): the high word reduced modulo p, then one Montgomery
// reduction of hi' 2^32 + lo < p 2^32, which is 0 exactly when p divides c
__device__ __forceinline__ bool divides64(uint64_t c, uint32_t p, uint32_t pinv) {
  const uint32_t hi = (uint32_t)(c >> 32) % p;
  return redc(((uint64_t)hi << 32) | (uint32_t)c, p, pinv) == 0u;
}

__global__ void __launch_bounds__(kPlanThreads) k_plan_single(Job J, Job* dst, int64_t* offs, Tables T,
                                                              int eval_group) {
  constexpr int kRows = kPlanThreads / 16;  // row slots per half
  __shared__ UF sh_uf[2][kRows];
  __shared__ int sh_int[2][kSlotInts * kRows];
  __shared__ PolySummary sf, sg;
  __shared__ Plan sP;
  __shared__ int64_t s_need;

  // the table's total, read now so that the check below does not wait for it
  const int64_t lg_all = threadIdx.x == 0 ? T.lg_prefix[T.T] : 0;
  // warm L2 with the input grids (read right below)
  if (threadIdx.x == blockDim.x - 1)
    l2_prefetch_range(J.f.c, sizeof(uint32_t) * (size_t)(J.f.dx + 1) * (J.f.dy + 1) * J.f.L);
  if (threadIdx.x == blockDim.x - 2)
    l2_prefetch_range(J.g.c, sizeof(uint32_t) * (size_t)(J.g.dx + 1) * (J.g.dy + 1) * J.g.L);
  // prime flags start at zero
  for (int i = threadIdx.x; i < J.cap_k_total; i += blockDim.x) J.pstat[i] = 0;
  // both halves run concurrently: threads [0, kPlanThreads/2) take f, the rest take g
  const bool first = threadIdx.x < kPlanThreads / 2;
  summarise_half(first ? J.f : J.g, J.var, threadIdx.x & (kPlanThreads / 2 - 1), first ? &sf : &sg,
                 sh_uf[first ? 0 : 1], sh_int[first ? 0 : 1]);
  if (threadIdx.x == 0) {
    int64_t need;
    sP = plan_head_logs(sf.l2S, sf.m, sf.td, sf.dego, sg.l2S, sg.m, sg.td, sg.dego, &need);
    s_need = need;
    if (sP.status == 0 && sP.trivial == 0 && lg_all < need) sP.status = kErrRange;
  }
  __syncthreads();
  if (threadIdx.x < 32 && sP.status == 0 && sP.trivial == 0) {
    const int lane = threadIdx.x;
    const int k = prime_count_warp(T.lg_prefix, T.T, s_need);
    // conservative count of primes that can divide a leading row; no coset spares when
    // both leading rows are monomials (they never vanish on a coset, which avoids 0)
    const bool mono = sf.lcnt == 1 && sg.lcnt == 1;
    if (lane == 0) plan_tail(sP, k, sf.lcb, sg.lcb, T.T, mono);
    __syncwarp();
    if (mono && J.f.L <= 2 && J.g.L <= 2 && sP.status == 0) {
      // both leading rows are single coefficients of at most 64 bits: count exactly the
      // table primes that divide one of them (the host plan's rule), 32 primes per round,
      // instead of the bound on how many can
      const uint64_t cf = mag_narrow(coef_ptr(J.f, J.var, sf.m, sf.lco), J.f.L);
      const uint64_t cg = mag_narrow(coef_ptr(J.g, J.var, sg.m, sg.lco), J.g.L);
      const int want = sP.k_need;
      const int Kmax = min(sP.k_total, T.T);  // the bound: want good primes lie below it
      // constants of the first four rounds of primes, all loaded at once
      uint32_t pp[4] = {1u, 1u, 1u, 1u}, pi[4] = {1u, 1u, 1u, 1u};
#pragma unroll
      for (int r = 0; r < 4; ++r) {
        const int j = 32 * r + lane;
        if (j < Kmax) {
          pp[r] = T.pc[j].p;
          pi[r] = T.pc[j].pinv;
        }
      }
      int K = Kmax, good = 0;
      for (int base = 0, r = 0; base < Kmax; base += 32, ++r) {
        const int j = base + lane;
        bool div = false;
        if (j < Kmax) {
          uint32_t p, pinv;
          if (r == 0) { p = pp[0]; pinv = pi[0]; }
          else if (r == 1) { p = pp[1]; pinv = pi[1]; }
          else if (r == 2) { p = pp[2]; pinv = pi[2]; }
          else if (r == 3) { p = pp[3]; pinv = pi[3]; }
          else { p = T.pc[j].p; pinv = T.pc[j].pinv; }
          div = divides64(cf, p, pinv) || divides64(cg, p, pinv);
        }
        const unsigned gm = __ballot_sync(0xffffffffu, j < Kmax && !div);
        const int g = __popc(gm);
        if (good + g >= want) {  // the want-th good prime lies in this round
          unsigned m = gm;
          for (int t = 1; t < want - good; ++t) m &= m - 1;  // drop the lower good primes
          K = base + __ffs(m);
          break;
        }
        good += g;
      }
      if (lane == 0 && K <= sP.k_total) sP.k_total = K;  // never above the bound
    }
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    Plan P = sP;
    // the plan must fit the capacities the host sized from the grid extents
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
    const bool run = (P.status == 0 && P.trivial == 0);
    *dst = J;
    // offsets of the stages (one job each): warp eval, smem eval, unires tiles, warp
    // intt, smem intt, crt tiles
    const bool wsize = P.logN <= kWarpLogNMax;
    for (int s = 0; s < kNumOffs; s += 2) offs[s] = 0;
    offs[kOffEvalW + 1] = (run && wsize) ? (int64_t)P.k_total * ((J.rows + eval_group - 1) / eval_group) : 0;
    offs[kOffEvalS + 1] = (run && !wsize) ? (int64_t)P.k_total * J.rows : 0;
    offs[kOffUni + 1] = run ? ((int64_t)P.k_total << P.logN) : 0;  // instances
    offs[kOffInttW + 1] = 0;  // a single job interpolates one block per prime
    offs[kOffInttS + 1] = run ? P.k_total : 0;
    offs[kOffCrt + 1] = ((int64_t)J.cap_deg + kCrtTile) / kCrtTile;
  }
  pdl_trigger();
}

// ------------------------------------------------------------------------------------
// (a) + (b): reduction, coset scaling, forward transform (decimation in frequency)
// ------------------------------------------------------------------------------------


// in-place inverse transform (decimation in time) of bit-reversed input; output natural
// order, scaled by N
// inverse transform in shared memory; Pi holds the packed inverse twiddles
// (Pi[len + j] = omega_{2 len}^-j), so the threads of a stage read consecutive words
__device__ __forceinline__ void dit_intt(uint32_t* sm, int logN, const uint32_t* Pi, const Mod M) {
  const int N = 1 << logN;
  for (int lg = 0; lg < logN; ++lg) {
    const int len = 1 << lg;
    for (int bf = threadIdx.x; bf < (N >> 1); bf += blockDim.x) {
      const int j = bf & (len - 1);
      const int i0 = ((bf >> lg) << (lg + 1)) + j;
      const int i1 = i0 + len;
      const uint32_t u = sm[i0];
      const uint32_t v = mmul(sm[i1], Pi[len + j], M);
      sm[i0] = madd(u, v, M.p);
      sm[i1] = msub(u, v, M.p);
    }
    __syncthreads();
  }
}

// Transforms of N = 1024 C points (C = 2 .. 16), one block of C warps per (prime, row).
// Thread t (of 32 C) holds the 32 points t + 32 C r in registers: the stages whose
// partners are 1024 or more apart pair registers (twiddles from the packed table in
// global memory); a transpose through shared memory then gives warp w the contiguous
// points [1024 w, 1024 w + 1024) in layout A, and the warp finishes with the 1024-point
// register transform (packed twiddles below 1024 staged in shared memory).  Blocks may
// have more warps than a job's C; the extra warps idle.
// Dynamic shared memory (words): [N_max transpose][1024 twiddles][C_max * 33 * 32 staging].
__global__ void __launch_bounds__(kEvalBigMaxWarps * 32) k_eval(const Job* jobs, WorkList wl, Tables T) {
  pdl_wait();
  extern __shared__ uint32_t sm[];
  const int cmax = blockDim.x >> 5;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  uint32_t* s_tw = sm + 1024 * cmax;            // after the largest transpose buffer
  uint32_t* sw = s_tw + 1024 + warp * (33 * 32);
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
    const int C = N >> 10;  // chunks of 1024 points; C <= cmax
    const bool isf = row <= me;
    const int e = isf ? row : row - me - 1;
    const Grid G = isf ? J->f : J->g;
    const int var = J->var;
    const PrimeConst pc = T.pc[q];
    const Mod M{pc.p, pc.pinv};
    const uint32_t* pw = T.pw + (int64_t)q * (kMaxLimbs + 1);
    const uint32_t* mpw = T.mpw + (int64_t)q * (kMaxLimbs + 1);
    const uint32_t* cp = T.cp + (int64_t)q * T.NT;
    const uint32_t* Pg = T.twp + (int64_t)q * T.NT;  // packed twiddles of this prime
    const int eo = ext_o(G, var);
    __syncthreads();  // the previous item is done with the shared buffers
    for (int t = threadIdx.x; t < 1024; t += blockDim.x) s_tw[t] = __ldg(Pg + t);
    const int tid = threadIdx.x;
    const bool active = warp < C;
    uint32_t v[32];
    if (active) {
      // residues times g^o at the points tid + 32 C r (folded modulo N)
#pragma unroll
      for (int r = 0; r < 32; ++r) {
        const int pt = tid + 32 * C * r;
        uint32_t acc = 0;
        for (int o = pt; o <= eo; o += N) {
          const uint32_t x = residue_m(coef_ptr(G, var, e, o), G.L, pw, mpw, M.p, M.pinv);
          const uint32_t s = (o < T.NT) ? __ldg(cp + o) : mpow(pc.c_m, (uint32_t)o, pc.one_m, M);
          acc = madd(acc, mmul(x, s, M), M.p);
        }
        v[r] = acc;
      }
      // stages with partners len = 512 C, 256 C, ..., 1024 apart: registers r, r + h
#pragma unroll
      for (int lh = 4; lh >= 1; --lh) {
        const int h = 1 << lh;
        if (h * C < 32) break;  // len = 32 C h < 1024: done in the chunks
        const int len = 32 * C * h;
#pragma unroll
        for (int r = 0; r < 32; ++r) {
          if (r & h) continue;
          const uint32_t w = __ldg(Pg + len + tid + 32 * C * (r & (h - 1)));
          const uint32_t a = v[r], b = v[r + h];
          v[r] = madd(a, b, M.p);
          v[r + h] = mmul(msub(a, b, M.p), w, M);
        }
      }
#pragma unroll
      for (int r = 0; r < 32; ++r) sm[tid + 32 * C * r] = v[r];
    }
    __syncthreads();
    if (active) {
#pragma unroll
      for (int r = 0; r < 32; ++r) v[r] = sm[1024 * warp + 32 * r + lane];
      // the stages above combine only points 1024 or more apart, so element e of this
      // warp's 1024 is a sum over the row's points e + 1024 k; a row reaches point
      // eo < 1024 at most, so only elements e <= eo can be nonzero: the first registers
      // of layout A, and the pruned transform skips the rest (rows of up to 96
      // coefficients, e.g. degree-64 curves)
      const uint32_t* S = T.tws + (int64_t)q * 64;
      if (eo < 64)
        warp_dif_1024_pk<0x3u>(v, sw, s_tw, S, M);
      else if (eo < 96)
        warp_dif_1024_pk<0x7u>(v, sw, s_tw, S, M);
      else
        warp_dif_1024_pk<0xffffffffu>(v, sw, s_tw, S, M);
      uint32_t* dst = J->ev + ((int64_t)q * rows + row) * N + 1024 * warp;
#pragma unroll
      for (int r = 0; r < 32; ++r) dst[32 * r + lane] = v[r];
    }
  }
  pdl_trigger();
}

// ------------------------------------------------------------------------------------
// (a) + (b) for N <= 2^kWarpLogNMax: one warp per (prime, row), one kernel per size class
// ------------------------------------------------------------------------------------
// Residues of row e of f (or g) times g^o, folded modulo N, in layout A: register r of
// lane l holds element 32 r + l.  Only the first NZ registers can be nonzero when the
// row has at most 32 NZ coefficients (and N > that count).
// NZ: registers of layout A that can hold a coefficient (the others are set to zero)
template <int R, int NZ = R>
__device__ __forceinline__ void eval_load_row(uint32_t (&v)[R], const Job* J, int q, int row,
                                              const Tables& T, uint32_t* sw, const uint32_t* s_cp,
                                              const PrimeConst& pc, const Mod& M, int N) {
  const int lane = threadIdx.x & 31;
  const int me = J->plan.me;
  const bool isf = row <= me;
  const int e = isf ? row : row - me - 1;
  const Grid G = isf ? J->f : J->g;
  const int var = J->var;
  const uint32_t* pw = T.pw + (int64_t)q * (kMaxLimbs + 1);
  const uint32_t* mpw = T.mpw + (int64_t)q * (kMaxLimbs + 1);
  const int eo = ext_o(G, var);
  // residues times g^o, folded modulo N, staged in this warp's shared slice (rolled loop)
  const int top = min(eo + 1, N);
  const int64_t gw = grid_words(G);
  for (int t = lane; t < top; t += 32) {
    uint32_t acc = 0;
    for (int o = t; o <= eo; o += N) {
      const uint32_t* cp = coef_ptr(G, var, e, o);
      if (!dbg_ok(cp >= G.c && cp + G.L <= G.c + gw, J->status, kDbgEvalIn)) continue;
      const uint32_t x = residue_m(cp, G.L, pw, mpw, M.p, M.pinv);
      const uint32_t s = (o < N) ? s_cp[o] : mpow(pc.c_m, (uint32_t)o, pc.one_m, M);
      acc = madd(acc, mmul(x, s, M), M.p);
    }
    sw[t] = acc;
  }
  __syncwarp();
#pragma unroll
  for (int r = 0; r < R; ++r) v[r] = (r < NZ && 32 * r + lane < top) ? sw[32 * r + lane] : 0u;
  __syncwarp();  // the transposes reuse sw
}

template <int R, int NZ>
__device__ __forceinline__ void eval_row_nz(const Job* J, int q, int row, const Tables& T, uint32_t* sw,
                                            const uint32_t* s_tw, const uint32_t* s_cp,
                                            const PrimeConst& pc, const Mod& M) {
  constexpr int N = 32 * R;
  constexpr uint32_t MASK = (NZ >= 32) ? 0xffffffffu : ((1u << NZ) - 1u);
  const int lane = threadIdx.x & 31;
  uint32_t v[R];
  eval_load_row<R, (NZ < R ? NZ : R)>(v, J, q, row, T, sw, s_cp, pc, M, N);
  if constexpr (R == 32)
    warp_dif_1024_pk<MASK>(v, sw, s_tw, T.tws + (int64_t)q * 64, M);
  else
    warp_dif_pk<R, MASK>(v, s_tw, T.tws + (int64_t)q * 64, M);
  uint32_t* dst = J->ev + ((int64_t)q * J->rows + row) * N;
  if (dbg_ok(((int64_t)q * J->rows + row + 1) * N <= job_ev_words(J), J->status, kDbgEvalOut)) {
#pragma unroll
    for (int r = 0; r < R; ++r) dst[32 * r + lane] = v[r];
  }
  __syncwarp();
}

// R = 1 covers every N <= 32
__device__ __forceinline__ void eval_row_small(const Job* J, int q, int row, const Tables& T,
                                               uint32_t* sw, const uint32_t* s_tw,
                                               const uint32_t* s_cp, const PrimeConst& pc,
                                               const Mod& M, int N) {
  const int lane = threadIdx.x & 31;
  uint32_t v[1];
  eval_load_row<1>(v, J, q, row, T, sw, s_cp, pc, M, N);
  if (N < 32)
    warp_dif_short(v[0], N, T.tws + (int64_t)q * 64, M);
  else
    warp_dif_pk<1, 1u>(v, s_tw, T.tws + (int64_t)q * 64, M);
  if (lane < N && dbg_ok(((int64_t)q * J->rows + row + 1) * N <= job_ev_words(J), J->status, kDbgEvalOut))
    J->ev[((int64_t)q * J->rows + row) * N + lane] = v[0];
  __syncwarp();
}

// one row of a transform of size N = 32 R (R = 1: any N <= 32), pruned by the row's
// coefficient count
template <int R>
__device__ __forceinline__ void eval_row_class(const Job* J, int q, int row, const Tables& T,
                                               uint32_t* sw, const uint32_t* s_tw,
                                               const uint32_t* s_cp, const PrimeConst& pc,
                                               const Mod& M) {
  if constexpr (R == 1) {
    eval_row_small(J, q, row, T, sw, s_tw, s_cp, pc, M, J->plan.N);
  } else {
    // how many registers of layout A the row's coefficients reach: rows of up to 64
    // coefficients share one pruned variant (a second one for rows of up to 32 would save
    // a few butterflies but doubles the code the warps of a block fetch)
    const bool isf = row <= J->plan.me;
    const int eo = ext_o(isf ? J->f : J->g, J->var);
    if (R >= 4 && eo < 64)
      eval_row_nz<R, 2>(J, q, row, T, sw, s_tw, s_cp, pc, M);
    else
      eval_row_nz<R, 32>(J, q, row, T, sw, s_tw, s_cp, pc, M);
  }
}

// R > 0: every job of the list has N = 32 R (R = 1: N <= 32).  R = 0: any N up to
// 2^kWarpLogNMax, dispatched per job (device-planned jobs, whose size the host does not
// know).  Four blocks per SM (64 registers) run the warps of several rows side by side.
template <int R>
__global__ void __launch_bounds__(kEvalThreads, 4) k_eval_w(const Job* jobs, WorkList wl,
                                                                          Tables T, PfHint pf) {
  pdl_wait();
  constexpr int NS = R == 0 ? (1 << kWarpLogNMax) : 32 * R;  // largest transform size
  __shared__ uint32_t s_stage[kEvalThreads / 32][(R == 32 || R == 0) ? 33 * 32 : NS];
  __shared__ uint32_t s_tw[NS];  // packed twiddles of this block's prime
  __shared__ uint32_t s_cp[NS];  // g^o, o < N
  const int warp = threadIdx.x >> 5;
  uint32_t* sw = s_stage[warp];
  const int nw = blockDim.x >> 5;
  const int64_t total = wl.off[wl.n];
  // the first blocks warm L2 with the tables of the later stages
  if (threadIdx.x == 0 && blockIdx.x < kPfIssuers && total > 0) {
    int kt = pf.kt, N = pf.N, kn = pf.kn;
    if (kt < 0) {  // device-planned job: take the plan of the first job
      const Plan& P0 = jobs[wl.ids ? wl.ids[0] : 0].plan;
      kt = P0.k_total;
      N = P0.N;
      kn = P0.k_need;
    }
    prefetch_late_tables(T, kt, N, kn, blockIdx.x, min((int)gridDim.x, kPfIssuers),
                         jobs[wl.ids ? wl.ids[0] : 0].status);
  }
  int cur_q = -1, cur_N = -1;
  for (int64_t item = blockIdx.x; item < total; item += gridDim.x) {
    const int ji = find_item(wl.off, wl.n, item);
    const Job* J = jobs + (wl.ids ? wl.ids[ji] : ji);
    const int64_t local = item - wl.off[ji];
    const int rows = J->rows;
    const int groups = (rows + nw - 1) / nw;
    const int q = (int)(local / groups);
    const int row = (int)(local - (int64_t)q * groups) * nw + warp;
    const int N = J->plan.N;
    // stage this prime's packed twiddles (s_tw[len + j] = omega_{2 len}^j) and coset
    // powers once per prime
    if (q != cur_q || N != cur_N) {
      __syncthreads();
      const uint32_t* twq = T.twp + (int64_t)q * T.NT;
      const uint32_t* cpq = T.cp + (int64_t)q * T.NT;
      const bool tab_ok = dbg_ok(q < T.Tt && N <= T.NT && N <= NS, J->status, kDbgEvalTab);
      for (int t = threadIdx.x; t < N && tab_ok; t += blockDim.x) {
        s_tw[t] = __ldg(twq + t);
        s_cp[t] = __ldg(cpq + t);
      }
      __syncthreads();
      cur_q = q;
      cur_N = N;
    }
    if (row >= rows) continue;
    const PrimeConst pc = T.pc[q];
    const Mod M{pc.p, pc.pinv};
    if constexpr (R > 0) {
      eval_row_class<R>(J, q, row, T, sw, s_tw, s_cp, pc, M);
    } else {
      switch (J->plan.logN) {
        case 0: case 1: case 2: case 3: case 4: case 5:
          eval_row_class<1>(J, q, row, T, sw, s_tw, s_cp, pc, M); break;
        case 6: eval_row_class<2>(J, q, row, T, sw, s_tw, s_cp, pc, M); break;
        case 7: eval_row_class<4>(J, q, row, T, sw, s_tw, s_cp, pc, M); break;
        case 8: eval_row_class<8>(J, q, row, T, sw, s_tw, s_cp, pc, M); break;
        case 9: eval_row_class<16>(J, q, row, T, sw, s_tw, s_cp, pc, M); break;
        default: eval_row_class<32>(J, q, row, T, sw, s_tw, s_cp, pc, M); break;
      }
    }
  }
  pdl_trigger();
}

// The same evaluation with independent warps: the work list counts single rows, each
// warp takes any (job, prime, row) item, and the prime's packed twiddles and coset powers
// are read through the L1 cache instead of being staged per block, so no block waits at
// a barrier for a change of prime and no warp idles at the end of a prime's rows.  Blocks
// of seven warps at 56 registers, five per SM: 35 resident warps per SM instead of 32 at
// 64 registers, which takes the 5,200 rows of 80 primes x 65 rows in one wave of 5,320
// warps (at 32 per SM, 336 rows ran in a second wave behind the first).
template <int R>
__global__ void __launch_bounds__(kEvalIwWarps * 32, kEvalIwBlocksPerSm)
    k_eval_iw(const Job* jobs, WorkList wl, Tables T, PfHint pf) {
  pdl_wait();
  constexpr int NS = R == 0 ? (1 << kWarpLogNMax) : 32 * R;  // largest transform size
  __shared__ uint32_t s_stage[kEvalIwWarps][(R == 32 || R == 0) ? 33 * 32 : NS];
  const int warp = threadIdx.x >> 5;
  uint32_t* sw = s_stage[warp];
  const int nw = blockDim.x >> 5;
  const int64_t total = wl.off[wl.n];
  if (threadIdx.x == 0 && blockIdx.x < kPfIssuers && total > 0) {
    int kt = pf.kt, N = pf.N, kn = pf.kn;
    if (kt < 0) {
      const Plan& P0 = jobs[wl.ids ? wl.ids[0] : 0].plan;
      kt = P0.k_total;
      N = P0.N;
      kn = P0.k_need;
    }
    prefetch_late_tables(T, kt, N, kn, blockIdx.x, min((int)gridDim.x, kPfIssuers),
                         jobs[wl.ids ? wl.ids[0] : 0].status);
  }
  for (int64_t item = (int64_t)blockIdx.x * nw + warp; item < total; item += (int64_t)gridDim.x * nw) {
    const int ji = find_item(wl.off, wl.n, item);
    const Job* J = jobs + (wl.ids ? wl.ids[ji] : ji);
    const int64_t local = item - wl.off[ji];
    const int rows = J->rows;
    const int q = (int)(local / rows);
    const int row = (int)(local - (int64_t)q * rows);
    const int N = J->plan.N;
    if (!dbg_ok(q < T.Tt && N <= T.NT && N <= NS, J->status, kDbgEvalTab)) continue;
    const uint32_t* tw = T.twp + (int64_t)q * T.NT;
    const uint32_t* cp = T.cp + (int64_t)q * T.NT;
    const PrimeConst pc = T.pc[q];
    const Mod M{pc.p, pc.pinv};
    if constexpr (R > 0) {
      eval_row_class<R>(J, q, row, T, sw, tw, cp, pc, M);
    } else {
      switch (J->plan.logN) {
        case 0: case 1: case 2: case 3: case 4: case 5:
          eval_row_class<1>(J, q, row, T, sw, tw, cp, pc, M); break;
        case 6: eval_row_class<2>(J, q, row, T, sw, tw, cp, pc, M); break;
        case 7: eval_row_class<4>(J, q, row, T, sw, tw, cp, pc, M); break;
        case 8: eval_row_class<8>(J, q, row, T, sw, tw, cp, pc, M); break;
        case 9: eval_row_class<16>(J, q, row, T, sw, tw, cp, pc, M); break;
        default: eval_row_class<32>(J, q, row, T, sw, tw, cp, pc, M); break;
      }
    }
  }
  pdl_trigger();
}

// ------------------------------------------------------------------------------------
// (c): univariate resultants, one per thread
// ------------------------------------------------------------------------------------
// Work list offsets count (prime, point) instances; thread i of the grid-stride sweep
// takes instance i of the flat index space and finds its job by binary search, so any
// block size works and no thread idles at the end of a job.
template <int L, class AT>
__device__ __forceinline__ void unires_instance(const Job* J, int64_t inst, const Tables& T, AT& A, AT& B) {
  const int logN = J->plan.logN;
  const int N = 1 << logN;
  const int q = (int)(inst >> logN);
  const int t = (int)(inst & (N - 1));
  const int me = J->plan.me, ne = J->plan.ne;
  const int rows = J->rows;
  if (!dbg_ok(q < T.T && q < J->plan.k_total, J->status, kDbgUniPrime)) return;
  const PrimeConst pc = T.pc[q];
  const Mod M{pc.p, pc.pinv};
  const int64_t b0 = (int64_t)q * rows * N + t;
  const uint32_t* bf = J->ev + b0;
  const uint32_t* bg = bf + (int64_t)(me + 1) * N;
  if (!dbg_ok(b0 + (int64_t)(rows - 1) * N < job_ev_words(J), J->status, kDbgUniIn)) return;
#pragma unroll
  for (int s = 0; s < Arr<L>::N; ++s) {
    A[s] = (s <= me) ? __ldg(bf + (int64_t)(me - s) * N) : 0u;
    B[s] = (s <= ne) ? __ldg(bg + (int64_t)(ne - s) * N) : 0u;
  }
  if (A[0] == 0 || B[0] == 0) J->pstat[q] = 1;  // unlucky: a leading coefficient vanishes
  uint32_t den;
  // the table's first primes have 3p < 2^32 (no fold in the fused updates)
  const uint32_t num = pc.p <= kSmallPrimeMax ? unires_numden<L, true>(A, me + 1, B, ne + 1, M, pc.one_m, &den)
                                              : unires_numden<L, false>(A, me + 1, B, ne + 1, M, pc.one_m, &den);
  if (!dbg_ok(inst < job_vals_words(J), J->status, kDbgUniOut)) return;
  if (J->den_in_ev) {  // the warp interpolation divides (one inversion per prime)
    J->vals[inst] = num;
    J->ev[b0] = den;   // this instance's own first evaluation word, read above
  } else {
    J->vals[inst] = mmul(num, minv(den, pc.one_m, M), M);
  }
}

template <int L>
__global__ void __launch_bounds__(kUniMaxThreads) k_unires(const Job* jobs, WorkList wl, Tables T) {
  pdl_wait();
  const int64_t total = wl.off[wl.n];
  for (int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; g < total;
       g += (int64_t)gridDim.x * blockDim.x) {
    const int ji = find_item(wl.off, wl.n, g);
    uint32_t A[Arr<L>::N], B[Arr<L>::N];
    unires_instance<L>(jobs + (wl.ids ? wl.ids[ji] : ji), g - wl.off[ji], T, A, B);
  }
  pdl_trigger();
}

// ------------------------------------------------------------------------------------
// the division of the univariate values (jobs with den_in_ev): Montgomery's simultaneous
// inversion.  With d_0 ... d_(n-1) the denominators of one prime, one inversion of their
// product G and prefix / suffix products give every 1/d_i = (1/G) (d_0...d_(i-1))
// (d_(i+1)...d_(n-1)); each thread holds a few values, the threads' products are joined
// with shuffles.  Every denominator is a product of nonzero leading-coefficient powers, so
// G is invertible.
// ------------------------------------------------------------------------------------

// v[k] /= d[k] for the R values of each lane of a warp (padding: d = one, any v)
template <int R>
__device__ __forceinline__ void warp_divide(uint32_t (&v)[R], const uint32_t (&d)[R], const Mod& M,
                                            uint32_t one) {
  const int lane = threadIdx.x & 31;
  uint32_t pl[R];  // pl[k] = d[0] ... d[k]
  pl[0] = d[0];
#pragma unroll
  for (int k = 1; k < R; ++k) pl[k] = mmul(pl[k - 1], d[k], M);
  uint32_t pre = pl[R - 1], suf = pl[R - 1];  // inclusive products over the lanes
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t a = __shfl_up_sync(0xffffffffu, pre, o);
    const uint32_t b = __shfl_down_sync(0xffffffffu, suf, o);
    if (lane >= o) pre = mmul(pre, a, M);
    if (lane + o < 32) suf = mmul(suf, b, M);
  }
  const uint32_t G = __shfl_sync(0xffffffffu, pre, 31);
  uint32_t epre = __shfl_up_sync(0xffffffffu, pre, 1);
  uint32_t esuf = __shfl_down_sync(0xffffffffu, suf, 1);
  if (lane == 0) epre = one;
  if (lane == 31) esuf = one;
  uint32_t inv = mmul(minv(G, one, M), mmul(epre, esuf, M), M);  // 1 / pl[R - 1]
#pragma unroll
  for (int k = R - 1; k >= 0; --k) {
    const uint32_t invd = k ? mmul(inv, pl[k - 1], M) : inv;
    v[k] = mmul(v[k], invd, M);
    if (k) inv = mmul(inv, d[k], M);
  }
}

// ------------------------------------------------------------------------------------
// prime selection + (d): inverse transform, unscaling, degree check
// ------------------------------------------------------------------------------------
__global__ void __launch_bounds__(kEvalThreads) k_intt(const Job* jobs, WorkList wl, Tables T) {
  pdl_wait();
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
    // stage the values, this prime's packed inverse twiddles and inverse coset powers
    // before the selection, so that all loads are in flight together (a prime that turns
    // out to be rejected or not needed skips the transform)
    const int logN = J->plan.logN;
    const int N = 1 << logN;
    uint32_t* sit = sm + N;
    uint32_t* sic = sit + N;
    {
      const uint32_t* src = J->vals + ((int64_t)q << logN);
      const uint32_t* itq = T.itwp + (int64_t)q * T.NT;
      const uint32_t* icq = T.icp + (int64_t)q * T.NT;
      const bool in_ok = dbg_ok(((int64_t)(q + 1) << logN) <= job_vals_words(J), J->status, kDbgInttIn) &&
                         dbg_ok(q < T.Tt && N <= T.NT, J->status, kDbgInttTab);
      for (int t = threadIdx.x; t < N && in_ok; t += blockDim.x) {  // all in flight at once
        cp_async4(sm + t, src + t);
        cp_async4(sit + t, itq + t);
        cp_async4(sic + t, icq + t);
      }
    }
    // the prime's constants, read now so that they arrive with the staged values
    const PrimeConst pc = T.pc[q];
    const uint32_t ni = T.ninv[q * (kLogNMax + 1) + logN];
    int cnt = 0;
    for (int j = threadIdx.x; j < q; j += blockDim.x) cnt += (J->pstat[j] == 0);
    if (cnt) atomicAdd(&s_rank, cnt);
    if (q == 0) {
      int g = 0;
      for (int j = threadIdx.x; j < k_total; j += blockDim.x) g += (J->pstat[j] == 0);
      if (g) atomicAdd(&s_good, g);
    }
    cp_async_wait_all();
    __syncthreads();
    const int r = s_rank;
    if (q == 0) {
      if (s_good < k_need) {
        // too few good primes: the job fails.  The selection slots no good prime fills get
        // a valid index and the job is marked, so that the reconstruction writes zeros
        // for it instead of reading unset slots.
        for (int j = s_good + (int)threadIdx.x; j < k_need; j += blockDim.x) J->sel[j] = 0;
        if (threadIdx.x == 0) {
          set_status(J->status, kErrUnlucky);
          const_cast<Job*>(J)->plan.status = kErrUnlucky;
        }
      }
      if (threadIdx.x == 0 && J->rejected) atomicAdd(J->rejected, k_total - s_good);
    }
    const bool good = J->pstat[q] == 0;
    __syncthreads();
    if (!good || r >= k_need) continue;
    const int D = J->plan.D;
    const Mod M{pc.p, pc.pinv};
    dit_intt(sm, logN, sit, M);
    uint32_t* dst = J->rmod + (int64_t)r * (D + 1);
    const bool out_ok = dbg_ok((int64_t)(r + 1) * (D + 1) <= job_rmod_words(J), J->status, kDbgInttOut);
    bool bad = false;
    for (int i = threadIdx.x; i < N; i += blockDim.x) {
      const uint32_t v = mmul(mmul(sm[i], sic[i], M), ni, M);
      if (i <= D) {
        if (out_ok) dst[i] = v;
      } else if (v != 0) {
        bad = true;
      }
    }
    if (bad) set_status(J->status, kErrInternal);
    if (threadIdx.x == 0 && dbg_ok(r < k_need, J->status, kDbgInttSel)) J->sel[r] = q;
    __syncthreads();
  }
  pdl_trigger();
}

// ------------------------------------------------------------------------------------
// prime selection + (d) for N <= 2^kWarpInttLogNMax: one warp per (job, prime), the
// inverse transform in registers (larger transforms have too few primes to fill the GPU
// one warp each; they run one block per prime)
// ------------------------------------------------------------------------------------
template <int R>
__device__ __forceinline__ void intt_prime_warp(const Job* J, int q, int r, const Tables& T,
                                                uint32_t* sw, uint32_t* Pi) {
  const int lane = threadIdx.x & 31;
  const int logN = J->plan.logN;
  const int N = 1 << logN;
  const int D = J->plan.D;
  const PrimeConst pc = T.pc[q];
  const Mod M{pc.p, pc.pinv};
  const uint32_t* src = J->vals + ((int64_t)q << logN);
  if (!dbg_ok(((int64_t)(q + 1) << logN) <= job_vals_words(J), J->status, kDbgInttIn) ||
      !dbg_ok(q < T.Tt && N <= T.NT && N <= 32 * R, J->status, kDbgInttTab))
    return;
  // the prime's packed inverse twiddles, staged in this warp's shared slice (all loads in
  // flight at once instead of one L2 round trip per butterfly)
  const uint32_t* Pg = T.itwp + (int64_t)q * T.NT;
#pragma unroll
  for (int k = 0; k < R; ++k)
    if (32 * k + lane < N) Pi[32 * k + lane] = __ldg(Pg + 32 * k + lane);
  uint32_t v[R];
#pragma unroll
  for (int k = 0; k < R; ++k) v[k] = (32 * k + lane < N) ? src[32 * k + lane] : 0u;
  if (J->den_in_ev &&
      dbg_ok(((int64_t)q * J->rows + 1) * N <= job_ev_words(J), J->status, kDbgInttIn)) {  // uniform
    const uint32_t* den = J->ev + (int64_t)q * J->rows * N;
    uint32_t d[R];
#pragma unroll
    for (int k = 0; k < R; ++k) d[k] = (32 * k + lane < N) ? den[32 * k + lane] : pc.one_m;
    warp_divide<R>(v, d, M, pc.one_m);
  }
  __syncwarp();
  if constexpr (R == 32)
    warp_dit_1024_pk(v, sw, Pi, M);
  else
    warp_dit_pk<R>(v, N, Pi, M);
  const uint32_t* icp = T.icp + (int64_t)q * T.NT;
  const uint32_t ni = T.ninv[q * (kLogNMax + 1) + logN];
  uint32_t* dst = J->rmod + (int64_t)r * (D + 1);
  const bool out_ok = dbg_ok((int64_t)(r + 1) * (D + 1) <= job_rmod_words(J), J->status, kDbgInttOut);
  bool bad = false;
#pragma unroll
  for (int k = 0; k < R; ++k) {
    const int i = 32 * k + lane;
    if (i >= N) continue;
    const uint32_t x = mmul(mmul(v[k], icp[i], M), ni, M);
    if (i <= D) {
      if (out_ok) dst[i] = x;
    } else if (x != 0) {
      bad = true;
    }
  }
  if (__any_sync(0xffffffffu, bad) && lane == 0) set_status(J->status, kErrInternal);
  if (lane == 0 && dbg_ok(r < J->plan.k_need, J->status, kDbgInttSel)) J->sel[r] = q;
  __syncwarp();  // Pi and sw are reused by the warp's next prime
}

__global__ void __launch_bounds__(kInttWarps * 32) k_intt_w(const Job* jobs, WorkList wl, Tables T) {
  pdl_wait();
  __shared__ uint32_t s_stage[kInttWarps][32];
  __shared__ uint32_t s_tw[kInttWarps][1 << kWarpInttLogNMax];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  uint32_t* sw = s_stage[warp];
  uint32_t* Pi = s_tw[warp];
  const int64_t total = wl.off[wl.n];
  for (int64_t item = (int64_t)blockIdx.x * kInttWarps + warp; item < total;
       item += (int64_t)gridDim.x * kInttWarps) {
    const int ji = find_item(wl.off, wl.n, item);
    const Job* J = jobs + (wl.ids ? wl.ids[ji] : ji);
    const int q = (int)(item - wl.off[ji]);
    const int k_need = J->plan.k_need, k_total = J->plan.k_total;
    // rank of prime q among the good primes (ballots over the prime flags); the warp of
    // prime 0 also checks that enough good primes exist
    int r = 0;
    for (int j0 = 0; j0 < q; j0 += 32) {
      const int j = j0 + lane;
      r += __popc(__ballot_sync(0xffffffffu, j < q && J->pstat[j] == 0));
    }
    if (q == 0) {
      int good = 0;
      for (int j0 = 0; j0 < k_total; j0 += 32) {
        const int j = j0 + lane;
        good += __popc(__ballot_sync(0xffffffffu, j < k_total && J->pstat[j] == 0));
      }
      if (good < k_need) {  // as in k_intt: a failed job with valid slots
        for (int j = good + lane; j < k_need; j += 32) J->sel[j] = 0;
        if (lane == 0) {
          set_status(J->status, kErrUnlucky);
          const_cast<Job*>(J)->plan.status = kErrUnlucky;
        }
      }
      if (lane == 0 && J->rejected) atomicAdd(J->rejected, k_total - good);
    }
    if (J->pstat[q] != 0 || r >= k_need) continue;  // uniform across the warp
    switch (J->plan.logN) {
      case 0: case 1: case 2: case 3: case 4: case 5: intt_prime_warp<1>(J, q, r, T, sw, Pi); break;
      case 6: intt_prime_warp<2>(J, q, r, T, sw, Pi); break;
      case 7: intt_prime_warp<4>(J, q, r, T, sw, Pi); break;
      case 8: intt_prime_warp<8>(J, q, r, T, sw, Pi); break;
      default: intt_prime_warp<16>(J, q, r, T, sw, Pi); break;
    }
  }
  pdl_trigger();
}

// ------------------------------------------------------------------------------------
// (e): mixed-radix reconstruction, a tile of kCrtTile coefficients per block
// ------------------------------------------------------------------------------------
// Shared memory of one block (words): [inv k*k when k <= kCrtInvSmem][X k*kCrtTile]
// [p k][pinv k][sel k][V 3*lmax per warp].  Garner's digits are computed for the whole
// tile with the primes spread over the block; each warp then turns one coefficient's
// digits d_j into c = sum_j d_j P_j (P_j = p_0 ... p_{j-1}, the context's prefix-product
// table) -- an exact dot product per output limb -- and one lane propagates the carries.
// Jobs that rejected a prime among their first k use their own prime order; for them
// the warp runs Horner's rule c = c p_j + d_j from the top digit instead.
__device__ __forceinline__ void crt_carry_out(const uint32_t* V, int nlimbs, int cap, bool neg,
                                              uint32_t* out, bool* ovf) {
  // V holds, per limb l, a 96-bit value (V[3l], V[3l+1], V[3l+2]) of weight 2^(32 l)
  uint64_t carry_lo = 0;  // pending carry (up to 66 bits: lo 64 + hi 2)
  uint32_t carry_hi = 0;
  for (int l = 0; l < cap; ++l) {
    uint64_t a = 0;
    uint32_t ah = 0;
    if (l < nlimbs) {
      a = (uint64_t)V[3 * l] | ((uint64_t)V[3 * l + 1] << 32);
      ah = V[3 * l + 2];
    }
    // s = a + carry (96-bit)
    const uint64_t s = a + carry_lo;
    const uint32_t sh = ah + carry_hi + (s < a ? 1u : 0u);
    const uint32_t limb = (uint32_t)s;
    out[l] = neg ? ~limb : limb;
    carry_lo = (s >> 32) | ((uint64_t)sh << 32);
    carry_hi = 0;
  }
  if (carry_lo != 0) *ovf = true;
}

// skip_big: leave table-ordered jobs with k_need > kCrtWarpMaxK to the weighted-sum
// kernels of many primes (this kernel then serves their jobs with rejected primes)
__global__ void __launch_bounds__(kCrtWarps * 32) k_crt(const Job* jobs, WorkList wl, Tables T,
                                                        int kmax, int lmax, int staged, int skip_big) {
  pdl_wait();
  extern __shared__ uint32_t smc[];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int nthr = blockDim.x;
  const bool inv_in_smem = staged != 0;
  uint32_t* sinv = smc;
  uint32_t* X = smc + (inv_in_smem ? (size_t)kmax * kmax : 0);
  uint32_t* pq = X + (size_t)kmax * kCrtTile;
  uint32_t* pinvq = pq + kmax;
  uint32_t* selq = pinvq + kmax;
  uint32_t* spp = selq + kmax;  // [kmax + 1][lmax] prefix rows when staged (table order)
  uint32_t* V = spp + (inv_in_smem ? (size_t)(kmax + 1) * lmax : 0) + (size_t)warp * 3 * lmax;
  __shared__ int s_neg[kCrtTile];
  const int64_t total = wl.off[wl.n];
  for (int64_t item = blockIdx.x; item < total; item += gridDim.x) {
    const int ji = find_item(wl.off, wl.n, item);
    const Job* J = jobs + (wl.ids ? wl.ids[ji] : ji);
    const int i0 = (int)(item - wl.off[ji]) * kCrtTile;
    const int cap = J->cap_limbs;
    const Plan P = J->plan;
    const int ncoef = min(kCrtTile, J->cap_deg + 1 - i0);
    if (P.status != 0 || P.trivial != 0 || i0 > P.D) {
      for (int t = threadIdx.x; t < ncoef * cap; t += nthr) {
        const int c = t / cap, l = t - c * cap;
        const uint32_t v0 = (P.status == 0 && P.trivial == 2 && i0 + c == 0 && l == 0) ? 1u : 0u;
        J->out[(int64_t)(i0 + c) * cap + l] = v0;
      }
      continue;  // uniform across the block
    }
    const int k = P.k_need, D = P.D, Tg = T.Tg;
    const int nvalid = min(ncoef, D + 1 - i0);  // coefficients of this tile that exist
    // ---- stage residues, prime constants and (small k) the inverse table
    for (int j = threadIdx.x; j < k; j += nthr) {
      const int s = J->sel[j];
      const PrimeConst pc = T.pc[s];
      pq[j] = pc.p;
      pinvq[j] = pc.pinv;
      selq[j] = (uint32_t)s;
    }
    for (int t = threadIdx.x; t < k * kCrtTile; t += nthr) {
      const int j = t / kCrtTile, c = t - j * kCrtTile;
      X[t] = (c < nvalid) ? J->rmod[(int64_t)j * (D + 1) + i0 + c] : 0u;
    }
    __syncthreads();
    const bool table_order = (selq[k - 1] == (uint32_t)(k - 1));
    if (skip_big && table_order && k > kCrtWarpMaxK) {  // uniform across the block
      __syncthreads();  // every thread has read selq before the next item restages it
      continue;
    }
    const int nl = min(min(P.out_limbs, lmax), T.LPP);  // limbs of the magnitude
    if (inv_in_smem) {
      // all loads of the staging are independent: unrolled so many are in flight
#pragma unroll 4
      for (int t = threadIdx.x; t < k * k; t += nthr) {
        const int a = t / k, b = t - a * k;
        sinv[t] = __ldg(T.ginv + (int64_t)selq[a] * Tg + selq[b]);
      }
      if (table_order) {
#pragma unroll 4
        for (int t = threadIdx.x; t < k * nl; t += nthr) {
          const int j = t / nl, l = t - j * nl;
          spp[j * nl + l] = __ldg(T.pp + (int64_t)j * T.LPP + l);
        }
      }
    }
    __syncthreads();
    // ---- Garner: x_q <- (x_q - d_j) p_j^-1 mod p_q for q > j, whole tile
    {
      const int c = threadIdx.x % kCrtTile;
      const int grp = threadIdx.x / kCrtTile;
      const int ngrp = nthr / kCrtTile;
      for (int j = 0; j < k - 1; ++j) {
        const uint32_t d = X[j * kCrtTile + c];
        for (int q = j + 1 + grp; q < k; q += ngrp) {
          const uint32_t p = pq[q];
          const uint32_t dd = d >= p ? d - p : d;
          const uint32_t w = inv_in_smem ? sinv[j * k + q] : T.ginv[(int64_t)selq[j] * Tg + selq[q]];
          const Mod M{p, pinvq[q]};
          X[q * kCrtTile + c] = mmul(msub(X[q * kCrtTile + c], dd, p), w, M);
        }
        __syncthreads();
      }
    }
    // ---- per coefficient (warp c): sign, complement, conversion to limbs
    for (int c = warp; c < ncoef; c += nthr / 32) {
      uint32_t* out = J->out + (int64_t)(i0 + c) * cap;
      if (c >= nvalid) {  // above the degree bound
        for (int l = lane; l < cap; l += 32) out[l] = 0u;
        continue;
      }
      int hi = -1;
      for (int j = lane; j < k; j += 32)
        if (X[j * kCrtTile + c] != (pq[j] - 1) / 2) hi = j;
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) hi = max(hi, __shfl_xor_sync(0xffffffffu, hi, o));
      const bool neg = hi >= 0 && X[hi * kCrtTile + c] > (pq[hi] - 1) / 2;
      __syncwarp();
      if (neg)
        for (int j = lane; j < k; j += 32) X[j * kCrtTile + c] = pq[j] - 1 - X[j * kCrtTile + c];
      __syncwarp();
      bool ovf = false;
      if (table_order) {
        // c = sum_j d_j P_j.  P_j < 2^(31 j), so limb l of P_j vanishes unless
        // 31 j > 32 l; a 32-limb chunk starts at the first row its lowest limb needs, so
        // all lanes read the same row (coalesced) and the rows' zero limbs add nothing
        for (int l = lane; l < (nl + 31) / 32 * 32; l += 32) {
          uint64_t acc = 0;
          uint32_t ah = 0;
          const int lb = l - lane;
          const int j0 = max(0, (32 * lb - 31) / 31);
          const int lc = min(l, T.LPP - 1);
#pragma unroll 8
          for (int j = j0; j < k; ++j) {
            const uint32_t pl = inv_in_smem ? (l < nl ? spp[j * nl + l] : 0u)
                                            : __ldg(T.pp + (int64_t)j * T.LPP + lc);
            const uint64_t prod = (uint64_t)X[j * kCrtTile + c] * pl;
            const uint64_t s = acc + prod;
            ah += (s < acc) ? 1u : 0u;
            acc = s;
          }
          if (l < nl) {
            V[3 * l] = (uint32_t)acc;
            V[3 * l + 1] = (uint32_t)(acc >> 32);
            V[3 * l + 2] = ah;
          }
        }
        __syncwarp();
        if (lane == 0) crt_carry_out(V, nl, cap, neg, out, &ovf);
      } else {
        // Horner from the top digit; limbs spread over lanes, ballot carries
        uint32_t* limb = V;
        for (int l = lane; l < cap; l += 32) limb[l] = 0;
        __syncwarp();
        int alen = 0;
        for (int j = k - 1; j >= 0; --j) {
          const uint32_t pj = pq[j];
          alen = alen + 1 < cap ? alen + 1 : cap;
          uint32_t cin = 0, hprev = X[j * kCrtTile + c];
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
            const uint32_t Xm = G | Pm;
            const uint64_t S = (uint64_t)Xm + G + cin;
            const uint32_t C = (uint32_t)S ^ Xm ^ G;
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
        for (int l = lane; l < cap; l += 32) out[l] = neg ? ~limb[l] : limb[l];
      }
      if (__any_sync(0xffffffffu, ovf) && lane == 0) set_status(J->status, kErrInternal);
      __syncwarp();
    }
    __syncthreads();
  }
  pdl_trigger();
}

// ------------------------------------------------------------------------------------
// (e) for up to kCrtWarpMaxK primes: one warp per coefficient, Garner in registers
// ------------------------------------------------------------------------------------
// Adds the three-word column sums V_l = a_l + b_l 2^32 + c_l 2^64 (weight 2^(32 l)) into
// limbs: the result is A + (B shifted one limb) + (C shifted two limbs), two additions
// whose one-bit carries are resolved per 32-limb chunk with generate/propagate ballots.

// The prefix products P_j (table order) are read from the context's table through L1
// (ppg: row j at ppg + j * lpp), not staged: that keeps the block's shared memory small.
template <int S>
__device__ __forceinline__ void crt_coef_warp(const Job* J, const Plan& P, int i, int c,
                                              const uint32_t* Xt, const uint32_t* sinv,
                                              const uint32_t* ppg, int lpp, int nl, const uint32_t* pq,
                                              const uint32_t* pinvq, uint32_t* sd,
                                              uint32_t* Vw, bool table_order) {
  const int lane = threadIdx.x & 31;
  const int k = P.k_need;
  const int cap = J->cap_limbs;
  uint32_t x[S], p[S], pinv[S];
#pragma unroll
  for (int s = 0; s < S; ++s) {
    const int q = 32 * s + lane;
    x[s] = q < k ? Xt[q * kCrtTile + c] : 0u;
    p[s] = q < k ? pq[q] : 3u;
    pinv[s] = q < k ? pinvq[q] : 0u;
  }
  // Garner: x_q <- (x_q - d_j) p_j^-1 mod p_q for q > j; the digit d_j sits in lane j%32
#pragma unroll
  for (int s0 = 0; s0 < S; ++s0) {
    const int jend = min(32, k - 1 - 32 * s0);
    for (int jj = 0; jj < jend; ++jj) {
      const int j = 32 * s0 + jj;
      const uint32_t d = __shfl_sync(0xffffffffu, x[s0], jj);
#pragma unroll
      for (int s = s0; s < S; ++s) {
        const int q = 32 * s + lane;
        if (q > j && q < k) {
          const uint32_t dd = d >= p[s] ? d - p[s] : d;
          const Mod M{p[s], pinv[s]};
          x[s] = mmul(msub(x[s], dd, p[s]), sinv[j * k + q], M);
        }
      }
    }
  }
  // sign: digits above ((p_j - 1) / 2)_j from the top mean the value exceeds (P - 1) / 2
  int hi = -1;
#pragma unroll
  for (int s = 0; s < S; ++s) {
    const int q = 32 * s + lane;
    const unsigned b = __ballot_sync(0xffffffffu, q < k && x[s] != (p[s] - 1) / 2);
    if (b) hi = 32 * s + 31 - __clz((int)b);
  }
  uint32_t top = 0, tophalf = 0;
#pragma unroll
  for (int s = 0; s < S; ++s) {
    const uint32_t xv = __shfl_sync(0xffffffffu, x[s], hi & 31);
    const uint32_t pv = __shfl_sync(0xffffffffu, p[s], hi & 31);
    if (hi >= 0 && (hi >> 5) == s) {
      top = xv;
      tophalf = (pv - 1) / 2;
    }
  }
  const bool neg = hi >= 0 && top > tophalf;
#pragma unroll
  for (int s = 0; s < S; ++s) {
    const int q = 32 * s + lane;
    if (q < k) sd[q] = neg ? p[s] - 1 - x[s] : x[s];
  }
  __syncwarp();
  uint32_t* out = J->out + (int64_t)i * cap;
  bool ovf = false;
  if (table_order) {
    // column sums V_l = sum_j d_j P_j[l], kept as three words in registers per chunk
    uint32_t cin1 = 0, cin2 = 0, bprev = 0, cprev1 = 0, cprev2 = 0;
    for (int b0 = 0; b0 < cap; b0 += 32) {
      const int l = b0 + lane;
      uint64_t acc = 0;
      uint32_t ah = 0;
      if (b0 < nl) {
        const int j0 = max(0, (32 * b0 - 31) / 31);
#pragma unroll 8
        for (int j = j0; j < k; ++j) {
          const uint32_t pl = l < nl ? __ldg(ppg + (int64_t)j * lpp + l) : 0u;
          const uint64_t prod = (uint64_t)sd[j] * pl;
          const uint64_t s = acc + prod;
          ah += (s < acc) ? 1u : 0u;
          acc = s;
        }
      }
      const uint32_t a = (uint32_t)acc, bw = (uint32_t)(acc >> 32), cw = ah;
      // B shifted by one limb, C by two (values of the previous chunk feed lanes 0, 1)
      uint32_t bin = __shfl_up_sync(0xffffffffu, bw, 1);
      uint32_t cin_w = __shfl_up_sync(0xffffffffu, cw, 2);
      const uint32_t c31 = __shfl_sync(0xffffffffu, cw, 31), c30 = __shfl_sync(0xffffffffu, cw, 30);
      const uint32_t b31 = __shfl_sync(0xffffffffu, bw, 31);
      if (lane == 0) {
        bin = bprev;
        cin_w = cprev2;
      }
      if (lane == 1) cin_w = cprev1;
      uint32_t r = ballot_add(a, bin, cin1, lane);
      r = ballot_add(r, cin_w, cin2, lane);
      if (l < cap) out[l] = neg ? ~r : r;
      bprev = b31;
      cprev2 = c30;
      cprev1 = c31;
    }
    if (cin1 || cin2 || bprev || cprev1 || cprev2) ovf = true;
  } else {
    // Horner from the top digit (jobs that rejected a prime among their first k)
    uint32_t* limb = Vw;
    for (int l = lane; l < cap; l += 32) limb[l] = 0;
    __syncwarp();
    int alen = 0;
    for (int j = k - 1; j >= 0; --j) {
      const uint32_t pj = pq[j];
      alen = alen + 1 < cap ? alen + 1 : cap;
      uint32_t cin = 0, hprev = sd[j];
      for (int b = 0; b < alen; b += 32) {
        const int l = b + lane;
        const uint32_t v = l < alen ? limb[l] : 0u;
        const uint64_t prod = (uint64_t)v * pj;
        const uint32_t lo = (uint32_t)prod, hi32 = (uint32_t)(prod >> 32);
        uint32_t hin = __shfl_up_sync(0xffffffffu, hi32, 1);
        if (lane == 0) hin = hprev;
        const uint32_t res = ballot_add(lo, hin, cin, lane);
        __syncwarp();
        if (l < alen)
          limb[l] = res;
        else if (l == alen && res != 0)
          ovf = true;
        hprev = __shfl_sync(0xffffffffu, hi32, 31);
      }
      if ((alen & 31) == 0 && (cin != 0 || hprev != 0)) ovf = true;
      __syncwarp();
    }
    for (int l = lane; l < cap; l += 32) out[l] = neg ? ~limb[l] : limb[l];
  }
  if (__any_sync(0xffffffffu, ovf) && lane == 0) set_status(J->status, kErrInternal);
  __syncwarp();
}

// Weighted-sum reconstruction of one coefficient (table order, k <= WK): with
// P = p_0 ... p_{k-1}, M_i = P / p_i and y_i = M_i^-1 mod p_i,
//   c = sum_i t_i M_i - q P,  t_i = r_i y_i mod p_i,  q = round(sum_i t_i / p_i),
// where sum_i t_i / p_i is taken in Q62 fixed point (t_i floor(2^62 / p_i)); its error is
// below k 2^-31, far inside the 1/4 margin that prod p > 4B leaves around an integer, so
// q is exact.  c comes out directly in two's complement.  Msm holds M_k (k rows of L
// limbs), sd receives t_i.

// sy, sq62, sPk: y_k[q], floor(2^62 / p_q) and the limbs of P_k, staged by the block
template <int S>
__device__ __forceinline__ void crt_ws_warp(const Job* J, const Plan& P, int i, int c,
                                            const uint32_t* Xt, const uint32_t* Msm, int L,
                                            const uint32_t* pq, const uint32_t* pinvq,
                                            uint32_t* sd, const uint32_t* sy, const uint32_t* sq62,
                                            const uint32_t* sPk) {
  const int lane = threadIdx.x & 31;
  const int k = P.k_need;
  const int cap = J->cap_limbs;
  uint64_t flo = 0;
  uint32_t fhi = 0;
#pragma unroll
  for (int s = 0; s < S; ++s) {
    const int q = 32 * s + lane;
    if (q < k) {
      const Mod M{pq[q], pinvq[q]};
      const uint32_t t = mmul(Xt[q * kCrtTile + c], sy[q], M);
      sd[q] = t;
      const uint64_t prod = (uint64_t)t * sq62[q];
      flo += prod;
      fhi += (flo < prod) ? 1u : 0u;
    }
  }
#pragma unroll
  for (int x = 16; x > 0; x >>= 1) {
    const uint64_t olo = __shfl_xor_sync(0xffffffffu, flo, x);
    const uint32_t ohi = __shfl_xor_sync(0xffffffffu, fhi, x);
    const uint64_t nlo = flo + olo;
    fhi = fhi + ohi + (nlo < flo ? 1u : 0u);
    flo = nlo;
  }
  // round(S / 2^62) with S = fhi 2^64 + flo
  const uint64_t half = 1ull << 61;
  const uint64_t rlo = flo + half;
  const uint32_t rhi = fhi + (rlo < flo ? 1u : 0u);
  const uint32_t qr = (rhi << 2) | (uint32_t)(rlo >> 62);
  __syncwarp();
  uint32_t* out = J->out + (int64_t)i * cap;
  uint32_t cin1 = 0, cin2 = 0, cq = 0, bsub = 0;
  uint32_t bprev = 0, cprev1 = 0, cprev2 = 0, qhprev = 0;
  for (int b0 = 0; b0 < cap; b0 += 32) {
    const int l = b0 + lane;
    uint64_t acc = 0;
    uint32_t ah = 0;
    if (b0 < L) {
      // two independent accumulation chains, each adding the sum of two products at a
      // time: t_q < p_q < 2^31 and a limb is below 2^32, so a product is below 2^63 and the
      // sum of two fits 64 bits (one carry test per two products)
      uint64_t a0 = 0, a1 = 0;
      uint32_t h0 = 0, h1 = 0;
      const int lc = l < L ? l : 0;
      const uint32_t keep = l < L ? 0xffffffffu : 0u;
      int q = 0;
#pragma unroll 2
      for (; q + 3 < k; q += 4) {
        const uint64_t pa = (uint64_t)sd[q] * (Msm[q * L + lc] & keep) +
                            (uint64_t)sd[q + 1] * (Msm[(q + 1) * L + lc] & keep);
        const uint64_t pb = (uint64_t)sd[q + 2] * (Msm[(q + 2) * L + lc] & keep) +
                            (uint64_t)sd[q + 3] * (Msm[(q + 3) * L + lc] & keep);
        const uint64_t s0 = a0 + pa, s1 = a1 + pb;
        h0 += (s0 < a0) ? 1u : 0u;
        h1 += (s1 < a1) ? 1u : 0u;
        a0 = s0;
        a1 = s1;
      }
      for (; q < k; ++q) {
        const uint64_t p0 = (uint64_t)sd[q] * (Msm[q * L + lc] & keep);
        const uint64_t s0 = a0 + p0;
        h0 += (s0 < a0) ? 1u : 0u;
        a0 = s0;
      }
      acc = a0 + a1;
      ah = h0 + h1 + ((acc < a0) ? 1u : 0u);
    }
    // c' = sum_i t_i M_i from the three-word column sums
    const uint32_t a = (uint32_t)acc, bw = (uint32_t)(acc >> 32), cw = ah;
    uint32_t bin = __shfl_up_sync(0xffffffffu, bw, 1);
    uint32_t cin_w = __shfl_up_sync(0xffffffffu, cw, 2);
    const uint32_t c31 = __shfl_sync(0xffffffffu, cw, 31), c30 = __shfl_sync(0xffffffffu, cw, 30);
    const uint32_t b31 = __shfl_sync(0xffffffffu, bw, 31);
    if (lane == 0) {
      bin = bprev;
      cin_w = cprev2;
    }
    if (lane == 1) cin_w = cprev1;
    uint32_t r = ballot_add(a, bin, cin1, lane);
    r = ballot_add(r, cin_w, cin2, lane);
    bprev = b31;
    cprev2 = c30;
    cprev1 = c31;
    // q P (q < 2^13): limb l = lo(q P_l) + hi(q P_{l-1}) + carry
    const uint64_t qp = (uint64_t)qr * (l < L ? sPk[l] : 0u);
    uint32_t qh = __shfl_up_sync(0xffffffffu, (uint32_t)(qp >> 32), 1);
    const uint32_t qh31 = __shfl_sync(0xffffffffu, (uint32_t)(qp >> 32), 31);
    if (lane == 0) qh = qhprev;
    qhprev = qh31;
    const uint32_t qpl = ballot_add((uint32_t)qp, qh, cq, lane);
    // c = c' - q P, two's complement
    const uint32_t res = ballot_sub(r, qpl, bsub, lane);
    if (l < cap) out[l] = res;
  }
  __syncwarp();
}

// Block: kCrtTile coefficients of one job, one warp each.  Shared memory (words):
// [inv or M_k: k*(k+1)][X k*kCrtTile][p k][pinv k][sel k][digits kCrtTile*k]
// [limbs kCrtTile*lmax][y_k k][q62 k][P_k k+4]
template <int TILE>
__global__ void __launch_bounds__(TILE * 32) k_crt_w(const Job* jobs, WorkList wl, Tables T,
                                                         int kmax, int lmax) {
  pdl_wait();
  extern __shared__ uint32_t smc[];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int nthr = blockDim.x;
  constexpr int tile = TILE;  // coefficients per block, one warp each (<= kCrtTile)
  uint32_t* sinv = smc;  // kmax (kmax + 1) words: Garner's k x k inverses or M_k
  uint32_t* X = sinv + (size_t)kmax * (kmax + 1);
  uint32_t* pq = X + (size_t)kmax * kCrtTile;
  uint32_t* pinvq = pq + kmax;
  uint32_t* selq = pinvq + kmax;
  uint32_t* sd = selq + kmax + (size_t)warp * kmax;
  uint32_t* Vw = selq + kmax + (size_t)kCrtTile * kmax + (size_t)warp * lmax;
  uint32_t* sy = selq + kmax + (size_t)kCrtTile * kmax + (size_t)kCrtTile * lmax;  // weighted sum
  uint32_t* sq62 = sy + kmax;
  uint32_t* sPk = sq62 + kmax;  // kmax + 4 words
  const int64_t total = wl.off[wl.n];
  for (int64_t item = blockIdx.x; item < total; item += gridDim.x) {
    const int ji = find_item(wl.off, wl.n, item);
    const Job* J = jobs + (wl.ids ? wl.ids[ji] : ji);
    const int i0 = (int)(item - wl.off[ji]) * tile;
    const int cap = J->cap_limbs;
    const Plan P = J->plan;
    const int ncoef = min(tile, J->cap_deg + 1 - i0);
    if (P.status != 0 || P.trivial != 0 || i0 > P.D) {
      for (int t = threadIdx.x; t < ncoef * cap; t += nthr) {
        const int c = t / cap, l = t - c * cap;
        const uint32_t v0 = (P.status == 0 && P.trivial == 2 && i0 + c == 0 && l == 0) ? 1u : 0u;
        J->out[(int64_t)(i0 + c) * cap + l] = v0;
      }
      continue;  // uniform across the block
    }
    const int k = P.k_need, D = P.D, Tg = T.Tg;
    const int nvalid = min(ncoef, D + 1 - i0);
    const int nl = min(min(P.out_limbs, lmax), T.LPP);
    // Every staging copy is issued before any is waited for: the tables and the residues
    // go to shared memory by asynchronous copies (all in flight at once, one round trip),
    // while the selected primes' constants come through registers.
    const int L = ws_len(k);
    if (k <= T.WK &&
        dbg_ok(T.ws_moff[k] + (int64_t)k * L <= T.ws_m_words && k <= T.Tg && L <= kmax + 4 &&
                   (int64_t)k * L <= (int64_t)kmax * (kmax + 1),
               J->status, kDbgCrtWs)) {
      // weighted-sum tables (they depend on k only; the Garner path below overwrites them
      // when the selected primes are not the first k): M_k is k rows of L limbs, contiguous
      const uint32_t* Mk = T.ws_m + T.ws_moff[k];
      const int n = k * L;
      for (int t = threadIdx.x; t < n; t += nthr) cp_async4(sinv + t, Mk + t);
      const uint32_t* yk = T.ws_y + T.ws_yoff[k];
      for (int t = threadIdx.x; t < k; t += nthr) {
        cp_async4(sy + t, yk + t);
        cp_async4(sq62 + t, T.q62 + t);
      }
      const uint32_t* Pk = T.pp + (int64_t)k * T.LPP;
      for (int t = threadIdx.x; t < L; t += nthr) {
        if (t < T.LPP)
          cp_async4(sPk + t, Pk + t);
        else
          sPk[t] = 0u;
      }
    }
    const bool x_ok = dbg_ok((int64_t)(k - 1) * (D + 1) + i0 + nvalid <= job_rmod_words(J), J->status, kDbgCrtIn);
    for (int t = threadIdx.x; t < k * kCrtTile; t += nthr) {  // columns >= tile stay unused
      const int j = t / kCrtTile, c = t - j * kCrtTile;
      if (c < nvalid && x_ok)
        cp_async4(X + t, J->rmod + (int64_t)j * (D + 1) + i0 + c);
      else
        X[t] = 0u;
    }
    for (int j = threadIdx.x; j < k; j += nthr) {
      // the constants of table prime j are read together with the slot: a table-ordered
      // selection (the usual one) then needs no second round trip
      const int js = j < T.Tg ? j : 0;
      const uint32_t pj = T.pc[js].p, pinvj = T.pc[js].pinv;
      int s = J->sel[j];
      if (!dbg_ok(s >= 0 && s < T.Tg && s < J->plan.k_total, J->status, kDbgCrtSel) || s < 0 || s >= T.Tg)
        s = 0;  // never read outside the tables, whatever the slot holds
      pq[j] = s == j ? pj : T.pc[s].p;
      pinvq[j] = s == j ? pinvj : T.pc[s].pinv;
      selq[j] = (uint32_t)s;
    }
    cp_async_wait_all();
    __syncthreads();
    const bool table_order = (selq[k - 1] == (uint32_t)(k - 1));
    // weighted-sum path for table-ordered jobs with tabulated k; Garner otherwise
    const bool ws = table_order && k <= T.WK;
    if (!ws) {
      dbg_ok(k <= kmax && nl <= lmax && nl <= T.LPP && k <= Tg, J->status, kDbgCrtGinv);
      for (int a = warp; a < k; a += nthr / 32) {
        const int64_t rowa = (int64_t)selq[a] * Tg;
#pragma unroll 4
        for (int b = lane; b < k; b += 32) sinv[a * k + b] = __ldg(T.ginv + rowa + selq[b]);
      }
    }
    __syncthreads();
    for (int c = warp; c < ncoef; c += nthr / 32) {
      if (!dbg_ok(i0 + c <= J->cap_deg && J->cap_limbs <= lmax, J->status, kDbgCrtOut)) continue;
      if (c >= nvalid) {  // above the degree bound
        uint32_t* out = J->out + (int64_t)(i0 + c) * cap;
        for (int l = lane; l < cap; l += 32) out[l] = 0u;
        continue;
      }
      if (ws) {
        switch ((k + 31) >> 5) {
          case 1: crt_ws_warp<1>(J, P, i0 + c, c, X, sinv, L, pq, pinvq, sd, sy, sq62, sPk); break;
          case 2: crt_ws_warp<2>(J, P, i0 + c, c, X, sinv, L, pq, pinvq, sd, sy, sq62, sPk); break;
          case 3: crt_ws_warp<3>(J, P, i0 + c, c, X, sinv, L, pq, pinvq, sd, sy, sq62, sPk); break;
          case 4: crt_ws_warp<4>(J, P, i0 + c, c, X, sinv, L, pq, pinvq, sd, sy, sq62, sPk); break;
          default: crt_ws_warp<5>(J, P, i0 + c, c, X, sinv, L, pq, pinvq, sd, sy, sq62, sPk); break;
        }
        continue;
      }
      switch ((k + 31) >> 5) {
        case 1: crt_coef_warp<1>(J, P, i0 + c, c, X, sinv, T.pp, T.LPP, nl, pq, pinvq, sd, Vw, table_order); break;
        case 2: crt_coef_warp<2>(J, P, i0 + c, c, X, sinv, T.pp, T.LPP, nl, pq, pinvq, sd, Vw, table_order); break;
        case 3: crt_coef_warp<3>(J, P, i0 + c, c, X, sinv, T.pp, T.LPP, nl, pq, pinvq, sd, Vw, table_order); break;
        case 4: crt_coef_warp<4>(J, P, i0 + c, c, X, sinv, T.pp, T.LPP, nl, pq, pinvq, sd, Vw, table_order); break;
        default: crt_coef_warp<5>(J, P, i0 + c, c, X, sinv, T.pp, T.LPP, nl, pq, pinvq, sd, Vw, table_order); break;
      }
    }
    __syncthreads();
  }
  pdl_trigger();
}

static thread_local bool tl_pdl = false;
void set_launch_pdl(bool on) { tl_pdl = on; }

// launch with programmatic stream serialisation when enabled for this thread's enqueue
template <typename... KArgs, typename... Args>
static void launch_k(void (*kern)(KArgs...), int grid, int block, size_t smem, cudaStream_t s,
                     Args... args) {
  if (tl_pdl) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(block);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    cudaLaunchKernelEx(&cfg, kern, args...);
  } else {
    kern<<<grid, block, smem, s>>>(args...);
  }
}

void launch_crt_w(int grid, int tile, size_t smem, cudaStream_t s, const Job* jobs, WorkList wl,
                  Tables T, int kmax, int lmax) {
  switch (tile) {
    case 1: launch_k(k_crt_w<1>, grid, 32, smem, s, jobs, wl, T, kmax, lmax); break;
    case 2: launch_k(k_crt_w<2>, grid, 64, smem, s, jobs, wl, T, kmax, lmax); break;
    case 4: launch_k(k_crt_w<4>, grid, 128, smem, s, jobs, wl, T, kmax, lmax); break;
    default: launch_k(k_crt_w<8>, grid, 256, smem, s, jobs, wl, T, kmax, lmax); break;
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
static int occ1(int threads) {
  int b = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_unires<L>, threads, 0);
  return b > 0 ? b : 1;
}

int uni_occupancy(int cls, int threads) {
  switch (cls) {
    case 0: return occ1<8>(threads);
    case 1: return occ1<16>(threads);
    case 2: return occ1<24>(threads);
    case 3: return occ1<33>(threads);
    case 4: return occ1<48>(threads);
    default: return occ1<65>(threads);
  }
}


void launch_uni(int cls, int grid, int threads, cudaStream_t s, const Job* jobs, WorkList wl, Tables T) {
  switch (cls) {
    case 0: launch_k(k_unires<8>, grid, threads, 0, s, jobs, wl, T); break;
    case 1: launch_k(k_unires<16>, grid, threads, 0, s, jobs, wl, T); break;
    case 2: launch_k(k_unires<24>, grid, threads, 0, s, jobs, wl, T); break;
    case 3: launch_k(k_unires<33>, grid, threads, 0, s, jobs, wl, T); break;
    case 4: launch_k(k_unires<48>, grid, threads, 0, s, jobs, wl, T); break;
    default: launch_k(k_unires<65>, grid, threads, 0, s, jobs, wl, T); break;
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

void launch_eval(int grid, int warps, cudaStream_t s, const Job* jobs, WorkList wl, Tables T) {
  const size_t smem = sizeof(uint32_t) * ((size_t)1024 * warps + 1024 + (size_t)warps * 33 * 32);
  launch_k(k_eval, grid, warps * 32, smem, s, jobs, wl, T);
}
void launch_eval_iw(int cls, int grid, cudaStream_t s, const Job* jobs, WorkList wl, Tables T, PfHint pf) {
  const int th = kEvalIwWarps * 32;
  switch (cls) {
    case -1: launch_k(k_eval_iw<0>, grid, th, 0, s, jobs, wl, T, pf); break;
    case 0: launch_k(k_eval_iw<1>, grid, th, 0, s, jobs, wl, T, pf); break;
    case 1: launch_k(k_eval_iw<2>, grid, th, 0, s, jobs, wl, T, pf); break;
    case 2: launch_k(k_eval_iw<4>, grid, th, 0, s, jobs, wl, T, pf); break;
    case 3: launch_k(k_eval_iw<8>, grid, th, 0, s, jobs, wl, T, pf); break;
    case 4: launch_k(k_eval_iw<16>, grid, th, 0, s, jobs, wl, T, pf); break;
    default: launch_k(k_eval_iw<32>, grid, th, 0, s, jobs, wl, T, pf); break;
  }
}

void launch_eval_w(int cls, int grid, int warps, cudaStream_t s, const Job* jobs, WorkList wl,
                   Tables T, PfHint pf) {
  const int th = warps * 32;
  switch (cls) {
    case -1: launch_k(k_eval_w<0>, grid, th, 0, s, jobs, wl, T, pf); break;
    case 0: launch_k(k_eval_w<1>, grid, th, 0, s, jobs, wl, T, pf); break;
    case 1: launch_k(k_eval_w<2>, grid, th, 0, s, jobs, wl, T, pf); break;
    case 2: launch_k(k_eval_w<4>, grid, th, 0, s, jobs, wl, T, pf); break;
    case 3: launch_k(k_eval_w<8>, grid, th, 0, s, jobs, wl, T, pf); break;
    case 4: launch_k(k_eval_w<16>, grid, th, 0, s, jobs, wl, T, pf); break;
    default: launch_k(k_eval_w<32>, grid, th, 0, s, jobs, wl, T, pf); break;
  }
}
void launch_intt_w(int grid, cudaStream_t s, const Job* jobs, WorkList wl, Tables T) {
  launch_k(k_intt_w, grid, kInttWarps * 32, 0, s, jobs, wl, T);
}
void launch_intt(int grid, size_t smem, cudaStream_t s, const Job* jobs, WorkList wl, Tables T) {
  launch_k(k_intt, grid, kEvalThreads, smem, s, jobs, wl, T);
}
void launch_crt(int grid, int threads, size_t smem, cudaStream_t s, const Job* jobs, WorkList wl,
                Tables T, int kmax, int lmax, int staged, int skip_big) {
  launch_k(k_crt, grid, threads, smem, s, jobs, wl, T, kmax, lmax, staged, skip_big);
}
void launch_plan_single(cudaStream_t s, const Job& J, Job* dst, int64_t* offs, Tables T, int eval_group) {
  k_plan_single<<<1, kPlanThreads, 0, s>>>(J, dst, offs, T, eval_group);
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
  rc |= set_dyn_smem_limit((const void*)k_crt_w<1>, optin);
  rc |= set_dyn_smem_limit((const void*)k_crt_w<2>, optin);
  rc |= set_dyn_smem_limit((const void*)k_crt_w<4>, optin);
  rc |= set_dyn_smem_limit((const void*)k_crt_w<8>, optin);
  return rc;
}

}  // namespace bs
