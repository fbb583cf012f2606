// Forward transforms of length N = 32 R held by one warp (step (b) of the modular
// algorithm, Sec. 5.1: evaluation at the N points of a coset of the order-N subgroup).
//
// Layout A: lane l, register r holds element i = 32 r + l.  Butterflies whose partners
// are 32 or more apart stay in registers; the stages with partners closer than 32 pair
// lanes through shuffles (R < 32) or run in registers after a transpose through shared
// memory (R = 32, layout B: lane l, register r holds element 32 l + r).
//
// Decimation in frequency with omega of order N: position i ends up holding the value at
// omega^{bitreverse(i)} (times the coset scaling applied to the input).
//
// Twiddles come from a packed table P with P[len + j] = omega_{2 len}^j for the stage
// whose butterfly partners are len apart (len = 1, 2, ..., N/2; P[0] unused), so every
// stage reads consecutive entries: lanes never collide on a shared-memory bank.  The
// table does not depend on N, only on the prime.
//
// MASK marks the registers that may be nonzero on input (bit r for register r).  The
// butterflies of the register stages are specialised at compile time: a pair with both
// inputs zero is skipped, a pair with one zero input costs one multiplication.  Rows
// with few coefficients (a polynomial of degree < 32 k evaluated at N points) thus skip
// most of the first stages.
#pragma once
#include "modarith.cuh"

namespace bs {

// mask after a register stage with partner distance h: each pair with a nonzero input
// has two nonzero outputs
__host__ __device__ constexpr uint32_t stage_mask(uint32_t mask, int h) {
  uint32_t out = mask;
  for (int r = 0; r < 32; ++r)
    if (!(r & h) && (((mask >> r) & 1u) || ((mask >> (r + h)) & 1u))) out |= (1u << r) | (1u << (r + h));
  return out;
}

// register stages with partner distance h = 2^LH, 2^(LH-1), ..., 1 (in register
// indices), twiddles P[LEN0 h + LEN0 (r mod h) + LANEMUL lane]: layout A uses LEN0 = 32,
// LANEMUL = 1 (element distance 32 h); layout B uses LEN0 = 1, LANEMUL = 0.
template <int R, int LH, uint32_t MASK, int LEN0, int LANEMUL>
struct RegStages {
  static __device__ __forceinline__ void run(uint32_t (&v)[R], const uint32_t* P, int lane,
                                             const Mod& M) {
    constexpr int h = 1 << LH;
#pragma unroll
    for (int r = 0; r < R; ++r) {
      if (r & h) continue;
      const bool az = !((MASK >> r) & 1u);
      const bool bz = !((MASK >> (r + h)) & 1u);
      if (az && bz) continue;
      const uint32_t w = P[LEN0 * h + LEN0 * (r & (h - 1)) + LANEMUL * lane];
      if (bz) {  // (a, 0) -> (a, a w)
        v[r + h] = mmul(v[r], w, M);
      } else if (az) {  // (0, b) -> (b, -b w)
        const uint32_t b = v[r + h];
        v[r] = b;
        v[r + h] = mmul(mneg(b, M.p), w, M);
      } else {
        const uint32_t a = v[r], b = v[r + h];
        v[r] = madd(a, b, M.p);
        v[r + h] = mmul(msub(a, b, M.p), w, M);
      }
    }
    RegStages<R, LH - 1, stage_mask(MASK, h), LEN0, LANEMUL>::run(v, P, lane, M);
  }
};

template <int R, uint32_t MASK, int LEN0, int LANEMUL>
struct RegStages<R, -1, MASK, LEN0, LANEMUL> {
  static __device__ __forceinline__ void run(uint32_t (&)[R], const uint32_t*, int, const Mod&) {}
};

// layout B register stages h = 2^LH .. 1 on full registers with Shoup's products: the
// twiddle of a pair is the same in every lane, S[2 j] = omega_{2h}^(r mod h) in standard
// form (j = h + r mod h) and S[2 j + 1] = floor(S[2 j] 2^32 / p); the results are the same
// residues as with the Montgomery-form twiddles of P
template <int R, int LH>
struct RegStagesS {
  static __device__ __forceinline__ void run(uint32_t (&v)[R], const uint32_t* S, const Mod& M) {
    constexpr int h = 1 << LH;
#pragma unroll
    for (int r = 0; r < R; ++r) {
      if (r & h) continue;
      const int j = h + (r & (h - 1));
      const uint32_t w = __ldg(S + 2 * j), ws = __ldg(S + 2 * j + 1);
      const uint32_t a = v[r], b = v[r + h];
      v[r] = madd(a, b, M.p);
      v[r + h] = mmul_shoup(msub(a, b, M.p), w, ws, M.p);
    }
    RegStagesS<R, LH - 1>::run(v, S, M);
  }
};

template <int R>
struct RegStagesS<R, -1> {
  static __device__ __forceinline__ void run(uint32_t (&)[R], const uint32_t*, const Mod&) {}
};

template <int R>
struct Log2R {
  static constexpr int v = (R >= 32) ? 5 : (R >= 16) ? 4 : (R >= 8) ? 3 : (R >= 4) ? 2 : (R >= 2) ? 1 : 0;
};

// N = 32 R, 2 <= R <= 16 (R = 1 with N = 32 as well): register stages, then five
// shuffle stages (len = 16 .. 1)
// (the shuffle stages multiply by Shoup's method with the prime's pairs S, the pair of 1
// for the lanes that only add)
template <int R, uint32_t MASK>
__device__ __forceinline__ void warp_dif_pk(uint32_t (&v)[R], const uint32_t* P, const uint32_t* S,
                                            const Mod M) {
  const int lane = threadIdx.x & 31;
  RegStages<R, Log2R<R>::v - 1, MASK, 32, 1>::run(v, P, lane, M);
#pragma unroll 1
  for (int lg = 4; lg >= 0; --lg) {
    const int len = 1 << lg;
    const bool upper = (lane & len) != 0;
    const uint2 ww = __ldg(reinterpret_cast<const uint2*>(S) + (upper ? len + (lane & (len - 1)) : 0));
#pragma unroll
    for (int r = 0; r < R; ++r) {
      const uint32_t x = v[r];
      const uint32_t y = __shfl_xor_sync(0xffffffffu, x, len);
      const uint32_t t = upper ? msub(y, x, M.p) : madd(x, y, M.p);
      v[r] = mmul_shoup(t, ww.x, ww.y, M.p);
    }
  }
}

// N < 32: one register per lane, lanes >= N hold zeros; stages len = N/2 .. 1
__device__ __forceinline__ void warp_dif_short(uint32_t& v, int N, const uint32_t* S, const Mod M) {
  const int lane = threadIdx.x & 31;
  for (int len = N >> 1; len >= 1; len >>= 1) {
    const bool upper = (lane & len) != 0;
    const uint2 ww = __ldg(reinterpret_cast<const uint2*>(S) + (upper ? len + (lane & (len - 1)) : 0));
    const uint32_t x = v;
    const uint32_t y = __shfl_xor_sync(0xffffffffu, x, len);
    v = mmul_shoup(upper ? msub(y, x, M.p) : madd(x, y, M.p), ww.x, ww.y, M.p);
  }
}

// layout A <-> B through shared memory (row stride 33: row writes and column reads are
// free of bank conflicts); sw holds 33 * 32 words private to the warp
__device__ __forceinline__ void warp_transpose_ab(uint32_t (&v)[32], uint32_t* sw) {
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int r = 0; r < 32; ++r) sw[33 * r + lane] = v[r];
  __syncwarp();
#pragma unroll
  for (int r = 0; r < 32; ++r) v[r] = sw[33 * lane + r];
  __syncwarp();
}

__device__ __forceinline__ void warp_transpose_ba(uint32_t (&v)[32], uint32_t* sw) {
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int r = 0; r < 32; ++r) sw[33 * lane + r] = v[r];
  __syncwarp();
#pragma unroll
  for (int r = 0; r < 32; ++r) v[r] = sw[33 * r + lane];
  __syncwarp();
}

// N = 1024: five register stages in layout A (len = 512 .. 32), transpose, five register
// stages in layout B (len = 16 .. 1, Shoup's products with the prime's pairs S), transpose
// back
template <uint32_t MASK>
__device__ __forceinline__ void warp_dif_1024_pk(uint32_t (&v)[32], uint32_t* sw, const uint32_t* P,
                                                 const uint32_t* S, const Mod M) {
  const int lane = threadIdx.x & 31;
  RegStages<32, 4, MASK, 32, 1>::run(v, P, lane, M);
  warp_transpose_ab(v, sw);
  RegStagesS<32, 4>::run(v, S, M);
  warp_transpose_ba(v, sw);
}

}  // namespace bs

namespace bs {

// ---- inverse transforms (decimation in time), bit-reversed order in, natural order out
// (times N); Pi[len + j] = omega_{2 len}^-j.  A butterfly maps (a, b) to (a + b w, a - b w).

// register stages with partner distance h = 1, 2, ..., 2^LH (in register indices)
template <int R, int LH, int LEN0, int LANEMUL>
__device__ __forceinline__ void reg_stages_dit(uint32_t (&v)[R], const uint32_t* Pi, int lane,
                                               const Mod& M) {
#pragma unroll
  for (int lh = 0; lh <= LH; ++lh) {
    const int h = 1 << lh;
#pragma unroll
    for (int r = 0; r < R; ++r) {
      if (r & h) continue;
      const uint32_t w = Pi[LEN0 * h + LEN0 * (r & (h - 1)) + LANEMUL * lane];
      const uint32_t a = v[r];
      const uint32_t b = mmul(v[r + h], w, M);
      v[r] = madd(a, b, M.p);
      v[r + h] = msub(a, b, M.p);
    }
  }
}

// N = 32 R, R <= 16 (R = 1 also covers N < 32): shuffle stages len = 1 .. min(16, N/2)
// within each register (elements 32 r .. 32 r + 31), then the register stages
template <int R>
__device__ __forceinline__ void warp_dit_pk(uint32_t (&v)[R], int N, const uint32_t* Pi, const Mod M) {
  const int lane = threadIdx.x & 31;
  const int nmax = (N < 32 ? N : 32) >> 1;
#pragma unroll 1
  for (int len = 1; len <= nmax; len <<= 1) {
    const bool upper = (lane & len) != 0;
    const uint32_t w = Pi[len + (lane & (len - 1))];
#pragma unroll
    for (int r = 0; r < R; ++r) {
      const uint32_t x = v[r];
      const uint32_t y = __shfl_xor_sync(0xffffffffu, x, len);
      const uint32_t t = mmul(upper ? x : y, w, M);
      v[r] = upper ? msub(y, t, M.p) : madd(x, t, M.p);
    }
  }
  reg_stages_dit<R, Log2R<R>::v - 1, 32, 1>(v, Pi, lane, M);
}

// N = 1024: layout A in, transpose to B, stages len = 1 .. 16 in registers, transpose
// back, stages len = 32 .. 512 in registers
__device__ __forceinline__ void warp_dit_1024_pk(uint32_t (&v)[32], uint32_t* sw, const uint32_t* Pi,
                                                 const Mod M) {
  const int lane = threadIdx.x & 31;
  warp_transpose_ab(v, sw);
  reg_stages_dit<32, 4, 1, 0>(v, Pi, lane, M);
  warp_transpose_ba(v, sw);
  reg_stages_dit<32, 4, 32, 1>(v, Pi, lane, M);
}

}  // namespace bs
