// Transforms of length N = 32 R held by one warp: lane l, register r holds element
// i = 32 r + l.  Butterflies whose partners are 32 or more apart stay in registers;
// the last five stages of the forward transform (first five of the inverse) pair lanes
// l and l ^ len through shuffles.
//
// Forward: decimation in frequency with omega of order N; position i ends up holding the
// value at omega^{bitreverse(i)} (times the coset scaling applied to the input).
// Inverse: decimation in time from that bit-reversed order; natural order out, times N.
#pragma once
#include "modarith.cuh"

namespace bs {

template <int R>
__device__ __forceinline__ void warp_dif(uint32_t (&v)[R], const uint32_t* tw, int logNT,
                                         const Mod M, uint32_t one_m) {
  constexpr int logR = (R >= 64) ? 6 : (R >= 32) ? 5 : (R >= 16) ? 4 : (R >= 8) ? 3 : (R >= 4) ? 2 : (R >= 2) ? 1 : 0;
  const int lane = threadIdx.x & 31;
  // in-register stages: len = 32 h, h = R/2 .. 1
#pragma unroll
  for (int lh = logR - 1; lh >= 0; --lh) {
    const int h = 1 << lh;
    const int lg = lh + 5;                      // len = 2^lg
    const int sh = logNT - (lg + 1);            // twiddle stride shift
#pragma unroll
    for (int r = 0; r < R; ++r) {
      if (r & h) continue;
      const int m = r & (h - 1);                // j = 32 m + lane
      const uint32_t w = tw[(32 * m + lane) << sh];
      const uint32_t a = v[r], b = v[r + h];
      v[r] = madd(a, b, M.p);
      v[r + h] = mmul(msub(a, b, M.p), w, M);
    }
  }
  // shuffle stages: len = 16 .. 1 (kept rolled: one copy of the body keeps the code
  // small enough for the instruction cache)
#pragma unroll 1
  for (int lg = 4; lg >= 0; --lg) {
    const int len = 1 << lg;
    const bool upper = (lane & len) != 0;
    const int sh = logNT - (lg + 1);
    const uint32_t w = upper ? tw[(lane & (len - 1)) << sh] : one_m;
#pragma unroll
    for (int r = 0; r < R; ++r) {
      const uint32_t x = v[r];
      const uint32_t y = __shfl_xor_sync(0xffffffffu, x, len);
      const uint32_t t = upper ? msub(y, x, M.p) : madd(x, y, M.p);
      v[r] = mmul(t, w, M);
    }
  }
}

template <int R>
__device__ __forceinline__ void warp_dit(uint32_t (&v)[R], const uint32_t* itw, int logNT,
                                         const Mod M, uint32_t one_m) {
  constexpr int logR = (R >= 64) ? 6 : (R >= 32) ? 5 : (R >= 16) ? 4 : (R >= 8) ? 3 : (R >= 4) ? 2 : (R >= 2) ? 1 : 0;
  const int lane = threadIdx.x & 31;
#pragma unroll 1
  for (int lg = 0; lg <= 4; ++lg) {
    const int len = 1 << lg;
    const bool upper = (lane & len) != 0;
    const int sh = logNT - (lg + 1);
    const uint32_t w = itw[(lane & (len - 1)) << sh];
#pragma unroll
    for (int r = 0; r < R; ++r) {
      const uint32_t x = v[r];
      const uint32_t y = __shfl_xor_sync(0xffffffffu, x, len);
      // lower lane: x + y w ; upper lane: y - x w
      const uint32_t t = mmul(upper ? x : y, w, M);
      v[r] = upper ? msub(y, t, M.p) : madd(x, t, M.p);
    }
  }
#pragma unroll
  for (int lh = 0; lh < logR; ++lh) {
    const int h = 1 << lh;
    const int lg = lh + 5;
    const int sh = logNT - (lg + 1);
#pragma unroll
    for (int r = 0; r < R; ++r) {
      if (r & h) continue;
      const int m = r & (h - 1);
      const uint32_t w = itw[(32 * m + lane) << sh];
      const uint32_t a = v[r];
      const uint32_t b = mmul(v[r + h], w, M);
      v[r] = madd(a, b, M.p);
      v[r + h] = msub(a, b, M.p);
    }
  }
  (void)one_m;
}

}  // namespace bs

namespace bs {

// 1024-point transforms held by one warp with every stage in registers: the stages
// whose butterfly partners are >= 32 apart run on layout A (lane l, register r holds
// element 32 r + l); a transpose through shared memory (row stride 33, so both the
// row-wise writes and the column-wise reads are free of bank conflicts) switches to
// layout B (lane l, register r holds element 32 l + r) for the stages with partners < 32
// apart.  sw must hold 33 * 32 words private to the warp.
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

// forward (decimation in frequency), input and output in layout A
__device__ __forceinline__ void warp_dif_1024(uint32_t (&v)[32], uint32_t* sw, const uint32_t* tw,
                                              int logNT, const Mod M) {
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int lh = 4; lh >= 0; --lh) {  // len = 512 .. 32 (layout A, partner r + h)
    const int h = 1 << lh;
    const int sh = logNT - (lh + 6);
#pragma unroll
    for (int r = 0; r < 32; ++r) {
      if (r & h) continue;
      const uint32_t w = tw[(32 * (r & (h - 1)) + lane) << sh];
      const uint32_t a = v[r], b = v[r + h];
      v[r] = madd(a, b, M.p);
      v[r + h] = mmul(msub(a, b, M.p), w, M);
    }
  }
  warp_transpose_ab(v, sw);
#pragma unroll
  for (int lg = 4; lg >= 0; --lg) {  // len = 16 .. 1 (layout B, partner r + len)
    const int len = 1 << lg;
    const int sh = logNT - (lg + 1);
#pragma unroll
    for (int r = 0; r < 32; ++r) {
      if (r & len) continue;
      const uint32_t w = tw[(r & (len - 1)) << sh];
      const uint32_t a = v[r], b = v[r + len];
      v[r] = madd(a, b, M.p);
      v[r + len] = mmul(msub(a, b, M.p), w, M);
    }
  }
  warp_transpose_ba(v, sw);
}

// inverse (decimation in time), input and output in layout A
__device__ __forceinline__ void warp_dit_1024(uint32_t (&v)[32], uint32_t* sw, const uint32_t* itw,
                                              int logNT, const Mod M) {
  const int lane = threadIdx.x & 31;
  warp_transpose_ab(v, sw);
#pragma unroll
  for (int lg = 0; lg <= 4; ++lg) {  // len = 1 .. 16 (layout B)
    const int len = 1 << lg;
    const int sh = logNT - (lg + 1);
#pragma unroll
    for (int r = 0; r < 32; ++r) {
      if (r & len) continue;
      const uint32_t w = itw[(r & (len - 1)) << sh];
      const uint32_t a = v[r];
      const uint32_t b = mmul(v[r + len], w, M);
      v[r] = madd(a, b, M.p);
      v[r + len] = msub(a, b, M.p);
    }
  }
  warp_transpose_ba(v, sw);
#pragma unroll
  for (int lh = 0; lh <= 4; ++lh) {  // len = 32 .. 512 (layout A)
    const int h = 1 << lh;
    const int sh = logNT - (lh + 6);
#pragma unroll
    for (int r = 0; r < 32; ++r) {
      if (r & h) continue;
      const uint32_t w = itw[(32 * (r & (h - 1)) + lane) << sh];
      const uint32_t a = v[r];
      const uint32_t b = mmul(v[r + h], w, M);
      v[r] = madd(a, b, M.p);
      v[r + h] = msub(a, b, M.p);
    }
  }
}

}  // namespace bs
