// Warp-wide big integers and the content (gcd of the coefficients) of an integer
// polynomial, computed by one warp or by the warps of a block splitting the coefficients.
//
// A non-negative integer of up to 32 K limbs is spread over the lanes: lane l, slot s
// holds limb 32 s + l.  Comparisons, subtraction and shifts resolve carries across lanes
// with ballots.  The gcd of two full-size numbers takes Lehmer steps on their leading 31
// bits (Knuth's Algorithm L), with a binary (Stein) step when a round makes no progress;
// once the running gcd fits in 64 bits every further coefficient is reduced modulo it by
// the whole warp and the gcd finishes in 64-bit arithmetic.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "ballot.cuh"

namespace bs {

template <int K>
struct WBig {
  uint32_t v[K];
};

template <int K>
__device__ __forceinline__ bool wb_is_zero(const WBig<K>& a) {
  bool nz = false;
#pragma unroll
  for (int s = 0; s < K; ++s) nz = nz || (a.v[s] != 0);
  return !__any_sync(0xffffffffu, nz);
}

// index of the highest nonzero limb (-1 for zero)
template <int K>
__device__ __forceinline__ int wb_top(const WBig<K>& a) {
  int top = -1;
#pragma unroll
  for (int s = 0; s < K; ++s) {
    const unsigned m = __ballot_sync(0xffffffffu, a.v[s] != 0);
    if (m) top = 32 * s + 31 - __clz((int)m);
  }
  return top;
}

// a > b ?
template <int K>
__device__ __forceinline__ bool wb_gt(const WBig<K>& a, const WBig<K>& b) {
  int hi = -1;
#pragma unroll
  for (int s = 0; s < K; ++s) {
    const unsigned m = __ballot_sync(0xffffffffu, a.v[s] != b.v[s]);
    if (m) hi = 32 * s + 31 - __clz((int)m);
  }
  if (hi < 0) return false;
  uint32_t av = 0, bv = 0;
#pragma unroll
  for (int s = 0; s < K; ++s) {
    const uint32_t x = __shfl_sync(0xffffffffu, a.v[s], hi & 31);
    const uint32_t y = __shfl_sync(0xffffffffu, b.v[s], hi & 31);
    if ((hi >> 5) == s) {
      av = x;
      bv = y;
    }
  }
  return av > bv;
}

// a -= b (a >= b).  Borrow into lane l: generate where x < y, propagate where x == y;
// the carry chain of G + (G | P) + borrow_in yields all borrows at once.
template <int K>
__device__ __forceinline__ void wb_sub(WBig<K>& a, const WBig<K>& b) {
  const int lane = threadIdx.x & 31;
  uint32_t bin = 0;
#pragma unroll
  for (int s = 0; s < K; ++s) {
    const uint32_t x = a.v[s], y = b.v[s];
    const uint32_t dd = x - y;
    const uint32_t G = __ballot_sync(0xffffffffu, x < y);
    const uint32_t Pm = __ballot_sync(0xffffffffu, dd == 0u) & ~G;
    const uint32_t X = G | Pm;
    const uint64_t Sx = (uint64_t)X + G + bin;
    const uint32_t C = (uint32_t)Sx ^ X ^ G;
    bin = (uint32_t)(Sx >> 32);
    a.v[s] = dd - ((C >> lane) & 1u);
  }
}

// number of trailing zero bits (a != 0)
template <int K>
__device__ __forceinline__ int wb_ctz(const WBig<K>& a) {
  int res = -1;
#pragma unroll
  for (int s = K - 1; s >= 0; --s) {
    const unsigned m = __ballot_sync(0xffffffffu, a.v[s] != 0);
    if (m) {
      const int ln = __ffs(m) - 1;
      const uint32_t x = __shfl_sync(0xffffffffu, a.v[s], ln);
      res = 32 * (32 * s + ln) + __ffs(x) - 1;
    }
  }
  return res;
}

// a >>= n
template <int K>
__device__ __forceinline__ void wb_shr(WBig<K>& a, int n) {
  const int lane = threadIdx.x & 31;
  while (n >= 32) {  // one limb down
#pragma unroll
    for (int s = 0; s < K; ++s) {
      const uint32_t x = __shfl_down_sync(0xffffffffu, a.v[s], 1);
      const uint32_t nxt = (s + 1 < K) ? __shfl_sync(0xffffffffu, a.v[s + 1 < K ? s + 1 : s], 0) : 0u;
      a.v[s] = (lane == 31) ? nxt : x;
    }
    n -= 32;
  }
  if (n > 0) {
#pragma unroll
    for (int s = 0; s < K; ++s) {
      uint32_t up = __shfl_down_sync(0xffffffffu, a.v[s], 1);
      const uint32_t nxt = (s + 1 < K) ? __shfl_sync(0xffffffffu, a.v[s + 1 < K ? s + 1 : s], 0) : 0u;
      if (lane == 31) up = nxt;
      a.v[s] = (a.v[s] >> n) | (up << (32 - n));
    }
  }
}

// a <<= n (the result must fit in 32 K limbs)
template <int K>
__device__ __forceinline__ void wb_shl(WBig<K>& a, int n) {
  const int lane = threadIdx.x & 31;
  while (n > 0) {
    const int step = n < 31 ? n : 31;
#pragma unroll
    for (int s = K - 1; s >= 0; --s) {
      uint32_t lo = __shfl_up_sync(0xffffffffu, a.v[s], 1);
      const uint32_t prv = (s > 0) ? __shfl_sync(0xffffffffu, a.v[s > 0 ? s - 1 : 0], 31) : 0u;
      if (lane == 0) lo = prv;
      a.v[s] = (a.v[s] << step) | (lo >> (32 - step));
    }
    n -= step;
  }
}

// |c| of a two's complement coefficient of L limbs (limbs beyond L are zero)
template <int K>
__device__ __forceinline__ void wb_load_abs(WBig<K>& a, const uint32_t* c, int L) {
  const int lane = threadIdx.x & 31;
  const bool neg = (c[L - 1] >> 31) != 0;
#pragma unroll
  for (int s = 0; s < K; ++s) {
    const int l = 32 * s + lane;
    a.v[s] = l < L ? (neg ? ~c[l] : c[l]) : 0u;
  }
  if (neg) {  // + 1, the carry resolved with a ballot of all-ones limbs
    uint32_t cin = 1;
#pragma unroll
    for (int s = 0; s < K; ++s) {
      const uint32_t x = a.v[s];
      const uint32_t Pm = __ballot_sync(0xffffffffu, x == 0xffffffffu);
      const uint64_t Sx = (uint64_t)Pm + cin;
      const uint32_t C = (uint32_t)Sx ^ Pm;
      cin = (uint32_t)(Sx >> 32);
      a.v[s] = x + ((C >> lane) & 1u);
    }
#pragma unroll
    for (int s = 0; s < K; ++s)
      if (32 * s + lane >= L) a.v[s] = 0u;
  }
}

__device__ __forceinline__ uint64_t gcd64(uint64_t a, uint64_t b) {
  while (b) {
    const uint64_t t = a % b;
    a = b;
    b = t;
  }
  return a;
}

__device__ __forceinline__ uint64_t mulmod64(uint64_t a, uint64_t b, uint64_t m) {
  return (uint64_t)(((unsigned __int128)a * b) % m);
}

__device__ __forceinline__ uint64_t addmod64(uint64_t a, uint64_t b, uint64_t m) {
  const uint64_t s = a + b;  // a, b < m < 2^64: the sum may wrap once
  return (s < a || s >= m) ? s - m : s;
}

// Residues used to reduce a warp-wide integer modulo m (2 <= m < 2^64): W = 2^(32 * 32) mod m
// steps between the slots of one lane, P = 2^(32 * lane) mod m places the lane.  For
// m < 2^63 the products by these fixed factors use Shoup's method (V. Shoup, NTL): with
// w' = floor(w 2^64 / m), a w mod m = a w - hi(a w') m, less m at most once, which needs
// no division; larger moduli fall back to 128-bit remainders.
struct Mod64Pow {
  uint64_t m = 0, W = 0, P = 0, Ws = 0, Ps = 0;
  bool shoup = false;
  __device__ void set(uint64_t mod) {
    m = mod;
    const uint64_t t32 = ((uint64_t)1 << 32) % m;  // 2^32 mod m
    uint64_t w = t32;
#pragma unroll 1
    for (int i = 0; i < 5; ++i) w = mulmod64(w, w, m);  // (2^32)^32
    W = w;
    uint64_t pl = 1 % m, b = t32;
    for (int e = threadIdx.x & 31; e; e >>= 1) {  // (2^32)^lane
      if (e & 1) pl = mulmod64(pl, b, m);
      b = mulmod64(b, b, m);
    }
    P = pl;
    shoup = m < ((uint64_t)1 << 63);
    if (shoup) {
      Ws = (uint64_t)(((unsigned __int128)W << 64) / m);
      Ps = (uint64_t)(((unsigned __int128)P << 64) / m);
    }
  }
  // a w mod m for the fixed factor w (ws its Shoup companion)
  __device__ __forceinline__ uint64_t mul(uint64_t a, uint64_t w, uint64_t ws) const {
    if (!shoup) return mulmod64(a % m, w, m);
    const uint64_t q = __umul64hi(a, ws);
    const uint64_t r = a * w - q * m;  // in [0, 2m) < 2^64
    return r >= m ? r - m : r;
  }
};

template <int K>
__device__ __forceinline__ uint64_t wb_mod64(const WBig<K>& a, const Mod64Pow& mp) {
  const bool wide = mp.m > 0xffffffffull;  // every limb is already below m
  uint64_t acc = 0;
#pragma unroll
  for (int s = K - 1; s >= 0; --s) {
    const uint64_t limb = wide ? a.v[s] : (uint64_t)(a.v[s] % (uint32_t)mp.m);
    acc = addmod64(mp.mul(acc, mp.W, mp.Ws), limb, mp.m);
  }
  acc = mp.mul(acc, mp.P, mp.Ps);
#pragma unroll
  for (int o = 16; o; o >>= 1) acc = addmod64(acc, __shfl_xor_sync(0xffffffffu, acc, o), mp.m);
  return acc;
}

// limb l of a (0 beyond the number's 32 K limbs), on every lane
template <int K>
__device__ __forceinline__ uint32_t wb_limb(const WBig<K>& a, int l) {
  uint32_t x = 0;
#pragma unroll
  for (int s = 0; s < K; ++s) {
    const uint32_t y = __shfl_sync(0xffffffffu, a.v[s], l & 31);
    if ((l >> 5) == s) x = y;
  }
  return x;
}

// bit length (0 for zero)
template <int K>
__device__ __forceinline__ int wb_bits(const WBig<K>& a) {
  const int top = wb_top<K>(a);
  if (top < 0) return 0;
  return 32 * top + 32 - __clz((int)wb_limb<K>(a, top));
}

// 31 bits of a starting at bit s >= 0
template <int K>
__device__ __forceinline__ uint32_t wb_bits31(const WBig<K>& a, int s) {
  const int l = s >> 5, r = s & 31;
  const uint32_t lo = wb_limb<K>(a, l), hi = wb_limb<K>(a, l + 1);
  const uint32_t w = r ? (lo >> r) | (hi << (32 - r)) : lo;
  return w & 0x7fffffffu;
}

// x * s for a 32-bit s; the product must fit in 32 K limbs
template <int K>
__device__ __forceinline__ void wb_mul_small(const WBig<K>& x, uint32_t s, WBig<K>& out) {
  const int lane = threadIdx.x & 31;
  uint32_t cin = 0, hprev = 0;  // carry into the chunk; high word of the limb below the chunk
#pragma unroll
  for (int t = 0; t < K; ++t) {
    const uint64_t p = (uint64_t)x.v[t] * s;
    const uint32_t lo = (uint32_t)p, hi = (uint32_t)(p >> 32);
    uint32_t hin = __shfl_up_sync(0xffffffffu, hi, 1);
    const uint32_t h31 = __shfl_sync(0xffffffffu, hi, 31);
    if (lane == 0) hin = hprev;
    hprev = h31;
    out.v[t] = ballot_add(lo, hin, cin, lane);
  }
}

template <int K>
__device__ __forceinline__ void wb_strip2(WBig<K>& a) {
  if (!wb_is_zero<K>(a)) wb_shr<K>(a, wb_ctz<K>(a));
}

// gcd of odd u and v (in place in u).  Lehmer's method on the leading 31 bits (Knuth,
// TAOCP vol. 2, Algorithm 4.5.2L): single-precision Euclid steps on the leading words
// give a cofactor matrix whose quotients are the true ones while both tests agree; it is
// applied to the full numbers as |A| u - |B| v or |B| v - |A| u (the cofactors of a row
// have opposite signs or one of them is zero; the sign of the second decides).  Factors of two are stripped after every step (the gcd is odd).  A round that
// makes no progress takes one binary step (Stein) instead; once v fits in 64 bits the gcd
// finishes in 64-bit arithmetic.
template <int K>
__device__ void wb_gcd_odd(WBig<K>& u, WBig<K>& v) {
  const int lane = threadIdx.x & 31;
  for (int it = 0; it < (1 << 22); ++it) {  // every round removes at least one bit
    if (wb_gt<K>(v, u)) {
      const WBig<K> t = u;
      u = v;
      v = t;
    }
    if (wb_is_zero<K>(v)) return;
    const int nu = wb_bits<K>(u), nv = wb_bits<K>(v);
    if (nv <= 64) {  // u mod v and the rest in 64-bit arithmetic
      const uint64_t m = (uint64_t)wb_limb<K>(v, 0) | ((uint64_t)wb_limb<K>(v, 1) << 32);
      uint64_t g = 1;
      if (m > 1) {
        Mod64Pow mp;
        mp.set(m);
        g = gcd64(m, wb_mod64<K>(u, mp));
      }
#pragma unroll
      for (int s = 0; s < K; ++s) u.v[s] = (s == 0 && lane == 0) ? (uint32_t)g : (s == 0 && lane == 1) ? (uint32_t)(g >> 32) : 0u;
      return;
    }
    bool stepped = false;
    if (nu - nv < 31 && nu + 31 <= 32 * 32 * K) {
      const int sh = nu - 31;
      int64_t x = wb_bits31<K>(u, sh), y = wb_bits31<K>(v, sh);
      int64_t A = 1, B = 0, C = 0, D = 1;
      for (int k = 0; k < 64; ++k) {
        if (y + C == 0 || y + D == 0) break;
        const int64_t q = (x + A) / (y + C), q2 = (x + B) / (y + D);
        if (q != q2) break;
        int64_t t = A - q * C;
        A = C;
        C = t;
        t = B - q * D;
        B = D;
        D = t;
        t = x - q * y;
        x = y;
        y = t;
      }
      if (B != 0) {
        WBig<K> X, Y, nu2, nv2;
        wb_mul_small<K>(u, (uint32_t)(A < 0 ? -A : A), X);
        wb_mul_small<K>(v, (uint32_t)(B < 0 ? -B : B), Y);
        if (B <= 0) {  // A >= 0 >= B (A may be 0 only with B > 0)
          nu2 = X;
          wb_sub<K>(nu2, Y);
        } else {
          nu2 = Y;
          wb_sub<K>(nu2, X);
        }
        wb_mul_small<K>(u, (uint32_t)(C < 0 ? -C : C), X);
        wb_mul_small<K>(v, (uint32_t)(D < 0 ? -D : D), Y);
        if (D <= 0) {
          nv2 = X;
          wb_sub<K>(nv2, Y);
        } else {
          nv2 = Y;
          wb_sub<K>(nv2, X);
        }
        u = nu2;
        v = nv2;
        wb_strip2<K>(u);
        wb_strip2<K>(v);
        if (wb_is_zero<K>(v)) return;  // u is the gcd
        if (wb_is_zero<K>(u)) {
          u = v;
          return;
        }
        stepped = true;
      }
    }
    if (!stepped) {  // binary step: u - v is even and nonzero (u > v, both odd)
      wb_sub<K>(u, v);
      wb_strip2<K>(u);
    }
  }
}

// Running gcd of integers, held by one warp.  g = 0 stands for "no coefficient yet".
// Once the gcd fits in 64 bits every further coefficient is reduced modulo it by the
// whole warp (Horner's rule per lane over its limbs, then a shuffle sum of the lanes'
// shares) and the gcd continues in 64-bit arithmetic; until then Stein's binary
// algorithm runs on the warp-wide integers.
template <int K>
struct ContentAcc {
  WBig<K> g;
  bool small = false;  // g fits in 64 bits and lives in g64
  uint64_t g64 = 0;
  Mod64Pow mp;
  bool started = false;

  __device__ __forceinline__ bool is_one() const { return small && g64 == 1u; }

  // fold the n coefficients c[i * step * L .. i * step * L + L - 1] into the gcd
  __device__ void fold(const uint32_t* c, int n, int L, int step = 1) {
    const int64_t stride = (int64_t)step * L;
    int i = 0;
    for (; i < n && !small; ++i) {  // warp-wide gcds until the gcd fits in 64 bits
      WBig<K> b;
      wb_load_abs<K>(b, c + i * stride, L);
      if (wb_is_zero<K>(b)) continue;
      if (!started) {
        g = b;
        started = true;
      } else {
        // gcd of the odd parts, times the common power of two
        const int tg = wb_ctz<K>(g), tb = wb_ctz<K>(b);
        const int sh = tg < tb ? tg : tb;
        wb_shr<K>(g, tg);
        wb_shr<K>(b, tb);
        wb_gcd_odd<K>(g, b);
        wb_shl<K>(g, sh);
      }
      if (wb_top<K>(g) <= 1) {
        small = true;
        const uint64_t lo = __shfl_sync(0xffffffffu, g.v[0], 0);
        const uint64_t hi = __shfl_sync(0xffffffffu, g.v[0], 1);
        g64 = lo | (hi << 32);
        if (g64 > 1) mp.set(g64);
      }
    }
    // four coefficients at a time, their loads and reductions in flight together; a
    // residue modulo the gcd before an update still gives the right gcd after it (the new
    // gcd divides the old one)
    constexpr int B4 = K <= 4 ? 4 : 2;
    for (; i < n; i += B4) {
      if (g64 == 1u) return;
      WBig<K> b[B4];
#pragma unroll
      for (int j = 0; j < B4; ++j)
        if (i + j < n) wb_load_abs<K>(b[j], c + (i + j) * stride, L);
      uint64_t r[B4];
#pragma unroll
      for (int j = 0; j < B4; ++j) r[j] = (i + j < n) ? wb_mod64<K>(b[j], mp) : 0u;
      const uint64_t g0 = g64;
#pragma unroll
      for (int j = 0; j < B4; ++j)
        if (r[j]) g64 = gcd64(g64, r[j]);
      if (g64 != g0 && g64 > 1) mp.set(g64);
    }
  }

  // store the gcd (0 if every coefficient was zero) as Lout magnitude limbs
  __device__ void store(uint32_t* out, int Lout) const {
    const int lane = threadIdx.x & 31;
    if (small) {
      for (int l = lane; l < Lout; l += 32) out[l] = (l == 0) ? (uint32_t)g64 : (l == 1) ? (uint32_t)(g64 >> 32) : 0u;
      return;
    }
#pragma unroll
    for (int s = 0; s < K; ++s) {
      const int l = 32 * s + lane;
      if (l < Lout) out[l] = started ? g.v[s] : 0u;
    }
    for (int l = 32 * K + lane; l < Lout; l += 32) out[l] = 0u;
  }
};

// The gcd of the n1 coefficients at c1 (L1 limbs each, two's complement) and the n2 at c2
// (L2 limbs; n2 = 0 for none) by all warps of the block: warp w folds the coefficients
// w, w + W, w + 2W, ... of each sequence (W warps), so the first gcd of two full-size
// coefficients runs in every warp at once and the long tail of reductions modulo the (by
// then 64-bit) gcd runs W warps wide.  The W partial gcds meet in shared memory (part:
// W * Lp words, Lp >= max(L1, L2) so that a partial gcd, at most one coefficient's
// magnitude, fits) and warp 0 folds them into out (Lout magnitude limbs, which must hold
// the final gcd; 0 when every coefficient is zero).  Every thread of the block calls it;
// it starts and ends with a barrier and returns, in every thread, whether the gcd is 1.
template <int K>
__device__ __noinline__ bool block_content(const uint32_t* c1, int n1, int L1, const uint32_t* c2, int n2, int L2,
                                           uint32_t* part, int Lp, uint32_t* out, int Lout) {
  __shared__ int s_one;
  const int W = blockDim.x >> 5, w = threadIdx.x >> 5;
  __syncthreads();  // part and s_one may still be read by an earlier call
  {
    ContentAcc<K> h;
    const int m1 = n1 > w ? (n1 - w + W - 1) / W : 0;
    h.fold(c1 + (int64_t)w * L1, m1, L1, W);
    const int m2 = n2 > w ? (n2 - w + W - 1) / W : 0;
    if (m2 > 0 && !h.is_one()) h.fold(c2 + (int64_t)w * L2, m2, L2, W);
    h.store(part + (int64_t)w * Lp, Lp);
  }
  __syncthreads();
  if (w == 0) {
    ContentAcc<K> t;
    t.fold(part, W, Lp);
    t.store(out, Lout);
    if (threadIdx.x == 0) s_one = t.is_one() ? 1 : 0;
  }
  __syncthreads();
  return s_one != 0;
}

}  // namespace bs
