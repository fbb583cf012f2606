// Warp-wide big integers and the content (gcd of the coefficients) of an integer
// polynomial, computed by one warp.
//
// A non-negative integer of up to 32 K limbs is spread over the lanes: lane l, slot s
// holds limb 32 s + l.  Comparisons, subtraction and shifts resolve carries across lanes
// with ballots.  The gcd is Stein's binary algorithm; once the running gcd fits in 64
// bits every further coefficient is reduced modulo it by the whole warp and the gcd
// finishes in 64-bit arithmetic.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

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
// steps between the slots of one lane, P = 2^(32 * lane) mod m places the lane.
struct Mod64Pow {
  uint64_t m = 0, W = 0, P = 0;
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
  }
};

// a mod m for a warp-wide non-negative integer (every lane receives the result)
template <int K>
__device__ __forceinline__ uint64_t wb_mod64(const WBig<K>& a, const Mod64Pow& mp) {
  uint64_t acc = 0;
#pragma unroll
  for (int s = K - 1; s >= 0; --s) acc = addmod64(mulmod64(acc, mp.W, mp.m), a.v[s] % mp.m, mp.m);
  acc = mulmod64(acc, mp.P, mp.m);
#pragma unroll
  for (int o = 16; o; o >>= 1) acc = addmod64(acc, __shfl_xor_sync(0xffffffffu, acc, o), mp.m);
  return acc;
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

  // fold the n coefficients c[i * L .. i * L + L - 1] into the gcd
  __device__ void fold(const uint32_t* c, int n, int L) {
    for (int i = 0; i < n; ++i) {
      const uint32_t* ci = c + (int64_t)i * L;
      if (small && g64 == 1u) return;
      WBig<K> b;
      wb_load_abs<K>(b, ci, L);
      if (wb_is_zero<K>(b)) continue;
      if (small) {
        const uint64_t r = wb_mod64<K>(b, mp);
        const uint64_t ng = gcd64(g64, r);
        if (ng != g64) {
          g64 = ng;
          if (g64 > 1) mp.set(g64);
        }
        continue;
      }
      if (!started) {
        g = b;
        started = true;
      } else {
        // Stein's binary gcd of g and b
        const int tg = wb_ctz<K>(g), tb = wb_ctz<K>(b);
        const int sh = tg < tb ? tg : tb;
        wb_shr<K>(g, tg);
        for (int it = 0; it < (1 << 20); ++it) {  // each pass removes at least one bit
          wb_shr<K>(b, wb_ctz<K>(b));
          if (wb_gt<K>(g, b)) {
            const WBig<K> t = g;
            g = b;
            b = t;
          }
          wb_sub<K>(b, g);
          if (wb_is_zero<K>(b)) break;
        }
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

}  // namespace bs
