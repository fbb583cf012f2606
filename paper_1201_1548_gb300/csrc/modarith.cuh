// Arithmetic in Z_p for 31-bit primes 2^30 < p < 2^31 (the table's first primes also have
// 3p < 2^32, below kSmallPrimeMax).
//
// Multiplication uses Montgomery's reduction (P. L. Montgomery, "Modular multiplication
// without trial division", Math. Comp. 44 (1985)) with R = 2^32, in the variant that
// subtracts m*p instead of adding it:  for t < p * 2^32 and m = (t mod 2^32) * p^-1
// mod 2^32, the low words of t and m*p agree, so (t - m*p) / 2^32 = hi(t) - hi(m*p),
// which lies in (-p, p) and needs one conditional correction.
//
// Values are kept in [0, p).  "Montgomery form" of x is x * 2^32 mod p.  Every correction
// is an unsigned minimum of a value and its shift by p (a wrapped difference exceeds
// 2^31 > p), which needs no predicate.
#pragma once
#include <stdint.h>

#ifdef __CUDACC__
#define BS_HD __host__ __device__ __forceinline__
#else
#define BS_HD inline
#endif

namespace bs {

// primes up to this bound have 3p < 2^32: a sum of three products of residues stays below
// p 2^32 and needs no fold before Montgomery's reduction
constexpr uint32_t kSmallPrimeMax = 1431655765u;  // floor((2^32 - 1) / 3)

struct Mod {
  uint32_t p;     // the prime
  uint32_t pinv;  // p^-1 mod 2^32
};

BS_HD uint32_t umulhi32(uint32_t a, uint32_t b) {
#ifdef __CUDA_ARCH__
  return __umulhi(a, b);
#else
  return (uint32_t)(((uint64_t)a * b) >> 32);
#endif
}

// t < p * 2^32  ->  t * 2^-32 mod p in [0, p)
BS_HD uint32_t redc(uint64_t t, uint32_t p, uint32_t pinv) {
  uint32_t tl = (uint32_t)t;
  uint32_t th = (uint32_t)(t >> 32);
  uint32_t m = tl * pinv;
  uint32_t h = umulhi32(m, p);
  uint32_t r = th - h;
  uint32_t r2 = r + p;  // th < h: r wrapped past 2^31 and r + p is the residue; else r < p
  return r2 < r ? r2 : r;
}

// t < 2^32 * 1.5p (e.g. a sum of three products of values < p): fold the high word
// once, then reduce.
BS_HD uint32_t redc_wide(uint64_t t, uint32_t p, uint32_t pinv) {
  uint32_t tl = (uint32_t)t;
  uint32_t th = (uint32_t)(t >> 32);
  uint32_t th2 = th - p;
  th = th2 < th ? th2 : th;  // th >= p ? th - p : th
  uint32_t m = tl * pinv;
  uint32_t h = umulhi32(m, p);
  uint32_t r = th - h;
  uint32_t r2 = r + p;
  return r2 < r ? r2 : r;
}

BS_HD uint32_t mmul(uint32_t a, uint32_t b, const Mod& M) {
  return redc((uint64_t)a * b, M.p, M.pinv);
}

BS_HD uint32_t madd(uint32_t a, uint32_t b, uint32_t p) {
  uint32_t s = a + b;  // < 2^32 since a, b < 2^31
  uint32_t s2 = s - p;
  return s2 < s ? s2 : s;
}

BS_HD uint32_t msub(uint32_t a, uint32_t b, uint32_t p) {
  uint32_t d = a - b;
  uint32_t d2 = d + p;  // a < b: d wrapped and d + p is the residue; else d < p < d + p
  return d2 < d ? d2 : d;
}

BS_HD uint32_t mneg(uint32_t a, uint32_t p) { return a ? p - a : 0; }

// a^e in Montgomery form (one_m = 2^32 mod p is the Montgomery form of 1)
BS_HD uint32_t mpow(uint32_t a, uint32_t e, uint32_t one_m, const Mod& M) {
  uint32_t r = one_m;
  while (e) {
    if (e & 1u) r = mmul(r, a, M);
    e >>= 1;
    if (e) a = mmul(a, a, M);
  }
  return r;
}

// x w mod p for x < p and a fixed w < p with ws = floor(w 2^32 / p) (Shoup's method): the
// quotient estimate umulhi(x, ws) is exact or one too small, so x w - q p lies in [0, 2p)
BS_HD uint32_t mmul_shoup(uint32_t x, uint32_t w, uint32_t ws, uint32_t p) {
  const uint32_t q = umulhi32(x, ws);
  const uint32_t r = x * w - q * p;
  const uint32_t r2 = r - p;
  return r2 < r ? r2 : r;
}

// inverse of a non-zero Montgomery-form value by Fermat's little theorem
BS_HD uint32_t minv(uint32_t a, uint32_t one_m, const Mod& M) {
  return mpow(a, M.p - 2, one_m, M);
}

// ------------------------------------------------------------------------------------
// host-side helpers (plain 64-bit arithmetic)
// ------------------------------------------------------------------------------------
inline uint32_t host_pinv(uint32_t p) {
  // Newton iteration for p^-1 mod 2^32 (p odd): x <- x * (2 - p x), doubling the
  // number of correct low bits each step, starting from x = p (correct to 3 bits).
  uint32_t x = p;
  for (int i = 0; i < 5; ++i) x *= 2u - p * x;
  return x;
}

inline uint32_t host_powmod(uint64_t a, uint64_t e, uint64_t p) {
  uint64_t r = 1 % p;
  a %= p;
  while (e) {
    if (e & 1) r = r * a % p;
    a = a * a % p;
    e >>= 1;
  }
  return (uint32_t)r;
}

inline uint32_t host_to_mont(uint64_t x, uint64_t p) { return (uint32_t)(((x % p) << 32) % p); }

}  // namespace bs
