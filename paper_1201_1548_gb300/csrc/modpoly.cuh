// Polynomials in Z[x] and Z_p[x] for the modular gcd kernels: reduction of a limb
// coefficient modulo a table prime, Euclid and exact division in shared memory, and the
// host-side helpers shared by the gcd, square-free part and square-free factorisation
// pipelines (Sec. 5.1, "Computing gcds in Z[x]").
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <cstring>

#include "ctx.cuh"
#include "plan.cuh"

namespace bs {

// ---- device ----------------------------------------------------------------------------
// Montgomery form of a two's complement coefficient of L limbs modulo the table prime.  The
// table of 2^(32 l) covers coefficients of up to kMaxLimbs limbs; wider ones (a resultant
// fed back as input) are reduced by Horner's rule on 64-bit remainders.
__device__ __forceinline__ uint32_t reduce_coef(const uint32_t* c, int L, const uint32_t* pw,
                                                const uint32_t* mpw, const PrimeConst& pc) {
  if (L <= kMaxLimbs) {
    uint32_t acc = 0;
    for (int l = 0; l < L; ++l) acc = madd(acc, redc((uint64_t)c[l] * pw[l], pc.p, pc.pinv), pc.p);
    if (c[L - 1] >> 31) acc = msub(acc, mpw[L], pc.p);
    return acc;
  }
  uint64_t r = 0;  // the raw L-limb value mod p
  for (int l = L - 1; l >= 0; --l) r = ((r << 32) | c[l]) % pc.p;
  if (c[L - 1] >> 31) {  // value = raw - 2^(32 L)
    uint64_t t = 1;
    for (int l = 0; l < L; ++l) t = (t << 32) % pc.p;
    r = (r + pc.p - t) % pc.p;
  }
  return redc(r * pc.r2, pc.p, pc.pinv);
}

// division-free Euclid on X (degree la) and Y (degree lb) in shared memory; returns the
// pointer holding the gcd and its degree in *dgo (the gcd is not normalised)
static __device__ uint32_t* smem_euclid(uint32_t* X, int la, uint32_t* Y, int lb, const Mod M, int* dgo,
                                 int* s_top) {
  while (true) {
    if (la < lb) {
      uint32_t* t = X;
      X = Y;
      Y = t;
      const int u = la;
      la = lb;
      lb = u;
    }
    if (lb < 0) break;
    const int sh = la - lb;
    const uint32_t a0 = X[la], b0 = Y[lb];
    const uint32_t na0 = mneg(a0, M.p);
    for (int i = threadIdx.x; i < la; i += blockDim.x) {
      const uint32_t bi = (i >= sh) ? Y[i - sh] : 0u;
      X[i] = redc((uint64_t)b0 * X[i] + (uint64_t)na0 * bi, M.p, M.pinv);
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      int l = la - 1;
      while (l >= 0 && X[l] == 0) --l;
      *s_top = l;
    }
    __syncthreads();
    la = *s_top;
    __syncthreads();
  }
  *dgo = la;
  return X;
}

// exact division in shared memory, in place: X (degree nx) by the monic G (degree e <=
// nx).  Afterwards X[e..nx] holds the quotient (degree nx - e) and X[0..e-1] the remainder.
// Y (degree ny, ny < e for none) is divided by the same G in the same passes.
static __device__ void smem_div2(uint32_t* X, int nx, uint32_t* Y, int ny, const uint32_t* G, int e,
                                 const Mod M) {
  const int tx = nx - e, ty = ny - e;
  for (int t = (tx > ty ? tx : ty); t >= 0; --t) {
    const uint32_t qx = (t <= tx) ? X[t + e] : 0u;
    const uint32_t qy = (t <= ty) ? Y[t + e] : 0u;
    for (int i = threadIdx.x; i < e; i += blockDim.x) {
      const uint32_t gi = G[i];
      if (t <= tx) X[t + i] = msub(X[t + i], mmul(qx, gi, M), M.p);
      if (t <= ty) Y[t + i] = msub(Y[t + i], mmul(qy, gi, M), M.p);
    }
    __syncthreads();
  }
}

// |c| mod p for a magnitude of L limbs
__device__ __forceinline__ uint32_t mag_mod(const uint32_t* c, int L, uint32_t p) {
  uint64_t acc = 0;
  for (int l = L - 1; l >= 0; --l) acc = ((acc << 32) | c[l]) % p;
  return (uint32_t)acc;
}

// ---- host ------------------------------------------------------------------------------
static inline bool limbs_zero(const uint32_t* c, int L) {
  for (int l = 0; l < L; ++l)
    if (c[l]) return false;
  return true;
}

static inline int trimmed_degree(const bs_upoly& u) {
  int d = u.deg;
  while (d >= 0 && limbs_zero(u.c + (size_t)d * u.limbs, u.limbs)) --d;
  return d;
}

// log2 ||u||_2 (Q16, rounded up) over the first d + 1 coefficients
static inline int64_t log2_norm2_q16(const bs_upoly& u, int d) {
  UF s2{0u, 0};
  for (int i = 0; i <= d; ++i) {
    bool nz;
    int bits;
    const UF m = mag_uf(u.c + (size_t)i * u.limbs, u.limbs, &nz, &bits);
    if (nz) s2 = uf_add(s2, uf_mul(m, m));
  }
  return s2.m ? (uf_log2_q16_up(s2) + 1) / 2 : 0;
}

static inline int lc_bits(const bs_upoly& u, int d) {
  bool nz;
  int bits = 0;
  mag_uf(u.c + (size_t)d * u.limbs, u.limbs, &nz, &bits);
  return bits;
}

// write `deg + 1` coefficients of src_limbs each into out (capacity checked)
static inline int put_result(bs_ctx* ctx, const uint32_t* src, int src_limbs, int deg, bs_upoly* out) {
  if (deg > out->deg) return ctx_fail(ctx, BS_ERR_CAPACITY, "output degree capacity too small");
  for (int i = 0; i <= deg; ++i) {
    const uint32_t* s = src + (size_t)i * src_limbs;
    uint32_t* d = out->c + (size_t)i * out->limbs;
    const uint32_t ext = (s[src_limbs - 1] >> 31) ? 0xffffffffu : 0u;
    for (int l = 0; l < out->limbs; ++l) d[l] = l < src_limbs ? s[l] : ext;
    const uint32_t kept = (d[out->limbs - 1] >> 31) ? 0xffffffffu : 0u;
    for (int l = out->limbs; l < src_limbs; ++l)
      if (s[l] != kept) return ctx_fail(ctx, BS_ERR_CAPACITY, "output limb capacity too small");
  }
  for (int i = deg + 1; i <= out->deg; ++i)
    std::memset(out->c + (size_t)i * out->limbs, 0, sizeof(uint32_t) * out->limbs);
  out->deg = deg;
  return 0;
}

}  // namespace bs
