// Univariate resultant mod p with formal degrees, one instance per thread (step (c) of
// the modular algorithm, Sec. 5.1).
//
// Both polynomials live in registers, top-aligned (index 0 holds the formal leading
// coefficient).  The longer one is reduced by the shorter with division-free
// elimination; when the length difference is at least one, two elimination steps are
// fused into one pass over the coefficients (a pseudo-remainder by a quadratic
// multiplier).  Every identity used keeps the result equal to the determinant of the
// formal-shape Sylvester matrix:
//
//   Res_{n,m}(A + hB, B)  = Res_{n,m}(A, B)                      (deg hB <= n)
//   Res_{n,m}(cA, B)      = c^m Res_{n,m}(A, B),   Res_{n,m}(A, cB) = c^n Res_{n,m}(A, B)
//   Res_{n,m}(A, B)       = (-1)^m b_m Res_{n-1,m}(A, B)         (a_n = 0)
//   Res_{n,m}(A, B)       = a_n Res_{n,m-1}(A, B)                (b_m = 0)
//   Res_{n,0}(A, b_0) = b_0^n,  Res_{0,m}(a_0, B) = a_0^m.
//
// The scaling factors form a product prod_i x_i^{e_i} with non-increasing exponents
// e_i = (degree of the pivot polynomial) - 1; it is accumulated with one running prefix
// product (prod_i x_i^{e_i} = prod_j (x_0 ... x_j)^{e_j - e_{j+1}}), so the generic
// step costs two multiplications instead of a power.  One inversion at the end divides
// it out.
#pragma once
#include "modarith.cuh"

namespace bs {

// Register arrays hold ceil4(L) + 2 entries; entries at or beyond a polynomial's length
// are zero.  The passes below update four coefficients per exit test, so independent
// updates overlap; updates past the length read only zeros and write zeros, which keeps
// the invariant.
template <int L>
struct Arr {
  static constexpr int LL = (L + 3) / 4 * 4;  // rounded-up length
  static constexpr int N = LL + 2;            // storage (two zeros of headroom)
};

// P[u] = c2 P[u+2] + nc1 Q[u+2] + nc0 Q[u+1] for u < lp - 2, the new length (Q is at
// most lp - 1 long).  The sum of the three products is below 3p^2; for a prime with
// 3p < 2^32 (SMALLP) that is below p 2^32 and Montgomery's reduction applies directly,
// otherwise the high word is folded once first.  The blocks of four stop at the first
// multiple of four at or above lp - 2: the updates there past lp - 2 read only zeros and
// write zeros, and each block clears the two entries after it (it has read them; the next
// block overwrites them), which leaves zeros in the at most two entries between the last
// block and lp.  No update is spent on the two entries that the pass removes.
template <int L, bool SMALLP = false, class AP, class AQ>
__device__ __forceinline__ void fused_pass(AP& P, int lp, const AQ& Q, uint32_t c2,
                                           uint32_t nc1, uint32_t nc0, uint32_t p, uint32_t pinv) {
  const int ln = lp - 2;
#pragma unroll
  for (int u0 = 0; u0 < Arr<L>::LL; u0 += 4) {
    if (u0 >= ln) break;
#pragma unroll
    for (int u = u0; u < u0 + 4; ++u) {
      const uint64_t t = (uint64_t)c2 * P[u + 2] + (uint64_t)nc1 * Q[u + 2] + (uint64_t)nc0 * Q[u + 1];
      P[u] = SMALLP ? redc(t, p, pinv) : redc_wide(t, p, pinv);
    }
    P[u0 + 4] = 0u;
    P[u0 + 5] = 0u;
  }
}

// P[u] = b0 P[u+1] + na0 Q[u+1] for u < lp
template <int L, class AP, class AQ>
__device__ __forceinline__ void single_pass(AP& P, int lp, const AQ& Q, uint32_t b0,
                                            uint32_t na0, uint32_t p, uint32_t pinv) {
#pragma unroll
  for (int u0 = 0; u0 < Arr<L>::LL; u0 += 4) {
    if (u0 >= lp) break;
#pragma unroll
    for (int u = u0; u < u0 + 4; ++u) {
      const uint64_t t = (uint64_t)b0 * P[u + 1] + (uint64_t)na0 * Q[u + 1];
      P[u] = redc(t, p, pinv);
    }
  }
}

template <int L, class AP>
__device__ __forceinline__ void shift_pass(AP& P, int lp) {
#pragma unroll
  for (int u0 = 0; u0 < Arr<L>::LL; u0 += 4) {
    if (u0 >= lp) break;
#pragma unroll
    for (int u = u0; u < u0 + 4; ++u) P[u] = P[u + 1];
  }
}

// Returns num (Montgomery form, sign applied) and stores den so that the resultant is
// num / den.  A and B hold la and lb coefficients (la, lb >= 1), zero beyond.
template <int L, bool SMALLP = false, class AT>
__device__ __forceinline__ uint32_t unires_numden(AT& A, int la, AT& B, int lb, const Mod M,
                                                  uint32_t one_m, uint32_t* den_out) {
  const uint32_t p = M.p, pinv = M.pinv;
  uint32_t num = one_m, den = one_m, pre = one_m;
  int eprev = -1;
  uint32_t neg = 0;
  while (la > 1 && lb > 1) {
    if (la >= lb) {
      const uint32_t b0 = B[0];
      if (b0 == 0) {  // drop the formal degree of B
        num = mmul(num, A[0], M);
        shift_pass<L>(B, lb);
        lb -= 1;
        continue;
      }
      const int e = lb - 2;
      if (eprev >= 0) {
        int d = eprev - e;
        if (d == 1)
          den = mmul(den, pre, M);
        else if (d > 1)
          den = mmul(den, mpow(pre, (uint32_t)d, one_m, M), M);
      }
      eprev = e;
      const uint32_t a0 = A[0];
      if (la > lb) {
        const uint32_t a1 = A[1], b1 = B[1];
        const uint32_t c2 = mmul(b0, b0, M);
        const uint32_t c1 = mmul(b0, a0, M);
        const uint32_t c0 = redc((uint64_t)b0 * a1 + (uint64_t)(p - a0) * b1, p, pinv);
        fused_pass<L, SMALLP>(A, la, B, c2, p - c1, p - c0, p, pinv);
        la -= 2;
        pre = mmul(pre, c2, M);
      } else {
        single_pass<L>(A, la, B, b0, p - a0, p, pinv);
        la -= 1;
        pre = mmul(pre, b0, M);
        neg ^= (uint32_t)(lb - 1) & 1u;
      }
    } else {
      const uint32_t a0 = A[0];
      if (a0 == 0) {  // drop the formal degree of A
        num = mmul(num, B[0], M);
        neg ^= (uint32_t)(lb - 1) & 1u;
        shift_pass<L>(A, la);
        la -= 1;
        continue;
      }
      const int e = la - 2;
      if (eprev >= 0) {
        int d = eprev - e;
        if (d == 1)
          den = mmul(den, pre, M);
        else if (d > 1)
          den = mmul(den, mpow(pre, (uint32_t)d, one_m, M), M);
      }
      eprev = e;
      const uint32_t b0 = B[0], b1 = B[1], a1 = A[1];
      const uint32_t c2 = mmul(a0, a0, M);
      const uint32_t c1 = mmul(a0, b0, M);
      const uint32_t c0 = redc((uint64_t)a0 * b1 + (uint64_t)(p - b0) * a1, p, pinv);
      fused_pass<L, SMALLP>(B, lb, A, c2, p - c1, p - c0, p, pinv);
      lb -= 2;
      pre = mmul(pre, c2, M);
    }
  }
  uint32_t r;
  if (lb == 1)
    r = mpow(B[0], (uint32_t)(la - 1), one_m, M);
  else
    r = mpow(A[0], (uint32_t)(lb - 1), one_m, M);
  num = mmul(num, r, M);
  if (eprev > 0) den = mmul(den, mpow(pre, (uint32_t)eprev, one_m, M), M);
  if (neg) num = mneg(num, p);
  *den_out = den;
  return num;
}

}  // namespace bs
