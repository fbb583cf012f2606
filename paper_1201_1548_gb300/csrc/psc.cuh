// Principal subresultant coefficients mod p with formal degrees, one instance per thread
// (Sec. 3.3: the psc sequence sr_0, ..., sr_(q-1) of the specialised pair at a point).
//
// The division-free elimination of unires.cuh changes the pair (A, B) of formal degrees
// (a, b) by steps whose effect on every principal subresultant coefficient of index
// i <= min(a, b) after the step is known:
//   A <- c A + h B (deg hB <= a):    sr_i(A, B) = c^-(b-i) sr_i(c A + h B, B)
//   B <- c B + h A (deg hA <= b):    sr_i(A, B) = c^-(a-i) sr_i(A, c B + h A)
//   a_a = 0:                         sr_i^(a,b) = (-1)^(b-i) b_b sr_i^(a-1,b)
//   b_b = 0:                         sr_i^(a,b) = a_a sr_i^(a,b-1)
// (the last two expand the determinant along its first column).  When the shorter
// polynomial has formal degree s and leading coefficient t and the longer one formal
// degree l > s, sr_s of the current pair is t^(l-s) (a triangular determinant; 0 for t = 0).
// The smaller formal degree falls by at most one per step, so every index q-1, ..., 0 is
// met once, in that order, and recorded there.
//
// With e the smaller formal degree at a scaling step, the factors combine into
//   sr_s(original) = (-1)^(sg + vneg s) U t^(l-s) / W_s,   W_s = prod c^(e - s),
// where U collects the leading coefficients of the degree drops, sg and vneg the signs,
// and W_s = W_(s+1) * (product of all scalings so far).  The numerators are stored as they
// are met, together with those products; one inversion of W_0 and a backward sweep
// (1/W_(s+1) = r_s / W_s) finish all q values.
#pragma once
#include "unires.cuh"

namespace bs {

// A, B top-aligned (index 0 holds the formal leading coefficient), la, lb >= 1 entries;
// q = min(la, lb) - 1 values are written to out[s * ostride] (Montgomery form), using
// scr[s * sstride] as scratch.
template <int L>
__device__ __forceinline__ void psc_seq(uint32_t (&A)[Arr<L>::N], int la, uint32_t (&B)[Arr<L>::N], int lb,
                                        const Mod M, uint32_t one_m, uint32_t* out, int64_t ostride,
                                        uint32_t* scr, int64_t sstride) {
  const uint32_t p = M.p, pinv = M.pinv;
  const int q = (la < lb ? la : lb) - 1;
  if (q <= 0) return;
  uint32_t U = one_m, Vabs = one_m, W = one_m;
  uint32_t sg = 0, vneg = 0;
  int rec = q - 1;
  // record sr_s when the smaller formal degree first equals s (and the other is larger)
  auto record = [&]() {
    const int s = (la < lb ? la : lb) - 1;
    if (s != rec || la == lb) return;
    const int l = (la < lb ? lb : la) - 1;
    const uint32_t t = (la < lb) ? A[0] : B[0];
    W = mmul(W, Vabs, M);
    uint32_t v = 0;
    if (t != 0) {
      v = mmul(U, mpow(t, (uint32_t)(l - s), one_m, M), M);
      if ((sg ^ (vneg & (uint32_t)s)) & 1u) v = mneg(v, p);
    }
    out[rec * ostride] = v;
    scr[rec * sstride] = Vabs;
    --rec;
  };
  while (la > 1 && lb > 1) {
    record();
    if (la >= lb) {
      const uint32_t b0 = B[0];
      const uint32_t a0 = A[0];
      if (b0 == 0) {  // drop the formal degree of B: factor a_a
        U = mmul(U, a0, M);
        shift_pass<L>(B, lb);
        lb -= 1;
        continue;
      }
      if (la > lb) {  // A <- b0^2 A - (...) B, then two drops of A (factor b0 each, signs cancel)
        const uint32_t a1 = A[1], b1 = B[1];
        const uint32_t c2 = mmul(b0, b0, M);
        const uint32_t c1 = mmul(b0, a0, M);
        const uint32_t c0 = redc((uint64_t)b0 * a1 + (uint64_t)(p - a0) * b1, p, pinv);
        fused_pass<L>(A, la, B, c2, p - c1, p - c0, p, pinv);
        la -= 2;
        Vabs = mmul(Vabs, c2, M);
        U = mmul(U, c2, M);
      } else {  // A <- b0 A - a0 B, then one drop of A: factor (-1)^(b-i) b0
        single_pass<L>(A, la, B, b0, p - a0, p, pinv);
        la -= 1;
        Vabs = mmul(Vabs, b0, M);
        U = mmul(U, b0, M);
        sg ^= (uint32_t)(lb - 1) & 1u;
        vneg ^= 1u;
      }
    } else {
      const uint32_t a0 = A[0];
      if (a0 == 0) {  // drop the formal degree of A: factor (-1)^(b-i) b_b
        U = mmul(U, B[0], M);
        sg ^= (uint32_t)(lb - 1) & 1u;
        vneg ^= 1u;
        shift_pass<L>(A, la);
        la -= 1;
        continue;
      }
      // B <- a0^2 B - (...) A, then two drops of B (factor a0 each)
      const uint32_t b0 = B[0], b1 = B[1], a1 = A[1];
      const uint32_t c2 = mmul(a0, a0, M);
      const uint32_t c1 = mmul(a0, b0, M);
      const uint32_t c0 = redc((uint64_t)a0 * b1 + (uint64_t)(p - b0) * a1, p, pinv);
      fused_pass<L>(B, lb, A, c2, p - c1, p - c0, p, pinv);
      lb -= 2;
      Vabs = mmul(Vabs, c2, M);
      U = mmul(U, c2, M);
    }
  }
  record();  // index 0: one polynomial is a constant
  // out[s] holds numerators; W = W_0.  1/W_(s+1) = r_s / W_s with r_s = scr[s].
  uint32_t inv = minv(W, one_m, M);
  for (int s = 0; s < q; ++s) {
    out[s * ostride] = mmul(out[s * ostride], inv, M);
    inv = mmul(inv, scr[s * sstride], M);
  }
}


// The d-th subresultant polynomial S_d(A, B) mod p with formal degrees (Sec. 3.3, the
// Sres_i matrix), 0 <= d < min(la, lb) - 1.  The row operations and column expansions
// above change every subresultant polynomial by the same factors as its principal
// coefficient, and when the shorter polynomial P (formal degree d, formal leading
// coefficient t) first meets index d next to a longer one of formal degree l > d, the
// current pair has S_d = t^(l-d-1) P (a triangular determinant whose last column holds
// the polynomials; for t = 0 and l > d + 1 it vanishes).  Hence
//   coefficient of y^j of S_d(original) = (-1)^(sg + vneg d) U t^(l-d-1) P[d - j] / W_d.
// The elimination stops there and the d + 1 coefficients (Montgomery form) go to
// out[j * ostride].  Returns false only if index d is never met (d out of range).
template <int L>
__device__ __forceinline__ bool sres_seq(uint32_t (&A)[Arr<L>::N], int la, uint32_t (&B)[Arr<L>::N], int lb,
                                         int d, const Mod M, uint32_t one_m, uint32_t* out, int64_t ostride) {
  const uint32_t p = M.p, pinv = M.pinv;
  uint32_t U = one_m, Vabs = one_m, W = one_m;
  uint32_t sg = 0, vneg = 0;
  int rec = (la < lb ? la : lb) - 2;  // the next index met (q - 1)
  bool met = false;
  while (true) {
    const int s = (la < lb ? la : lb) - 1;
    if (s == rec && la != lb) {
      W = mmul(W, Vabs, M);
      if (s == d) {
        met = true;
        break;
      }
      --rec;
    }
    if (!(la > 1 && lb > 1)) break;  // index d not met (d out of range)
    if (la >= lb) {
      const uint32_t b0 = B[0];
      const uint32_t a0 = A[0];
      if (b0 == 0) {
        U = mmul(U, a0, M);
        shift_pass<L>(B, lb);
        lb -= 1;
        continue;
      }
      if (la > lb) {
        const uint32_t a1 = A[1], b1 = B[1];
        const uint32_t c2 = mmul(b0, b0, M);
        const uint32_t c1 = mmul(b0, a0, M);
        const uint32_t c0 = redc((uint64_t)b0 * a1 + (uint64_t)(p - a0) * b1, p, pinv);
        fused_pass<L>(A, la, B, c2, p - c1, p - c0, p, pinv);
        la -= 2;
        Vabs = mmul(Vabs, c2, M);
        U = mmul(U, c2, M);
      } else {
        single_pass<L>(A, la, B, b0, p - a0, p, pinv);
        la -= 1;
        Vabs = mmul(Vabs, b0, M);
        U = mmul(U, b0, M);
        sg ^= (uint32_t)(lb - 1) & 1u;
        vneg ^= 1u;
      }
    } else {
      const uint32_t a0 = A[0];
      if (a0 == 0) {
        U = mmul(U, B[0], M);
        sg ^= (uint32_t)(lb - 1) & 1u;
        vneg ^= 1u;
        shift_pass<L>(A, la);
        la -= 1;
        continue;
      }
      const uint32_t b0 = B[0], b1 = B[1], a1 = A[1];
      const uint32_t c2 = mmul(a0, a0, M);
      const uint32_t c1 = mmul(a0, b0, M);
      const uint32_t c0 = redc((uint64_t)a0 * b1 + (uint64_t)(p - b0) * a1, p, pinv);
      fused_pass<L>(B, lb, A, c2, p - c1, p - c0, p, pinv);
      lb -= 2;
      Vabs = mmul(Vabs, c2, M);
      U = mmul(U, c2, M);
    }
  }
  if (!met) return false;
  const bool a_short = la < lb;
  const int l = (a_short ? lb : la) - 1;
  const uint32_t t = a_short ? A[0] : B[0];
  uint32_t v = mmul(U, mpow(t, (uint32_t)(l - d - 1), one_m, M), M);
  if ((sg ^ (vneg & (uint32_t)d)) & 1u) v = mneg(v, p);
  v = mmul(v, minv(W, one_m, M), M);
#pragma unroll
  for (int k = 0; k < Arr<L>::N; ++k)
    if (k <= d) out[(int64_t)(d - k) * ostride] = mmul(v, a_short ? A[k] : B[k], M);
  return true;
}

}  // namespace bs
