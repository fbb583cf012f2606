// Square-free part in Z[x] by the modular route (Sec. 2.1, BiProject: Yun's square-free
// factorisation starts from gcd(R, R'); Sec. 5.1, "Computing gcds in Z[x]" for the
// modular gcd).
//
//   R* = pp(R / gcd(R, R')), leading coefficient positive.
//
// With G the monic gcd of R and R' over Q, Q := R / G has leading coefficient lc(R) and
// integer coefficients (R* divides R over Z, so lc(R*) divides lc(R) and Q equals
// (lc(R) / lc(R*)) R*).  Mignotte's bound for the factor R* of R gives
// ||Q||_inf <= 2^deg(R*) ||R||_2 <= 2^d ||R||_2.  For a prime p that does not divide
// lc(R) the image of Q is (R mod p) / gcd_p(R, R') whenever the modular gcd has the
// minimal degree (Brown's rule: larger degrees mark unlucky primes).  Q is rebuilt by
// Chinese remaindering, its content c is removed (R*_p = Q_p (s c)^-1, s the sign of
// lc(R)) and R* is rebuilt the same way.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <vector>

#include "ctx.cuh"

namespace bs {

struct SqfParams {
  const uint32_t* R;  // input limbs [(d + 1) * L]
  int32_t d, L;
  int32_t k_total, k_need;
  uint32_t* A;        // [k_total][d + 1] R mod p (Montgomery form)
  uint32_t* Qp;       // [k_total][d + 1] quotient residues (standard form)
  int32_t* dg;        // [k_total] gcd degree (-2: prime divides lc(R))
  int32_t* sel;       // [k_need] selected table indices
  uint32_t* rmod;     // [k_need][d + 1] residues handed to the reconstruction
  int32_t* info;      // [0] degree of Q, [1] good primes, [2] minimal gcd degree
  uint32_t* content;  // [Lc] content of Q (magnitude limbs)
  int32_t Lc;
};

// ---- reduce R mod each prime (Montgomery form)
__global__ void k_sqf_reduce(SqfParams S, Tables T) {
  const int64_t total = (int64_t)S.k_total * (S.d + 1);
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < total;
       t += (int64_t)gridDim.x * blockDim.x) {
    const int q = (int)(t / (S.d + 1));
    const int i = (int)(t - (int64_t)q * (S.d + 1));
    const PrimeConst pc = T.pc[q];
    const uint32_t* c = S.R + (int64_t)i * S.L;
    const uint32_t* pw = T.pw + (int64_t)q * (kMaxLimbs + 1);
    const uint32_t* mpw = T.mpw + (int64_t)q * (kMaxLimbs + 1);
    uint32_t acc = 0;
    for (int l = 0; l < S.L; ++l) acc = madd(acc, redc((uint64_t)c[l] * pw[l], pc.p, pc.pinv), pc.p);
    if (c[S.L - 1] >> 31) acc = msub(acc, mpw[S.L], pc.p);
    S.A[(int64_t)q * (S.d + 1) + i] = acc;
  }
}

// ---- per prime: G = gcd(R, R') monic, Q = R / G (one block, polynomials in shared memory)
__global__ void k_sqf_gcd_div(SqfParams S, Tables T) {
  extern __shared__ uint32_t sm[];
  const int d = S.d;
  uint32_t* sA = sm;          // d + 1
  uint32_t* sB = sA + d + 1;  // d + 1
  uint32_t* sR = sB + d + 1;  // d + 1 (R, kept for the division)
  __shared__ int s_la, s_lb;
  for (int q = blockIdx.x; q < S.k_total; q += gridDim.x) {
    const PrimeConst pc = T.pc[q];
    const Mod M{pc.p, pc.pinv};
    const uint32_t* Aq = S.A + (int64_t)q * (d + 1);
    // derivative: R'_i = (i + 1) R_{i+1}; (i + 1) in Montgomery form is (i + 1) R mod p
    for (int i = threadIdx.x; i <= d; i += blockDim.x) {
      const uint32_t a = Aq[i];
      sA[i] = a;
      sR[i] = a;
      const uint32_t f = redc((uint64_t)(uint32_t)(i + 1) * pc.r2, pc.p, pc.pinv);
      sB[i] = (i < d) ? mmul(Aq[i + 1], f, M) : 0u;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      int la = d, lb = d - 1;
      while (la >= 0 && sA[la] == 0) --la;
      while (lb >= 0 && sB[lb] == 0) --lb;
      s_la = la;
      s_lb = lb;
    }
    __syncthreads();
    const int dR = s_la;
    if (dR < d) {  // p divides lc(R): unlucky
      if (threadIdx.x == 0) S.dg[q] = -2;
      __syncthreads();
      continue;
    }
    uint32_t* X = sA;
    uint32_t* Y = sB;
    int la = s_la, lb = s_lb;
    while (true) {  // division-free Euclid; each pass lowers the larger degree
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
        s_la = l;
      }
      __syncthreads();
      la = s_la;
    }
    // X holds gcd (degree la >= 0 since R != 0): make it monic
    const int dgq = la;
    const uint32_t ilc = minv(X[dgq], pc.one_m, M);
    for (int i = threadIdx.x; i <= dgq; i += blockDim.x) X[i] = mmul(X[i], ilc, M);
    __syncthreads();
    // Q = R / G by long division (G monic): top-down, one quotient coefficient per step
    const int dq = d - dgq;
    uint32_t* Qo = S.Qp + (int64_t)q * (d + 1);
    for (int s = dq; s >= 0; --s) {
      const uint32_t qc = sR[s + dgq];  // leading coefficient of the current remainder
      __syncthreads();
      for (int i = threadIdx.x; i < dgq; i += blockDim.x)
        sR[s + i] = msub(sR[s + i], mmul(qc, X[i], M), M.p);
      if (threadIdx.x == 0) Qo[s] = redc((uint64_t)qc, M.p, M.pinv);  // standard form
      __syncthreads();
    }
    for (int i = dq + 1 + threadIdx.x; i <= d; i += blockDim.x) Qo[i] = 0u;
    if (threadIdx.x == 0) S.dg[q] = dgq;
    __syncthreads();
  }
}

// ---- choose the primes: minimal gcd degree among primes not dividing lc(R); J points
// at the two reconstruction jobs
__global__ void k_sqf_select(SqfParams S, Job* J) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  int mind = 1 << 30;
  for (int q = 0; q < S.k_total; ++q)
    if (S.dg[q] >= 0 && S.dg[q] < mind) mind = S.dg[q];
  int r = 0;
  for (int q = 0; q < S.k_total && r < S.k_need; ++q)
    if (S.dg[q] == mind) S.sel[r++] = q;
  S.info[0] = S.d - mind;
  S.info[1] = r;
  S.info[2] = mind;
  if (r < S.k_need) set_status(J->status, kErrUnlucky);
  for (int t = 0; t < 2; ++t) {  // both reconstructions (Q, then R*) have degree d - mind
    J[t].plan.D = S.d - mind;
    if (r < S.k_need) J[t].plan.status = kErrUnlucky;
  }
}

// ---- per selected prime: (s c)^-1 mod p in Montgomery form, s the sign of lc(R)
__global__ void k_sqf_cmod(SqfParams S, Tables T, uint32_t* cinv) {
  for (int r = blockIdx.x * blockDim.x + threadIdx.x; r < S.k_need; r += gridDim.x * blockDim.x) {
    const int q = S.sel[r];
    const PrimeConst pc = T.pc[q];
    const Mod M{pc.p, pc.pinv};
    uint64_t acc = 0;
    for (int l = S.Lc - 1; l >= 0; --l) acc = ((acc << 32) | S.content[l]) % pc.p;
    uint32_t cm = (uint32_t)acc;
    if ((S.R[(int64_t)S.d * S.L + S.L - 1] >> 31) != 0) cm = mneg(cm, pc.p);
    const uint32_t cm_m = redc((uint64_t)cm * pc.r2, pc.p, pc.pinv);
    cinv[r] = minv(cm_m, pc.one_m, M);
  }
}

// ---- gather the selected primes' quotient residues, optionally times (s c)^-1
__global__ void k_sqf_gather(SqfParams S, Tables T, const uint32_t* cinv) {
  const int dq = S.info[0];
  const int64_t total = (int64_t)S.k_need * (dq + 1);
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < total;
       t += (int64_t)gridDim.x * blockDim.x) {
    const int r = (int)(t / (dq + 1));
    const int i = (int)(t - (int64_t)r * (dq + 1));
    const int q = S.sel[r];
    uint32_t v = S.Qp[(int64_t)q * (S.d + 1) + i];
    if (cinv) {
      // standard form times Montgomery form gives standard form
      const PrimeConst pc = T.pc[q];
      v = redc((uint64_t)v * cinv[r], pc.p, pc.pinv);
    }
    S.rmod[(int64_t)r * (dq + 1) + i] = v;
  }
}

// ---- content of Q: gcd of all coefficients, by one warp --------------------------------
// A big integer of up to 32 * K limbs is spread over the lanes: lane l, slot s holds limb
// 32 s + l.  Binary gcd (Stein's algorithm) with warp-wide compare, subtract and shift;
// once the running gcd fits in 32 bits each further coefficient is reduced modulo it
// with a Horner pass and the gcd finishes in 32-bit arithmetic.
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
  const int lane = threadIdx.x & 31;
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
  (void)lane;
  return av > bv;
}

// a -= b (a >= b)
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

template <int K>
__device__ __forceinline__ void wb_load_abs(WBig<K>& a, const uint32_t* c, int L) {
  // two's complement -> magnitude, limbs beyond L are zero
  const int lane = threadIdx.x & 31;
  const bool neg = (c[L - 1] >> 31) != 0;
#pragma unroll
  for (int s = 0; s < K; ++s) {
    const int l = 32 * s + lane;
    a.v[s] = l < L ? (neg ? ~c[l] : c[l]) : 0u;
  }
  if (neg) {  // + 1 with ballot carry
    uint32_t cin = 1;
#pragma unroll
    for (int s = 0; s < K; ++s) {
      const uint32_t x = a.v[s];
      const uint32_t Pm = __ballot_sync(0xffffffffu, x == 0xffffffffu);
      // carry into lane l iff cin and all lanes below are all-ones
      const uint64_t Sx = (uint64_t)Pm + cin;
      const uint32_t C = (uint32_t)Sx ^ Pm;
      cin = (uint32_t)(Sx >> 32);
      a.v[s] = x + ((C >> lane) & 1u);
    }
    // limbs at or beyond L stay zero (the magnitude fits in L limbs)
#pragma unroll
    for (int s = 0; s < K; ++s)
      if (32 * s + lane >= L) a.v[s] = 0u;
  }
}

__device__ __forceinline__ uint32_t gcd32(uint32_t a, uint32_t b) {
  while (b) {
    const uint32_t t = a % b;
    a = b;
    b = t;
  }
  return a;
}

// magnitude of coefficient c modulo m (32-bit), lane 0 result broadcast
__device__ __forceinline__ uint32_t abs_mod32(const uint32_t* c, int L, uint32_t m) {
  const bool neg = (c[L - 1] >> 31) != 0;
  uint64_t r = 0;
  // value of the two's complement number modulo m, then negate if negative
  for (int l = L - 1; l >= 0; --l) r = ((r << 32) | c[l]) % m;
  if (neg) {
    // v = raw - 2^(32 L); |v| = 2^(32 L) - raw
    uint64_t t = 1 % m;
    for (int l = 0; l < L; ++l) t = (t << 32) % m;
    r = (t + m - r) % m;
  }
  return (uint32_t)r;
}

template <int K>
__device__ void content_warp(const uint32_t* coef, int n, int L, uint32_t* out, int Lout) {
  const int lane = threadIdx.x & 31;
  WBig<K> g, b;
  // start from the first nonzero coefficient
  int i0 = -1;
  for (int i = 0; i < n; ++i) {
    bool nz = false;
    for (int l = lane; l < L; l += 32) nz = nz || coef[(int64_t)i * L + l] != 0;
    if (__any_sync(0xffffffffu, nz)) {
      i0 = i;
      break;
    }
  }
  if (i0 < 0) {
    for (int l = lane; l < Lout; l += 32) out[l] = (l == 0) ? 1u : 0u;
    return;
  }
  wb_load_abs<K>(g, coef + (int64_t)i0 * L, L);
  for (int i = i0 + 1; i < n; ++i) {
    if (wb_top<K>(g) == 0) {
      // small gcd: finish in 32-bit arithmetic
      uint32_t g32 = __shfl_sync(0xffffffffu, g.v[0], 0);
      for (int j = i; j < n && g32 != 1u; ++j) {
        uint32_t r = 0;
        if (lane == 0) r = abs_mod32(coef + (int64_t)j * L, L, g32);
        r = __shfl_sync(0xffffffffu, r, 0);
        g32 = gcd32(g32, r);
      }
#pragma unroll
      for (int s = 0; s < K; ++s) g.v[s] = (s == 0 && lane == 0) ? g32 : 0u;
      break;
    }
    wb_load_abs<K>(b, coef + (int64_t)i * L, L);
    if (wb_is_zero<K>(b)) continue;
    // binary gcd of g and b
    const int tg = wb_ctz<K>(g), tb = wb_ctz<K>(b);
    const int sh = tg < tb ? tg : tb;
    wb_shr<K>(g, tg);
    for (int it = 0; it < 1 << 20; ++it) {  // bounded: each pass removes >= one bit
      wb_shr<K>(b, wb_ctz<K>(b));
      if (wb_gt<K>(g, b)) {
        const WBig<K> t = g;
        g = b;
        b = t;
      }
      wb_sub<K>(b, g);
      if (wb_is_zero<K>(b)) break;
    }
    // g <<= sh
    for (int n2 = sh; n2 > 0;) {
      const int step = n2 < 31 ? n2 : 31;
#pragma unroll
      for (int s = K - 1; s >= 0; --s) {
        uint32_t lo = __shfl_up_sync(0xffffffffu, g.v[s], 1);
        const uint32_t prv = (s > 0) ? __shfl_sync(0xffffffffu, g.v[s > 0 ? s - 1 : 0], 31) : 0u;
        if (lane == 0) lo = prv;
        g.v[s] = (g.v[s] << step) | (lo >> (32 - step));
      }
      n2 -= step;
    }
  }
#pragma unroll
  for (int s = 0; s < K; ++s) {
    const int l = 32 * s + lane;
    if (l < Lout) out[l] = g.v[s];
  }
  for (int l = 32 * K + lane; l < Lout; l += 32) out[l] = 0u;
}

__global__ void k_sqf_content(SqfParams S, const uint32_t* qlimbs, int Lq) {
  if (blockIdx.x != 0 || threadIdx.x >= 32) return;
  const int n = S.info[0] + 1;
  const int K = (Lq + 31) / 32;
  if (K <= 1)
    content_warp<1>(qlimbs, n, Lq, S.content, S.Lc);
  else if (K <= 2)
    content_warp<2>(qlimbs, n, Lq, S.content, S.Lc);
  else if (K <= 4)
    content_warp<4>(qlimbs, n, Lq, S.content, S.Lc);
  else
    content_warp<8>(qlimbs, n, Lq, S.content, S.Lc);
}

}  // namespace bs

using namespace bs;

extern "C" int bs_squarefree_part(bs_ctx* ctx, const bs_upoly* r, bs_upoly* out) {
  if (!ctx) return BS_ERR_ARG;
  if (!r || !out || r->deg < -1 || r->limbs < 1 || r->limbs > kMaxLimbs || (r->deg >= 0 && !r->c))
    return ctx_fail(ctx, BS_ERR_ARG, "bad arguments");
  const int L = r->limbs;
  int d = r->deg;
  auto coef_zero = [&](int i) {
    for (int l = 0; l < L; ++l)
      if (r->c[(size_t)i * L + l]) return false;
    return true;
  };
  while (d >= 0 && coef_zero(d)) --d;
  if (d < 0) return ctx_fail(ctx, BS_ERR_ZERO, "square-free part of the zero polynomial");
  // ||R||_2^2 as an upper float; the quotient bound 2^d ||R||_2, one bit of margin
  UF s2{0u, 0};
  for (int i = 0; i <= d; ++i) {
    bool nz;
    int bits;
    const UF u = mag_uf(r->c + (size_t)i * L, L, &nz, &bits);
    if (nz) s2 = uf_add(s2, uf_mul(u, u));
  }
  const int64_t l2 = (uf_log2_q16_up(s2) + 1) / 2;  // log2 ||R||_2, Q16, rounded up
  const int64_t bitsB = (int64_t)d + (l2 + 65535) / 65536 + 1;
  const HostPrimes& H = host_primes();
  const int T = (int)H.p.size();
  const int64_t need = (bitsB + 2) * 65536;
  if (H.lg_prefix[T] < need) return ctx_fail(ctx, BS_ERR_RANGE, "bound exceeds the prime table");
  int k_need = prime_count_host(H.lg_prefix.data(), T, need);
  if (k_need < 1) k_need = 1;
  bool lcnz;
  int lcbits;
  mag_uf(r->c + (size_t)d * L, L, &lcnz, &lcbits);
  const int k_total = std::min(T, k_need + 4 + k_need / 8 + lcbits / 30);
  const int out_limbs = (int)((bitsB + 2 + 31) / 32);
  if (!out->c) {
    out->deg = d;
    out->limbs = out_limbs;
    return BS_OK;
  }
  if (d == 0) {  // a nonzero constant: the square-free part is 1
    if (out->limbs < 1 || out->deg < 0) return ctx_fail(ctx, BS_ERR_CAPACITY, "output capacity");
    std::memset(out->c, 0, sizeof(uint32_t) * (size_t)(out->deg + 1) * out->limbs);
    out->c[0] = 1;
    out->deg = 0;
    return BS_OK;
  }
  if (out->deg < d || out->limbs < 1) return ctx_fail(ctx, BS_ERR_CAPACITY, "output capacity");
  if (out_limbs > 256) return ctx_fail(ctx, BS_ERR_RANGE, "coefficients above 8192 bits");
  if ((size_t)3 * (d + 1) * sizeof(uint32_t) > (size_t)ctx->smem_optin - 64)
    return ctx_fail(ctx, BS_ERR_RANGE, "degree too large for one block");
  cudaSetDevice(ctx->device);
  int rc = ctx->tabs.ensure(k_total, 0, ctx->stream);
  if (rc) return ctx_fail(ctx, rc, "table setup failed");
  const int n1 = d + 1;
  Layout lay;
  const size_t o_R = lay.take(sizeof(uint32_t) * (size_t)n1 * L);
  const size_t o_A = lay.take(sizeof(uint32_t) * (size_t)k_total * n1);
  const size_t o_Q = lay.take(sizeof(uint32_t) * (size_t)k_total * n1);
  const size_t o_dg = lay.take(sizeof(int32_t) * k_total);
  const size_t o_sel = lay.take(sizeof(int32_t) * k_need);
  const size_t o_rmod = lay.take(sizeof(uint32_t) * (size_t)k_need * n1);
  const size_t o_info = lay.take(sizeof(int32_t) * 4);
  const size_t o_cont = lay.take(sizeof(uint32_t) * out_limbs);
  const size_t o_cinv = lay.take(sizeof(uint32_t) * k_need);
  const size_t o_qout = lay.take(sizeof(uint32_t) * (size_t)n1 * out_limbs);
  const size_t o_rout = lay.take(sizeof(uint32_t) * (size_t)n1 * out_limbs);
  const size_t o_jobs = lay.take(sizeof(Job) * 2);
  const size_t o_off = lay.take(sizeof(int64_t) * 2);
  const size_t o_st = lay.take(sizeof(int32_t) * 4);
  rc = ensure_workspace(ctx, lay.used);
  if (rc) return rc;
  char* base = (char*)ctx->ws;
  cudaStream_t s = ctx->stream;
  SqfParams S;
  S.R = (const uint32_t*)(base + o_R);
  S.d = d;
  S.L = L;
  S.k_total = k_total;
  S.k_need = k_need;
  S.A = (uint32_t*)(base + o_A);
  S.Qp = (uint32_t*)(base + o_Q);
  S.dg = (int32_t*)(base + o_dg);
  S.sel = (int32_t*)(base + o_sel);
  S.rmod = (uint32_t*)(base + o_rmod);
  S.info = (int32_t*)(base + o_info);
  S.content = (uint32_t*)(base + o_cont);
  S.Lc = out_limbs;
  // the two reconstructions (Q, then R*) as jobs of the common reconstruction kernels
  Job J[2];
  for (int t = 0; t < 2; ++t) {
    std::memset(&J[t], 0, sizeof(Job));
    J[t].plan.k_need = k_need;
    J[t].plan.k_total = k_total;
    J[t].plan.D = d;  // the selection kernel lowers it to deg Q
    J[t].plan.out_limbs = out_limbs;
    J[t].cap_deg = d;
    J[t].cap_limbs = out_limbs;
    J[t].sel = S.sel;
    J[t].rmod = S.rmod;
    J[t].out = (uint32_t*)(base + (t == 0 ? o_qout : o_rout));
    J[t].status = (int32_t*)(base + o_st);
  }
  Job* dJ = (Job*)(base + o_jobs);
  const int64_t offs[2] = {0, (int64_t)(d + kCrtTile) / kCrtTile};
  rc |= ctx_cuda(ctx, cudaMemcpyAsync(base + o_R, r->c, sizeof(uint32_t) * (size_t)n1 * L, cudaMemcpyHostToDevice, s), "h2d");
  rc |= ctx_cuda(ctx, cudaMemcpyAsync(dJ, J, sizeof(J), cudaMemcpyHostToDevice, s), "h2d");
  rc |= ctx_cuda(ctx, cudaMemcpyAsync(base + o_off, offs, sizeof(offs), cudaMemcpyHostToDevice, s), "h2d");
  rc |= ctx_cuda(ctx, cudaMemsetAsync(base + o_st, 0, sizeof(int32_t) * 4, s), "memset");
  if (rc) return rc;
  const Tables Tv = ctx->tabs.view();
  const size_t gsm = (size_t)3 * n1 * sizeof(uint32_t);
  if (gsm > 48 * 1024 && set_dyn_smem_limit((const void*)k_sqf_gcd_div, ctx->smem_optin) != 0)
    return ctx_fail(ctx, BS_ERR_CUDA, "shared memory limit");
  const int nthr = std::min(1024, std::max(32, (n1 + 31) / 32 * 32));
  k_sqf_reduce<<<std::min<int64_t>(4 * ctx->sms, ((int64_t)k_total * n1 + 255) / 256), 256, 0, s>>>(S, Tv);
  k_sqf_gcd_div<<<k_total, nthr, gsm, s>>>(S, Tv);
  k_sqf_select<<<1, 32, 0, s>>>(S, dJ);
  rc = ctx_cuda(ctx, cudaGetLastError(), "launch");
  if (rc) return rc;
  const WorkList wl{nullptr, (const int64_t*)(base + o_off), 1};
  const int crt_grid = (int)std::min<int64_t>(offs[1], (int64_t)4 * ctx->sms);
  const int lmax = out_limbs;
  auto crt = [&](const Job* jobp) {
    size_t smem = ((size_t)k_need * k_need + (size_t)k_need * lmax + (size_t)k_need * kCrtTile +
                   3 * (size_t)k_need + (size_t)kCrtTile * k_need + (size_t)kCrtTile * lmax) *
                  sizeof(uint32_t);
    if (k_need <= kCrtWarpMaxK && smem <= (size_t)ctx->smem_optin - 64) {
      launch_crt_w(crt_grid, smem, s, jobp, wl, Tv, k_need, lmax);
    } else {
      const size_t per = (size_t)3 * lmax * sizeof(uint32_t);
      const size_t fixed = ((size_t)k_need * kCrtTile + 3 * (size_t)k_need) * sizeof(uint32_t);
      if (fixed + per > (size_t)ctx->smem_optin - 64) return (int)kErrRange;
      const int w = (int)std::min<size_t>(kCrtWarps, ((size_t)ctx->smem_optin - 64 - fixed) / per);
      launch_crt(crt_grid, w * 32, fixed + per * w, s, jobp, wl, Tv, k_need, lmax, 0);
    }
    return 0;
  };
  k_sqf_gather<<<4 * ctx->sms, 256, 0, s>>>(S, Tv, nullptr);
  if (crt(dJ)) return ctx_fail(ctx, BS_ERR_RANGE, "too many primes for the reconstruction stage");
  k_sqf_content<<<1, 32, 0, s>>>(S, (const uint32_t*)(base + o_qout), out_limbs);
  k_sqf_cmod<<<(k_need + 127) / 128, 128, 0, s>>>(S, Tv, (uint32_t*)(base + o_cinv));
  k_sqf_gather<<<4 * ctx->sms, 256, 0, s>>>(S, Tv, (const uint32_t*)(base + o_cinv));
  if (crt(dJ + 1)) return ctx_fail(ctx, BS_ERR_RANGE, "too many primes for the reconstruction stage");
  rc = ctx_cuda(ctx, cudaGetLastError(), "launch");
  if (rc) return rc;
  std::vector<uint32_t> res((size_t)n1 * out_limbs);
  int32_t info[4], st[4];
  rc |= ctx_cuda(ctx, cudaMemcpyAsync(res.data(), base + o_rout, sizeof(uint32_t) * res.size(), cudaMemcpyDeviceToHost, s), "d2h");
  rc |= ctx_cuda(ctx, cudaMemcpyAsync(info, base + o_info, sizeof(info), cudaMemcpyDeviceToHost, s), "d2h");
  rc |= ctx_cuda(ctx, cudaMemcpyAsync(st, base + o_st, sizeof(st), cudaMemcpyDeviceToHost, s), "d2h");
  rc |= ctx_cuda(ctx, cudaStreamSynchronize(s), "stream");
  if (rc) return rc;
  if (st[0]) return ctx_fail(ctx, st[0], "device stage reported a failure");
  const int dq = info[0];
  // copy out, narrowing to the caller's limbs
  for (int i = 0; i <= dq; ++i) {
    const uint32_t* src = res.data() + (size_t)i * out_limbs;
    uint32_t* dst = out->c + (size_t)i * out->limbs;
    const uint32_t ext = (src[out_limbs - 1] >> 31) ? 0xffffffffu : 0u;
    for (int l = 0; l < out->limbs; ++l) dst[l] = l < out_limbs ? src[l] : ext;
    const uint32_t kept = (dst[out->limbs - 1] >> 31) ? 0xffffffffu : 0u;
    for (int l = out->limbs; l < out_limbs; ++l)
      if (src[l] != kept) return ctx_fail(ctx, BS_ERR_CAPACITY, "output limb capacity too small");
  }
  for (int i = dq + 1; i <= out->deg; ++i)
    std::memset(out->c + (size_t)i * out->limbs, 0, sizeof(uint32_t) * out->limbs);
  out->deg = dq;
  return BS_OK;
}
