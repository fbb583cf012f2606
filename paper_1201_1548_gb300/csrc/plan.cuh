// Planning of one resultant job: actual degrees, the degree bound D, the transform size
// N, the coefficient bound B, the number of primes, spare primes and output limbs.
// The same code runs on the host (host-resident inputs) and in a one-block-per-job
// device kernel (device-resident inputs).  No floating point is used: magnitudes are
// carried as "upper floats" (a 32-bit mantissa and a binary exponent, always rounded
// up), so every derived quantity is a guaranteed upper bound.
//
// Degree bound (Sec. 2, below the Sylvester matrix): deg R <= m * n for total degrees
// m, n; every term of det S also has degree <= n_e deg_o f + m_e deg_o g, where e is
// the eliminated variable and o the other one.  D is the smaller of the two.
//
// Coefficient bound: |coef R| <= B = (sum_j ||f_j||_1^2)^(n_e/2) (sum_j ||g_j||_1^2)^(m_e/2)
// (Hadamard's inequality on the unit circle); primes are taken until prod p > 4B,
// one bit more than symmetric residues need.
#pragma once
#include <stdint.h>

#include "modarith.cuh"

namespace bs {

constexpr int kLogNMax = 14;             // transform sizes up to 2^14 (p = 1 mod 2^14)
constexpr int kNMax = 1 << kLogNMax;
constexpr int kMaxLimbs = 64;            // input coefficients up to 2048 bits
constexpr int kMaxUniLimbs = 256;        // univariate inputs of the gcd pipelines: 8192 bits
constexpr int kUniMaxLen = 129;          // univariate stage: degrees up to 128
constexpr int kWsMaxK = 256;             // weighted-sum reconstruction up to 256 primes

BS_HD int clz64(uint64_t v) {
#ifdef __CUDA_ARCH__
  return __clzll((long long)v);
#else
  return v ? __builtin_clzll(v) : 64;
#endif
}
BS_HD int clz32(uint32_t v) {
#ifdef __CUDA_ARCH__
  return __clz((int)v);
#else
  return v ? __builtin_clz(v) : 32;
#endif
}

// value <= m * 2^e ; m == 0 encodes 0, otherwise 2^31 <= m < 2^32
struct UF {
  uint32_t m;
  int32_t e;
};

// an upper bound of v * 2^e (plus one unit of 2^e when `inexact`)
BS_HD UF uf_make(uint64_t v, int32_t e, bool inexact) {
  if (inexact) v += 1;
  if (v == 0) return UF{0u, 0};
  int lz = clz64(v);
  int sh = 32 - lz;
  if (sh > 0) {
    uint64_t lost = v & ((1ull << sh) - 1ull);
    uint64_t m = v >> sh;
    if (lost) m += 1;
    if (m >> 32) {
      m >>= 1;
      sh += 1;
    }
    return UF{(uint32_t)m, e + sh};
  }
  return UF{(uint32_t)(v << (-sh)), e + sh};
}

BS_HD UF uf_add(UF a, UF b) {
  if (!a.m) return b;
  if (!b.m) return a;
  if (a.e < b.e) {
    UF t = a;
    a = b;
    b = t;
  }
  int d = a.e - b.e;
  uint64_t A = (uint64_t)a.m << 31;
  uint64_t B = 0;
  bool inexact = false;
  if (d <= 31) {
    B = (uint64_t)b.m << (31 - d);
  } else if (d < 63) {
    int s = d - 31;
    B = (uint64_t)b.m >> s;
    inexact = ((uint64_t)b.m & ((1ull << s) - 1ull)) != 0;
  } else {
    inexact = true;
  }
  return uf_make(A + B, a.e - 31, inexact);
}

BS_HD UF uf_mul(UF a, UF b) {
  if (!a.m || !b.m) return UF{0u, 0};
  return uf_make((uint64_t)a.m * b.m, a.e + b.e, false);
}

// ceil-ish upper bound of log2(a) in Q16 fixed point (a > 0)
BS_HD int64_t uf_log2_q16_up(UF a) {
  // a <= m 2^e with m in [2^31, 2^32): log2 = e + 31 + log2(m / 2^31)
  uint32_t y = a.m;  // Q31 value in [1, 2)
  int32_t frac = 0;
  for (int i = 0; i < 16; ++i) {
    uint64_t sq = (uint64_t)y * y;  // Q62 in [1, 4)
    frac <<= 1;
    if (sq >> 63) {  // >= 2
      frac |= 1;
      uint64_t t = sq >> 32;
      if (sq & 0xffffffffull) t += 1;
      if (t >> 32) t = 0xffffffffull;  // stays an upper bound of y, < 2
      y = (uint32_t)t;
    } else {
      uint64_t t = sq >> 31;
      if (sq & 0x7fffffffull) t += 1;
      if (t >> 32) {  // rounded up to exactly 2: treat as the >= 2 branch next time
        t = 0xffffffffull;
      }
      y = (uint32_t)t;
    }
  }
  return (int64_t)(a.e + 31) * 65536 + frac + 1;
}

// floor-ish lower bound of log2(p) in Q16 for 2^30 < p < 2^31 (host)
inline int64_t log2_q16_down_u31(uint32_t p) {
  uint32_t y = p << 1;  // Q31 in [1, 2)
  int32_t frac = 0;
  for (int i = 0; i < 16; ++i) {
    uint64_t sq = (uint64_t)y * y;
    frac <<= 1;
    if (sq >> 63) {
      frac |= 1;
      y = (uint32_t)(sq >> 32);
    } else {
      y = (uint32_t)(sq >> 31);
    }
  }
  return (int64_t)30 * 65536 + frac;
}

// ------------------------------------------------------------------------------------
// coefficient access
// ------------------------------------------------------------------------------------
struct Grid {
  const uint32_t* c;
  int32_t dx, dy, L;
};

// pointer to the limbs of the coefficient with power e of the eliminated variable and
// power o of the other variable (var = 1: eliminate y, so e = j, o = i)
BS_HD const uint32_t* coef_ptr(const Grid& g, int var, int e, int o) {
  int i = var ? o : e;
  int j = var ? e : o;
  return g.c + ((int64_t)j * (g.dx + 1) + i) * g.L;
}
BS_HD int ext_e(const Grid& g, int var) { return var ? g.dy : g.dx; }
BS_HD int ext_o(const Grid& g, int var) { return var ? g.dx : g.dy; }

// magnitude of a two's complement multi-limb integer as an upper float; nonzero flag;
// bit length of the magnitude
BS_HD UF mag_uf(const uint32_t* c, int L, bool* nonzero, int* bits) {
  bool neg = (c[L - 1] >> 31) != 0;
  // walk limbs from the bottom, negating on the fly when negative
  uint32_t carry = 1;
  int top = -1;
  uint32_t v1 = 0, v0 = 0;  // magnitude limbs at top and top-1
  bool sticky = false;      // any nonzero limb below top-1
  for (int l = 0; l < L; ++l) {
    uint32_t x = c[l];
    if (neg) {
      uint32_t nx = ~x + carry;
      carry = (carry && nx == 0) ? 1u : 0u;
      x = nx;
    }
    if (x) {
      // limbs strictly between old top and l are zero
      if (top >= 0) {
        if (top == l - 1) {
          sticky = sticky || (v0 != 0);
          v0 = v1;
        } else {
          sticky = sticky || (v0 != 0) || (v1 != 0);
          v0 = 0;
        }
      }
      v1 = x;
      top = l;
    }
  }
  if (top < 0) {
    *nonzero = false;
    *bits = 0;
    return UF{0u, 0};
  }
  *nonzero = true;
  *bits = 32 * top + (32 - clz32(v1));
  if (top == 0) return uf_make((uint64_t)v1, 0, false);
  return uf_make(((uint64_t)v1 << 32) | v0, 32 * (top - 1), sticky);
}

// per-row statistics of row e (eliminated-variable power e)
struct RowStat {
  UF l1;          // >= sum_o |coef|
  int32_t max_o;  // highest o with a nonzero coefficient, -1 if the row is zero
  int32_t min_bits;  // bit length of the smallest nonzero magnitude (0 if zero row)
};

BS_HD RowStat row_stat(const Grid& g, int var, int e) {
  RowStat s{UF{0u, 0}, -1, 0};
  int eo = ext_o(g, var);
  for (int o = 0; o <= eo; ++o) {
    bool nz;
    int bits;
    UF u = mag_uf(coef_ptr(g, var, e, o), g.L, &nz, &bits);
    if (nz) {
      s.l1 = uf_add(s.l1, u);
      s.max_o = o;
      if (s.min_bits == 0 || bits < s.min_bits) s.min_bits = bits;
    }
  }
  return s;
}

// the plan of one job
struct Plan {
  int32_t status;     // BS_OK or an error code
  int32_t trivial;    // 0 general, 1 result is the zero polynomial, 2 result is 1
  int32_t me, ne;     // degrees of f and g in the eliminated variable
  int32_t D;          // degree bound of the result (-1 for the zero polynomial)
  int32_t logN, N;    // transform size (N >= D + 1)
  int32_t k_need;     // primes needed: prod p > 4B
  int32_t k_total;    // primes evaluated (k_need plus spares)
  int32_t out_limbs;  // limbs that hold every coefficient (two's complement)
  int64_t log2B_q16;  // upper bound of log2 B in Q16
};

// assemble the plan from per-polynomial summaries.
//   S*: sum over rows of l1^2 (upper float); m*: degree in eliminated var (-1: zero poly)
//   tdeg*: total degree; dego*: degree in the other variable; lcbits*: min nonzero
//   magnitude bits of the leading row.  plan_head() fills everything but the prime
//   count and returns the Q16 amount of log2(prod p) needed in *need (or a status);
//   plan_tail() completes it from k_need with a conservative spare count (the exact one,
//   exact_prime_total() below, needs the coefficients).  plan_head_logs() takes the
//   logarithms lf = log2 Sf, lg = log2 Sg (Q16, rounded up; 0 for 0) already computed.
BS_HD Plan plan_head_logs(int64_t lf, int mf, int tdf, int dof, int64_t lg, int mg, int tdg, int dog,
                          int64_t* need) {
  Plan P;
  P.status = 0;
  P.trivial = 0;
  P.me = mf;
  P.ne = mg;
  P.D = -1;
  P.logN = 0;
  P.N = 1;
  P.k_need = 0;
  P.k_total = 0;
  P.out_limbs = 1;
  P.log2B_q16 = 0;
  *need = 0;
  if (mf < 0 || mg < 0) {
    P.trivial = 1;
    return P;
  }
  if (mf == 0 && mg == 0) {
    P.trivial = 2;
    P.D = 0;
    return P;
  }
  int64_t d1 = (int64_t)tdf * tdg;
  int64_t d2 = (int64_t)mg * dof + (int64_t)mf * dog;
  int64_t D = d1 < d2 ? d1 : d2;
  if (D + 1 > kNMax) {
    P.status = 7;  // BS_ERR_RANGE
    return P;
  }
  P.D = (int32_t)D;
  int logN = 0;
  while ((1ll << logN) < D + 1) ++logN;
  P.logN = logN;
  P.N = 1 << logN;
  int64_t l2b = ((int64_t)mg * lf + (int64_t)mf * lg + 1) / 2 + 1;  // Q16, rounded up
  if (l2b < 0) l2b = 0;
  P.log2B_q16 = l2b;
  *need = l2b + 2 * 65536;  // prod p > 4B
  return P;
}

BS_HD Plan plan_head(UF Sf, int mf, int tdf, int dof, UF Sg, int mg, int tdg, int dog,
                     int64_t* need) {
  return plan_head_logs(Sf.m ? uf_log2_q16_up(Sf) : 0, mf, tdf, dof, Sg.m ? uf_log2_q16_up(Sg) : 0,
                        mg, tdg, dog, need);
}

BS_HD void plan_tail(Plan& P, int k_need, int lcbf, int lcbg, int table_size,
                     bool lc_monomials = false) {
  P.k_need = k_need < 1 ? 1 : k_need;
  // a prime p > 2^30 can divide every coefficient of a leading row only if it divides
  // the smallest one: at most (bits - 1) / 30 such primes; two more cover evaluation
  // sets that happen to contain a root of a leading coefficient (none needed when both
  // leading rows are monomials: c x^k never vanishes on a coset, which avoids 0)
  int spare = (lcbf > 0 ? (lcbf - 1) / 30 : 0) + (lcbg > 0 ? (lcbg - 1) / 30 : 0) +
              (lc_monomials ? 0 : 2);
  P.k_total = P.k_need + spare;
  if (P.k_total > table_size) {
    P.status = 7;
    return;
  }
  int64_t bits = (P.log2B_q16 + 65535) / 65536 + 2;
  P.out_limbs = (int32_t)((bits + 31) / 32);
}

// smallest k with lg_prefix[k] >= need (host: binary search)
inline int prime_count_host(const int64_t* lg_prefix, int table_size, int64_t need) {
  int lo = 0, hi = table_size;
  while (lo < hi) {
    int mid = (lo + hi) / 2;
    if (lg_prefix[mid] >= need)
      hi = mid;
    else
      lo = mid + 1;
  }
  return lo;
}

BS_HD Plan finish_plan(UF Sf, int mf, int tdf, int dof, int lcbf, UF Sg, int mg, int tdg,
                       int dog, int lcbg, const int64_t* lg_prefix, int table_size) {
  int64_t need;
  Plan P = plan_head(Sf, mf, tdf, dof, Sg, mg, tdg, dog, &need);
  if (P.status || P.trivial) return P;
  if (lg_prefix[table_size] < need) {
    P.status = 7;
    return P;
  }
  int lo = 0, hi = table_size;
  while (lo < hi) {
    int mid = (lo + hi) / 2;
    if (lg_prefix[mid] >= need)
      hi = mid;
    else
      lo = mid + 1;
  }
  plan_tail(P, lo, lcbf, lcbg, table_size);
  return P;
}

// |c| mod p of a two's complement coefficient of L limbs (host)
inline uint32_t host_residue(const uint32_t* c, int L, uint32_t p) {
  uint64_t acc = 0;
  for (int l = L - 1; l >= 0; --l) acc = ((acc << 32) | c[l]) % p;
  if (c[L - 1] >> 31) {  // value = raw - 2^(32 L)
    uint64_t t = 1;
    for (int l = 0; l < L; ++l) t = (t << 32) % p;
    acc = (acc + p - t) % p;
  }
  return (uint32_t)acc;
}

// Spare primes, exactly: a prime is rejected for a whole job when a leading row vanishes
// identically mod p, which needs p to divide that row's smallest coefficient (cf, cg);
// an evaluation point hits a root of a leading coefficient only when the row has more
// than one nonzero coefficient (a monomial c x^k never vanishes on the coset, which
// avoids 0), and then two more primes cover such hits.  The smallest K such that
// [0, K) holds k_need + coset primes dividing neither cf nor cg is returned; is_div(q)
// tells whether table prime q divides cf or cg.
template <class IsDiv>
BS_HD int exact_prime_total(int k_need, bool lc_monomials, int table_size, IsDiv is_div) {
  const int want = k_need + (lc_monomials ? 0 : 2);
  int K = want, d = 0, counted = 0;
  while (true) {
    for (; counted < K && counted < table_size; ++counted) d += is_div(counted) ? 1 : 0;
    if (K - d >= want || K >= table_size) return K < table_size ? K : table_size;
    K = want + d;
  }
}

// upper float of the exact value hi 2^64 + lo
BS_HD UF uf_from_u128(uint64_t hi, uint64_t lo) {
  if (!hi) return uf_make(lo, 0, false);
  const int sh = 64 - clz64(hi);  // keep the top 64 bits, round up by the rest
  const uint64_t top = (hi << (64 - sh)) | (lo >> sh);
  const bool sticky = (lo << (64 - sh)) != 0;
  return uf_make(top, sh, sticky);
}

// |c| of a two's complement coefficient of one or two limbs
BS_HD uint64_t mag_narrow(const uint32_t* c, int L) {
  if (L == 1) {
    const int64_t v = (int32_t)c[0];
    return (uint64_t)(v < 0 ? -v : v);
  }
  const uint64_t raw = ((uint64_t)c[1] << 32) | c[0];
  return (raw >> 63) ? ~raw + 1 : raw;  // |INT64_MIN| = 2^63 is representable
}

// row statistics for coefficients of at most two limbs (host): the magnitudes are summed
// exactly in 128 bits and rounded up to an upper float once per row
inline RowStat row_stat_narrow(const Grid& g, int var, int e) {
  RowStat s{UF{0u, 0}, -1, 0};
  unsigned __int128 sum = 0;
  const int eo = ext_o(g, var);
  for (int o = 0; o <= eo; ++o) {
    const uint64_t mag = mag_narrow(coef_ptr(g, var, e, o), g.L);
    if (!mag) continue;
    sum += mag;
    s.max_o = o;
    const int bits = 64 - clz64(mag);
    if (s.min_bits == 0 || bits < s.min_bits) s.min_bits = bits;
  }
  s.l1 = uf_from_u128((uint64_t)(sum >> 64), (uint64_t)sum);
  return s;
}

// host version: scan both grids
inline Plan plan_host(const Grid& f, const Grid& g, int var, const int64_t* lg_prefix,
                      int table_size, const uint32_t* primes = nullptr) {
  auto summarise = [&](const Grid& h, UF* S, int* m, int* td, int* dego, int* lcb) {
    *S = UF{0u, 0};
    *m = -1;
    *td = -1;
    *dego = -1;
    *lcb = 0;
    int ee = ext_e(h, var);
    for (int e = 0; e <= ee; ++e) {
      RowStat rs = h.L <= 2 ? row_stat_narrow(h, var, e) : row_stat(h, var, e);
      if (rs.max_o < 0) continue;
      *S = uf_add(*S, uf_mul(rs.l1, rs.l1));
      *m = e;
      *lcb = rs.min_bits;
      if (e + rs.max_o > *td) *td = e + rs.max_o;
      if (rs.max_o > *dego) *dego = rs.max_o;
    }
  };
  UF Sf, Sg;
  int mf, tf, df, lf, mg, tg, dg, lgb;
  summarise(f, &Sf, &mf, &tf, &df, &lf);
  summarise(g, &Sg, &mg, &tg, &dg, &lgb);
  Plan P = finish_plan(Sf, mf, tf, df, lf, Sg, mg, tg, dg, lgb, lg_prefix, table_size);
  if (!primes || P.status || P.trivial) return P;
  // leading rows: smallest nonzero coefficient and number of nonzero coefficients
  auto lead = [&](const Grid& h, int m, int* nnz) {
    const uint32_t* best = nullptr;
    int bb = 0;
    *nnz = 0;
    for (int o = 0; o <= ext_o(h, var); ++o) {
      bool nz;
      int bits;
      mag_uf(coef_ptr(h, var, m, o), h.L, &nz, &bits);
      if (!nz) continue;
      ++*nnz;
      if (!best || bits < bb) {
        best = coef_ptr(h, var, m, o);
        bb = bits;
      }
    }
    return best;
  };
  int nf, ng;
  const uint32_t* cf = lead(f, mf, &nf);
  const uint32_t* cg = lead(g, mg, &ng);
  const int K = exact_prime_total(P.k_need, nf == 1 && ng == 1, table_size, [&](int q) {
    return host_residue(cf, f.L, primes[q]) == 0 || host_residue(cg, g.L, primes[q]) == 0;
  });
  if (K < P.k_total) P.k_total = K;  // never above the conservative count
  return P;
}

}  // namespace bs
