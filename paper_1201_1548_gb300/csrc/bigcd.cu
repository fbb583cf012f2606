// The gcd of two bivariate polynomials in Z[x][y] and Teissier's Q exactly (Sec. 3.3,
// computation of n_alpha^+: h = gcd(f_x, f_y), f_x* = f_x / h, f_y* = f_y / h and
// Q = res(f_x*, f_y*; y)).
//
// gcd.  With d the index of the first principal subresultant coefficient of A and B that
// is not identically zero, d = deg_y gcd(A, B) and the subresultant polynomial S_d(A, B) is
// a multiple of the gcd over Q(x) (its leading coefficient is sr_d).  By Gauss's lemma
//   gcd(A, B) = gcd(cont A, cont B) * pp(S_d),
// cont the gcd in Z[x] of the rows, pp the rows divided by their content, normalised to a
// positive leading coefficient.  If every sr_i vanishes, the polynomial of smaller degree
// divides the other over Q(x) and takes the place of S_d.  Every step runs on the device:
// the psc sequence and S_d on the resultant's modular engine (psc.cu), contents and exact
// quotients on the modular gcd engine, products of polynomials by k_zmul.
//
// Q.  For A = G A*, B = G B* with deg G = d and formal degrees m, n,
//   sr_d(A, B) = lc(G)^(m + n - 2d) res(A*, B*)
// (the cofactor property of subresultants, checked at every point where no leading
// coefficient vanishes, hence an identity in Z[x]); so Q = sr_d(f_x, f_y) / lc_y(h)^e with
// e = m + n - 2d, one exact quotient.  If every sr_i vanishes, the cofactor of the smaller
// polynomial is free of y and Q is its power (m - d or n - d).
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <vector>

#include "ctx.cuh"
#include "modpoly.cuh"
#include "owned.cuh"

namespace bs {

constexpr int kZmulMaxLimbs = 320;  // limbs of a product coefficient of k_zmul

// c = a b in Z[x], two's complement limbs; one thread per coefficient of c.  The positive
// and the negative partial products are summed apart (magnitudes) and subtracted at the end.
__global__ void k_zmul(const uint32_t* a, int da, int La, const uint32_t* b, int db, int Lb, uint32_t* c,
                       int Lc) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k > da + db) return;
  uint32_t pos[kZmulMaxLimbs], neg[kZmulMaxLimbs], ma[kZmulMaxLimbs / 2], mb[kZmulMaxLimbs / 2];
  for (int l = 0; l < Lc; ++l) pos[l] = neg[l] = 0u;
  const int i0 = k - db > 0 ? k - db : 0, i1 = k < da ? k : da;
  for (int i = i0; i <= i1; ++i) {
    const uint32_t* x = a + (size_t)i * La;
    const uint32_t* y = b + (size_t)(k - i) * Lb;
    const bool nx = x[La - 1] >> 31, ny = y[Lb - 1] >> 31;
    uint64_t cx = 1, cy = 1;  // two's complement negation: invert and add one
    for (int l = 0; l < La; ++l) {
      if (nx) {
        cx += (uint32_t)~x[l];
        ma[l] = (uint32_t)cx;
        cx >>= 32;
      } else {
        ma[l] = x[l];
      }
    }
    for (int l = 0; l < Lb; ++l) {
      if (ny) {
        cy += (uint32_t)~y[l];
        mb[l] = (uint32_t)cy;
        cy >>= 32;
      } else {
        mb[l] = y[l];
      }
    }
    uint32_t* acc = (nx != ny) ? neg : pos;
    for (int u = 0; u < La; ++u) {
      if (ma[u] == 0u) continue;
      uint64_t carry = 0;
      int v = 0;
      for (; v < Lb; ++v) {
        const uint64_t t = (uint64_t)ma[u] * mb[v] + acc[u + v] + carry;
        acc[u + v] = (uint32_t)t;
        carry = t >> 32;
      }
      for (int w = u + v; carry && w < Lc; ++w) {
        const uint64_t t = (uint64_t)acc[w] + carry;
        acc[w] = (uint32_t)t;
        carry = t >> 32;
      }
    }
  }
  uint64_t borrow = 0;
  uint32_t* out = c + (size_t)k * Lc;
  for (int l = 0; l < Lc; ++l) {
    const uint64_t t = (uint64_t)pos[l] - neg[l] - borrow;
    out[l] = (uint32_t)t;
    borrow = (t >> 63) & 1u;
  }
}

// the trimmed degree of an owned polynomial (-1 for zero)
static int owned_degree(const HostPoly& h) { return trimmed_degree(h.u); }

static bool is_one(const HostPoly& h) {
  if (owned_degree(h) != 0) return false;
  const uint32_t* c = h.u.c;
  if (c[0] != 1u) return false;
  for (int l = 1; l < h.u.limbs; ++l)
    if (c[l]) return false;
  return true;
}

// a b in Z[x] on the device (k_zmul), into an owned polynomial
static int zmul_owned(bs_ctx* ctx, const bs_upoly& a, const bs_upoly& b, HostPoly* out) {
  const int da = trimmed_degree(a), db = trimmed_degree(b);
  if (da < 0 || db < 0) {
    out->c.assign(1, 0u);
    out->u = bs_upoly{-1, 1, out->c.data()};
    return BS_OK;
  }
  const int steps = da < db ? da + 1 : db + 1;  // terms of one coefficient
  int tb = 0;
  while ((1 << tb) < steps) ++tb;
  const int Lc = a.limbs + b.limbs + (tb + 31) / 32 + 1;
  if (Lc > kZmulMaxLimbs || a.limbs > kZmulMaxLimbs / 2 || b.limbs > kZmulMaxLimbs / 2)
    return ctx_fail(ctx, BS_ERR_RANGE, "product coefficients above 10240 bits");
  cudaSetDevice(ctx->device);
  Layout lay;
  const size_t o_a = lay.take(sizeof(uint32_t) * (size_t)(da + 1) * a.limbs);
  const size_t o_b = lay.take(sizeof(uint32_t) * (size_t)(db + 1) * b.limbs);
  const size_t o_c = lay.take(sizeof(uint32_t) * (size_t)(da + db + 1) * Lc);
  int rc = ensure_workspace(ctx, lay.used);
  if (rc) return rc;
  char* base = (char*)ctx->ws;
  cudaStream_t s = ctx->stream;
  rc = ctx_cuda(ctx, cudaMemcpyAsync(base + o_a, a.c, sizeof(uint32_t) * (size_t)(da + 1) * a.limbs,
                                     cudaMemcpyHostToDevice, s), "h2d");
  if (!rc)
    rc = ctx_cuda(ctx, cudaMemcpyAsync(base + o_b, b.c, sizeof(uint32_t) * (size_t)(db + 1) * b.limbs,
                                       cudaMemcpyHostToDevice, s), "h2d");
  if (rc) return rc;
  const int n = da + db + 1, th = 64;
  k_zmul<<<(n + th - 1) / th, th, 0, s>>>((const uint32_t*)(base + o_a), da, a.limbs,
                                          (const uint32_t*)(base + o_b), db, b.limbs, (uint32_t*)(base + o_c), Lc);
  rc = ctx_cuda(ctx, cudaGetLastError(), "launch");
  if (rc) return rc;
  out->c.assign((size_t)n * Lc, 0u);
  rc = ctx_cuda(ctx, cudaMemcpyAsync(out->c.data(), base + o_c, sizeof(uint32_t) * out->c.size(),
                                     cudaMemcpyDeviceToHost, s), "d2h");
  if (rc) return rc;
  rc = ctx_cuda(ctx, cudaStreamSynchronize(s), "stream");
  if (rc) return rc;
  out->u = bs_upoly{n - 1, Lc, out->c.data()};
  return BS_OK;
}

// a^e in Z[x] by repeated squaring (e >= 0)
static int zpow_owned(bs_ctx* ctx, const bs_upoly& a, int e, HostPoly* out) {
  HostPoly r, sq;
  r.c.assign(1, 1u);
  r.u = bs_upoly{0, 1, r.c.data()};
  sq.c.assign(a.c, a.c + (size_t)(std::max(a.deg, 0) + 1) * a.limbs);
  sq.u = bs_upoly{a.deg, a.limbs, sq.c.data()};
  while (e > 0) {
    int rc;
    if (e & 1) {
      HostPoly t;
      rc = zmul_owned(ctx, r.u, sq.u, &t);
      if (rc) return rc;
      r = std::move(t);
      r.u.c = r.c.data();
    }
    e >>= 1;
    if (e) {
      HostPoly t;
      rc = zmul_owned(ctx, sq.u, sq.u, &t);
      if (rc) return rc;
      sq = std::move(t);
      sq.u.c = sq.c.data();
    }
  }
  *out = std::move(r);
  out->u.c = out->c.data();
  return BS_OK;
}

// rows of a grid with respect to the eliminated variable, copied (trailing zero rows kept)
static void grid_rows(const bs_bipoly& f, int var, std::vector<HostPoly>* rows) {
  const int ne = var ? f.deg_y : f.deg_x, no = var ? f.deg_x : f.deg_y;
  const int L = f.limbs;
  rows->assign(ne + 1, HostPoly{});
  for (int e = 0; e <= ne; ++e) {
    HostPoly& r = (*rows)[e];
    r.c.assign((size_t)(no + 1) * L, 0u);
    for (int o = 0; o <= no; ++o) {
      const int j = var ? e : o, i = var ? o : e;
      std::memcpy(r.c.data() + (size_t)o * L, f.c + ((size_t)j * (f.deg_x + 1) + i) * L, sizeof(uint32_t) * L);
    }
    r.u = bs_upoly{no, L, r.c.data()};
  }
}

// a grid with rows as the powers of y (var = 1 layout) from owned rows
static void rows_grid(const std::vector<HostPoly>& rows, std::vector<uint32_t>* buf, bs_bipoly* out) {
  int dx = 0, L = 1;
  for (const auto& r : rows) {
    dx = std::max(dx, std::max(owned_degree(r), 0));
    L = std::max(L, r.u.limbs);
  }
  const int dy = (int)rows.size() - 1;
  buf->assign((size_t)(dy + 1) * (dx + 1) * L, 0u);
  for (int j = 0; j <= dy; ++j) {
    const HostPoly& r = rows[j];
    const int dr = owned_degree(r);
    for (int i = 0; i <= dr; ++i) {
      const uint32_t* s = r.u.c + (size_t)i * r.u.limbs;
      uint32_t* d = buf->data() + ((size_t)j * (dx + 1) + i) * L;
      const uint32_t ext = (s[r.u.limbs - 1] >> 31) ? 0xffffffffu : 0u;
      for (int l = 0; l < L; ++l) d[l] = l < r.u.limbs ? s[l] : ext;
    }
  }
  *out = bs_bipoly{dx, dy, L, buf->data()};
}

static void negate_owned(HostPoly* h) {
  const int d = std::max(h->u.deg, 0);
  for (int i = 0; i <= d; ++i) {
    uint32_t* c = h->u.c + (size_t)i * h->u.limbs;
    uint64_t carry = 1;
    for (int l = 0; l < h->u.limbs; ++l) {
      carry += (uint32_t)~c[l];
      c[l] = (uint32_t)carry;
      carry >>= 32;
    }
  }
}

// content (gcd of the rows in Z[x], positive leading coefficient) and the rows divided by it
static int content_owned(bs_ctx* ctx, const bs_bipoly& f, int var, HostPoly* cont, std::vector<HostPoly>* pp) {
  int32_t nrows = 0;
  bs_upoly hq{0, 0, nullptr};
  const int ne = var ? f.deg_y : f.deg_x;
  std::vector<bs_upoly> rq(ne + 1, bs_upoly{0, 0, nullptr});
  int rc = bs_content(ctx, &f, var, &hq, pp ? ne + 1 : 0, pp ? rq.data() : nullptr, &nrows);
  if (rc) return rc;
  cont->c.assign((size_t)(std::max(hq.deg, 0) + 1) * std::max(hq.limbs, 1), 0u);
  cont->u = bs_upoly{std::max(hq.deg, 0), std::max(hq.limbs, 1), cont->c.data()};
  if (pp) {
    pp->assign(nrows, HostPoly{});
    for (int e = 0; e < nrows; ++e) {
      (*pp)[e].c.assign((size_t)(std::max(rq[e].deg, 0) + 1) * std::max(rq[e].limbs, 1), 0u);
      rq[e] = bs_upoly{std::max(rq[e].deg, 0), std::max(rq[e].limbs, 1), (*pp)[e].c.data()};
    }
  }
  rc = bs_content(ctx, &f, var, &cont->u, pp ? nrows : 0, pp ? rq.data() : nullptr, &nrows);
  if (rc) return rc;
  if (pp)
    for (int e = 0; e < nrows; ++e) {
      (*pp)[e].u = rq[e];
      (*pp)[e].u.c = (*pp)[e].c.data();
    }
  return BS_OK;
}

static int gcd_z_owned(bs_ctx* ctx, const bs_upoly& a, const bs_upoly& b, HostPoly* out) {
  std::vector<HostPoly> o;
  int rc = modgcd_owned(ctx, {0}, {a}, {b}, &o);
  if (rc) return rc;
  *out = std::move(o[0]);
  out->u.c = out->c.data();
  return BS_OK;
}

static int divide_owned(bs_ctx* ctx, const bs_upoly& a, const bs_upoly& b, HostPoly* out) {
  std::vector<HostPoly> o;
  bs_upoly at = a;
  at.deg = trimmed_degree(a);
  int rc = modgcd_owned(ctx, {2}, {at}, {b}, &o);
  if (rc) return rc;
  *out = std::move(o[0]);
  out->u.c = out->c.data();
  return BS_OK;
}

// the exact psc sequence of (a, b) as owned host polynomials
static int psc_seq_owned(bs_ctx* ctx, const bs_bipoly& a, const bs_bipoly& b, int var, std::vector<HostPoly>* out) {
  int32_t q = 0;
  int rc = bs_psc(ctx, &a, &b, var, 0, &q, nullptr);
  if (rc) return rc;
  out->assign(q, HostPoly{});
  if (q == 0) return BS_OK;
  std::vector<bs_upoly> sr(q, bs_upoly{0, 0, nullptr});
  rc = bs_psc(ctx, &a, &b, var, q, &q, sr.data());
  if (rc) return rc;
  for (int i = 0; i < q; ++i) {
    (*out)[i].c.assign((size_t)(std::max(sr[i].deg, 0) + 1) * sr[i].limbs, 0u);
    sr[i].c = (*out)[i].c.data();
  }
  rc = bs_psc(ctx, &a, &b, var, q, &q, sr.data());
  if (rc) return rc;
  for (int i = 0; i < q; ++i) {
    (*out)[i].u = sr[i];
    (*out)[i].u.c = (*out)[i].c.data();
  }
  return BS_OK;
}

static int sres_owned(bs_ctx* ctx, const bs_bipoly& a, const bs_bipoly& b, int var, int d, std::vector<HostPoly>* out) {
  int32_t n = 0;
  int rc = bs_subresultant(ctx, &a, &b, var, d, 0, &n, nullptr);
  if (rc) return rc;
  std::vector<bs_upoly> s(n, bs_upoly{0, 0, nullptr});
  rc = bs_subresultant(ctx, &a, &b, var, d, n, &n, s.data());
  if (rc) return rc;
  out->assign(n, HostPoly{});
  for (int j = 0; j < n; ++j) {
    (*out)[j].c.assign((size_t)(std::max(s[j].deg, 0) + 1) * s[j].limbs, 0u);
    s[j].c = (*out)[j].c.data();
  }
  rc = bs_subresultant(ctx, &a, &b, var, d, n, &n, s.data());
  if (rc) return rc;
  for (int j = 0; j < n; ++j) {
    (*out)[j].u = s[j];
    (*out)[j].u.c = (*out)[j].c.data();
  }
  return BS_OK;
}

// degree of a grid in the eliminated variable (-1 for the zero polynomial)
static int elim_degree(const bs_bipoly& f, int var) {
  const int ne = var ? f.deg_y : f.deg_x, no = var ? f.deg_x : f.deg_y;
  for (int e = ne; e >= 0; --e)
    for (int o = 0; o <= no; ++o) {
      const int j = var ? e : o, i = var ? o : e;
      if (!limbs_zero(f.c + ((size_t)j * (f.deg_x + 1) + i) * f.limbs, f.limbs)) return e;
    }
  return -1;
}

struct BiGcd {
  std::vector<HostPoly> rows;  // h by powers of the eliminated variable
  int d = 0;                   // deg h in the eliminated variable
  bool all_vanish = false;     // every sr_i vanished (the smaller polynomial divides the other)
  int small = 0;               // then: 0 if A is the smaller, 1 if B
  std::vector<HostPoly> sr;    // the psc sequence of (A, B)
  HostPoly c;                  // gcd of the contents
  int ma = -1, mb = -1;        // degrees of A and B in the eliminated variable
};

static int bigcd(bs_ctx* ctx, const bs_bipoly& A, const bs_bipoly& B, int var, BiGcd* G) {
  G->ma = elim_degree(A, var);
  G->mb = elim_degree(B, var);
  if (G->ma < 0 && G->mb < 0) return BS_OK;  // gcd(0, 0) = 0: no rows
  int rc;
  if (G->ma < 0 || G->mb < 0) {  // gcd(0, B) = B with a positive leading coefficient
    std::vector<HostPoly> r;
    grid_rows(G->ma < 0 ? B : A, var, &r);
    const int top = G->ma < 0 ? G->mb : G->ma;
    r.resize(top + 1);
    const HostPoly& lr = r[top];
    const int dl = owned_degree(lr);
    if (lr.u.c[(size_t)dl * lr.u.limbs + lr.u.limbs - 1] >> 31)
      for (auto& x : r) negate_owned(&x);
    G->rows = std::move(r);
    for (auto& x : G->rows) x.u.c = x.c.data();
    G->d = top;
    return BS_OK;
  }
  HostPoly ca, cb;
  rc = content_owned(ctx, A, var, &ca, nullptr);
  if (!rc) rc = content_owned(ctx, B, var, &cb, nullptr);
  if (!rc) rc = gcd_z_owned(ctx, ca.u, cb.u, &G->c);
  if (rc) return rc;
  rc = psc_seq_owned(ctx, A, B, var, &G->sr);
  if (rc) return rc;
  const int q = (int)G->sr.size();
  int d = 0;
  while (d < q && owned_degree(G->sr[d]) < 0) ++d;
  G->d = d;
  std::vector<HostPoly> P;  // pp(S_d) by powers of the eliminated variable
  if (std::min(G->ma, G->mb) == 0 || d == 0) {
    P.assign(1, HostPoly{});
    P[0].c.assign(1, 1u);
    P[0].u = bs_upoly{0, 1, P[0].c.data()};
    G->d = 0;
  } else {
    std::vector<uint32_t> sbuf;
    bs_bipoly S;
    int svar = var;
    std::vector<HostPoly> srows;
    if (d == q) {  // the smaller polynomial divides the other over Q(x)
      G->all_vanish = true;
      G->small = G->ma <= G->mb ? 0 : 1;
      S = G->small == 0 ? A : B;
    } else {
      rc = sres_owned(ctx, A, B, var, d, &srows);
      if (rc) return rc;
      rows_grid(srows, &sbuf, &S);
      svar = 1;
    }
    HostPoly cs;
    rc = content_owned(ctx, S, svar, &cs, &P);
    if (rc) return rc;
    P.resize(d + 1);
    const HostPoly& lr = P[d];
    const int dl = owned_degree(lr);
    if (dl >= 0 && (lr.u.c[(size_t)dl * lr.u.limbs + lr.u.limbs - 1] >> 31))
      for (auto& x : P) negate_owned(&x);
  }
  if (is_one(G->c)) {
    G->rows = std::move(P);
  } else {
    G->rows.assign(P.size(), HostPoly{});
    for (size_t j = 0; j < P.size(); ++j) {
      rc = zmul_owned(ctx, P[j].u, G->c.u, &G->rows[j]);
      if (rc) return rc;
    }
  }
  for (auto& x : G->rows) x.u.c = x.c.data();
  return BS_OK;
}

// copy owned rows into caller outputs (a size query writes bounds only)
static int put_rows(bs_ctx* ctx, const std::vector<HostPoly>& rows, int cap, bs_upoly* out, int32_t* n) {
  *n = (int32_t)rows.size();
  if (!out || cap == 0) return BS_OK;
  const bool query = !out[0].c;
  if (!query && cap < (int)rows.size()) return ctx_fail(ctx, BS_ERR_CAPACITY, "fewer rows than the gcd has");
  for (int j = 0; j < std::min(cap, (int)rows.size()); ++j) {
    const int dj = owned_degree(rows[j]);
    if (query) {
      out[j].deg = std::max(dj, 0);
      out[j].limbs = rows[j].u.limbs;
      continue;
    }
    if (dj < 0) {
      for (int c = 0; c <= out[j].deg; ++c) std::memset(out[j].c + (size_t)c * out[j].limbs, 0, sizeof(uint32_t) * out[j].limbs);
      out[j].deg = -1;
      continue;
    }
    const int rc = put_result(ctx, rows[j].u.c, rows[j].u.limbs, dj, out + j);
    if (rc) return rc;
    out[j].deg = dj;
  }
  return BS_OK;
}

static int check_bipoly(bs_ctx* ctx, const bs_bipoly* p) {
  if (!p || p->deg_x < 0 || p->deg_y < 0 || p->limbs < 1 || p->limbs > kMaxLimbs || !p->c)
    return ctx_fail(ctx, BS_ERR_ARG, "bad bivariate polynomial");
  return 0;
}

// f_x (dv = 0) or f_y (dv = 1) with one more limb per coefficient
static void derivative_grid(const bs_bipoly& f, int dv, std::vector<uint32_t>* buf, bs_bipoly* out) {
  const int L = f.limbs, L1 = L + 1;
  const int dx = dv ? f.deg_x : std::max(f.deg_x - 1, 0);
  const int dy = dv ? std::max(f.deg_y - 1, 0) : f.deg_y;
  buf->assign((size_t)(dx + 1) * (dy + 1) * L1, 0u);
  for (int j = 0; j <= dy; ++j)
    for (int i = 0; i <= dx; ++i) {
      const int sj = dv ? j + 1 : j, si = dv ? i : i + 1;
      const uint32_t k = (uint32_t)(dv ? sj : si);
      if (sj > f.deg_y || si > f.deg_x) continue;
      const uint32_t* s = f.c + ((size_t)sj * (f.deg_x + 1) + si) * L;
      uint32_t* d = buf->data() + ((size_t)j * (dx + 1) + i) * L1;
      const uint32_t ext = (s[L - 1] >> 31) ? 0xffffffffu : 0u;
      uint64_t carry = 0;
      for (int l = 0; l < L1; ++l) {
        const uint64_t x = (uint64_t)(l < L ? s[l] : ext) * k + carry;
        d[l] = (uint32_t)x;
        carry = x >> 32;
      }
    }
  *out = bs_bipoly{dx, dy, L1, buf->data()};
}

}  // namespace bs

using namespace bs;

extern "C" int bs_gcd_bivariate(bs_ctx* ctx, const bs_bipoly* f, const bs_bipoly* g, int var, int cap_rows,
                                bs_upoly* rows, int32_t* nrows) {
  if (!ctx) return BS_ERR_ARG;
  if (!nrows || (var != 0 && var != 1) || cap_rows < 0 || (cap_rows > 0 && !rows))
    return ctx_fail(ctx, BS_ERR_ARG, "bad arguments");
  if (ctx->server) return ctx_fail(ctx, BS_ERR_ARG, "the context runs a serving loop");
  int rc = check_bipoly(ctx, f);
  if (!rc) rc = check_bipoly(ctx, g);
  if (rc) return rc;
  BiGcd G;
  rc = bigcd(ctx, *f, *g, var, &G);
  if (rc) return rc;
  return put_rows(ctx, G.rows, cap_rows, rows, nrows);
}

extern "C" int bs_teissier_q(bs_ctx* ctx, const bs_bipoly* f, int var, bs_upoly* Q, int32_t* d) {
  if (!ctx) return BS_ERR_ARG;
  if (!f || !Q || !d || (var != 0 && var != 1)) return ctx_fail(ctx, BS_ERR_ARG, "bad arguments");
  if (ctx->server) return ctx_fail(ctx, BS_ERR_ARG, "the context runs a serving loop");
  int rc = check_bipoly(ctx, f);
  if (rc) return rc;
  if (f->limbs >= kMaxLimbs) return ctx_fail(ctx, BS_ERR_RANGE, "the derivatives need more than 64 limbs");
  if (elim_degree(*f, var) < 0) return ctx_fail(ctx, BS_ERR_ZERO, "the zero polynomial");
  // the derivative in the other variable first: Q = res(f_x*, f_y*; y) for var = 1
  std::vector<uint32_t> obuf, ebuf;
  bs_bipoly fo, fe;
  derivative_grid(*f, 1 - var, &obuf, &fo);
  derivative_grid(*f, var, &ebuf, &fe);
  BiGcd G;
  rc = bigcd(ctx, fo, fe, var, &G);
  if (rc) return rc;
  HostPoly q;
  const int m = G.ma, n = G.mb;
  if (m < 0 || G.rows.empty()) {  // f_x = 0 (f free of x): f_x* = 0 and Q = 0
    q.c.assign(1, 0u);
    q.u = bs_upoly{-1, 1, q.c.data()};
  } else if (n < 0) {  // cannot happen for a nonconstant f; report it as the zero polynomial
    return ctx_fail(ctx, BS_ERR_ZERO, "the derivative in the eliminated variable vanishes");
  } else if (std::min(m, n) == 0 || G.all_vanish) {
    // one cofactor is free of the eliminated variable: Q = (that cofactor)^(degree of the other)
    const int small = std::min(m, n) == 0 ? (m == 0 ? 0 : 1) : G.small;
    std::vector<HostPoly> r;
    grid_rows(small == 0 ? fo : fe, var, &r);
    const int top = small == 0 ? m : n;
    const int other = (small == 0 ? n : m) - G.d;
    HostPoly cof;
    // the cofactor: the top row of the smaller polynomial over the top row of h
    rc = divide_owned(ctx, r[top].u, G.rows[G.d].u, &cof);
    if (rc) return rc;
    rc = zpow_owned(ctx, cof.u, other, &q);
    if (rc) return rc;
  } else {
    const HostPoly& sd = G.sr[G.d];
    const int e = m + n - 2 * G.d;
    const HostPoly& lam = G.rows[G.d];
    if (e == 0 || is_one(lam)) {
      q.c = sd.c;
      q.u = sd.u;
      q.u.c = q.c.data();
    } else {
      HostPoly le;
      rc = zpow_owned(ctx, lam.u, e, &le);
      if (!rc) rc = divide_owned(ctx, sd.u, le.u, &q);
      if (rc) return rc;
    }
  }
  *d = G.d;
  const int dq = owned_degree(q);
  if (!Q->c) {  // size query
    Q->deg = std::max(dq, 0);
    Q->limbs = q.u.limbs;
    return BS_OK;
  }
  if (dq < 0) {
    for (int c = 0; c <= Q->deg; ++c) std::memset(Q->c + (size_t)c * Q->limbs, 0, sizeof(uint32_t) * Q->limbs);
    Q->deg = -1;
    return BS_OK;
  }
  rc = put_result(ctx, q.u.c, q.u.limbs, dq, Q);
  if (!rc) Q->deg = dq;
  return rc;
}
