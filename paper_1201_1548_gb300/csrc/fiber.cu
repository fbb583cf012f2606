// The number of distinct points of a curve over its critical values (Sec. 3.3).
//
// For f without vertical asymptotes (constant leading coefficient in the eliminated
// variable) let R = res(f, f_y), R* its square-free part and sr_i the principal subresultant
// coefficients of f and f_y.  Over a root alpha of R*, deg gcd(f(alpha, y), f_y(alpha, y)) = k
// exactly when sr_1, ..., sr_(k-1) vanish at alpha and sr_k does not, so the chain
//   S_0 = R*,  S_i = gcd(S_(i-1), sr_i),  R_i = S_(i-1) / S_i
// splits R* by the number n_y - i of distinct roots of f(alpha, y), and
//   N = sum_i (n_y - i) deg R_i.
// The exact form runs the chain in Z[x] on the exact psc's; the modular form runs it over
// Z_p for one prime (the first table prime dividing no leading coefficient) from the
// residues of the psc's and the exact R*, which gives the lower bound N^- of Sec. 3.3
// (equal to N for all but finitely many primes).
//
// Every step runs on the device: the psc stage and the resultant engine, the square-free
// part and the gcds in Z[x] (modular, Brown's rule) or in Z_p[x].  The host only forms f_y
// and walks the chain.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <vector>

#include "ctx.cuh"
#include "modpoly.cuh"
#include "owned.cuh"

namespace bs {

// f_y (var = 1) or f_x (var = 0) with one more limb per coefficient
static void grid_derivative(const bs_bipoly& f, int var, std::vector<uint32_t>* buf, bs_bipoly* out) {
  const int L = f.limbs, L1 = L + 1;
  const int dx = var ? f.deg_x : std::max(f.deg_x - 1, 0);
  const int dy = var ? std::max(f.deg_y - 1, 0) : f.deg_y;
  buf->assign((size_t)(dx + 1) * (dy + 1) * L1, 0u);
  for (int j = 0; j <= dy; ++j)
    for (int i = 0; i <= dx; ++i) {
      const int sj = var ? j + 1 : j, si = var ? i : i + 1;
      const uint32_t k = (uint32_t)(var ? sj : si);
      uint32_t* d = buf->data() + ((size_t)j * (dx + 1) + i) * L1;
      if (sj > f.deg_y || si > f.deg_x) continue;  // f has degree 0 there: f_y = 0
      const uint32_t* s = f.c + ((size_t)sj * (f.deg_x + 1) + si) * L;
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

// degree of f in the eliminated variable and whether its leading coefficient is constant
static int lead_degree(const bs_bipoly& f, int var, bool* constant_lc) {
  const int ne = var ? f.deg_y : f.deg_x, no = var ? f.deg_x : f.deg_y;
  auto at = [&](int e, int o) {
    const int j = var ? e : o, i = var ? o : e;
    return f.c + ((size_t)j * (f.deg_x + 1) + i) * f.limbs;
  };
  for (int e = ne; e >= 0; --e) {
    bool any = false, only0 = true;
    for (int o = 0; o <= no; ++o)
      if (!limbs_zero(at(e, o), f.limbs)) {
        any = true;
        if (o > 0) only0 = false;
      }
    if (any) {
      *constant_lc = only0;
      return e;
    }
  }
  *constant_lc = true;
  return -1;
}

static uint32_t residue_of(const uint32_t* c, int L, uint32_t p) {
  uint64_t r = 0;
  for (int l = L - 1; l >= 0; --l) r = ((r << 32) | c[l]) % p;
  if (c[L - 1] >> 31) {  // value = raw - 2^(32 L)
    uint64_t t = 1;
    for (int l = 0; l < L; ++l) t = (t << 32) % p;
    r = (r + p - t) % p;
  }
  return (uint32_t)r;
}

static int run_fiber(bs_ctx* ctx, const bs_bipoly* f, int var, int mode, int cap, int32_t* degs, int32_t* s_out,
                     int64_t* N_out, uint32_t* p_out) {
  if (!f || f->deg_x < 0 || f->deg_y < 0 || f->limbs < 1 || !f->c)
    return ctx_fail(ctx, BS_ERR_ARG, "bad bivariate polynomial");
  if (f->limbs >= kMaxLimbs) return ctx_fail(ctx, BS_ERR_RANGE, "the derivative needs more than 64 limbs");
  *s_out = 0;
  *N_out = 0;
  *p_out = 0;
  bool clc = true;
  const int ny = lead_degree(*f, var, &clc);
  if (ny < 0) return ctx_fail(ctx, BS_ERR_ZERO, "the zero polynomial");
  if (!clc) return ctx_fail(ctx, BS_ERR_ARG, "the leading coefficient is not constant (vertical asymptote)");
  if (ny < 2) return BS_OK;  // at most one root in every fiber: no critical values
  std::vector<uint32_t> gbuf;
  bs_bipoly g;
  grid_derivative(*f, var, &gbuf, &g);
  int rc;
  if (mode == 2) {  // N^+ = deg R* n_y - deg R + deg gcd(R^inf mod p, Q mod p)
    std::vector<uint32_t> xbuf;
    bs_bipoly fx;
    grid_derivative(*f, 1 - var, &xbuf, &fx);
    int32_t q = 0, dmax = 0;
    uint32_t p = 0;
    rc = bs_psc_modp(ctx, &fx, &g, var, &q, &dmax, nullptr, nullptr, &p);
    if (rc) return rc;
    std::vector<int32_t> dq(std::max(q, 1));
    std::vector<uint32_t> coef((size_t)std::max(q, 1) * (dmax + 1));
    if (q > 0) {
      rc = bs_psc_modp(ctx, &fx, &g, var, &q, &dmax, dq.data(), coef.data(), &p);
      if (rc) return rc;
    }
    int d = 0;
    while (d < q && dq[d] < 0) ++d;
    std::vector<uint32_t> Qp;
    if (d < q)
      Qp.assign(coef.begin() + (size_t)d * (dmax + 1), coef.begin() + (size_t)d * (dmax + 1) + dq[d] + 1);
    else
      Qp.assign(1, 1u);
    if (p == 0) p = host_primes().p[0];  // q = 0: f_x or f_y constant in the variable
    HostPoly Rr;
    rc = fetch(&Rr, [&](bs_upoly* o) { return bs_resultant(ctx, f, &g, var, o); });
    if (rc) return rc;
    int dr = Rr.u.deg;
    while (dr >= 0 && limbs_zero(Rr.u.c + (size_t)dr * Rr.u.limbs, Rr.u.limbs)) --dr;
    if (dr < 0) return ctx_fail(ctx, BS_ERR_ZERO, "res(f, f_y) = 0: f is not square-free");
    Rr.u.deg = dr;
    HostPoly Rs;
    rc = fetch(&Rs, [&](bs_upoly* o) { return bs_squarefree_part(ctx, &Rr.u, o); });
    if (rc) return rc;
    std::vector<uint32_t> S(Rs.u.deg + 1);
    for (int i = 0; i <= Rs.u.deg; ++i) S[i] = residue_of(Rs.u.c + (size_t)i * Rs.u.limbs, Rs.u.limbs, p);
    int ds = Rs.u.deg;
    while (ds >= 0 && S[ds] == 0u) --ds;
    // T_1 = gcd(R* mod p, Q mod p), T_k = gcd(T_(k-1), Q^(k-1) mod p): sum deg T_k counts
    // the common roots with their multiplicities in Q
    int64_t total = 0;
    std::vector<uint32_t> T(std::max<size_t>(S.size(), Qp.size()) + 1);
    int dt = -1;
    rc = bs_gcd_modp(ctx, S.data(), ds, Qp.data(), (int)Qp.size() - 1, p, T.data(), &dt);
    if (rc) return rc;
    std::vector<uint32_t> dQ = Qp, G(T.size());
    while (dt > 0) {
      total += dt;
      for (size_t i = 0; i + 1 < dQ.size(); ++i)  // the derivative mod p
        dQ[i] = (uint32_t)((uint64_t)dQ[i + 1] * (uint64_t)((i + 1) % p) % p);
      dQ.pop_back();
      int ddq = (int)dQ.size() - 1;
      while (ddq >= 0 && dQ[ddq] == 0u) --ddq;
      int dg = -1;
      rc = bs_gcd_modp(ctx, T.data(), dt, dQ.data(), ddq, p, G.data(), &dg);
      if (rc) return rc;
      std::copy(G.begin(), G.begin() + (dg + 1), T.begin());
      dt = dg;
    }
    *N_out = (int64_t)Rs.u.deg * ny - dr + total;
    *p_out = p;
    return BS_OK;
  }
  std::vector<int32_t> dl;  // deg S_0, deg S_1, ...
  if (mode == 0) {
    // exact: the psc's, R* and the chain of gcds in Z[x]
    int32_t q = 0;
    rc = bs_psc(ctx, f, &g, var, 0, &q, nullptr);
    if (rc) return rc;
    std::vector<bs_upoly> sr(q, bs_upoly{0, 0, nullptr});
    rc = bs_psc(ctx, f, &g, var, q, &q, sr.data());
    if (rc) return rc;
    std::vector<std::vector<uint32_t>> bufs(q);
    for (int i = 0; i < q; ++i) {
      bufs[i].assign((size_t)(std::max(sr[i].deg, 0) + 1) * sr[i].limbs, 0u);
      sr[i].c = bufs[i].data();
    }
    rc = bs_psc(ctx, f, &g, var, q, &q, sr.data());
    if (rc) return rc;
    if (sr[0].deg < 0) return ctx_fail(ctx, BS_ERR_ZERO, "res(f, f_y) = 0: f is not square-free");
    HostPoly S;
    rc = fetch(&S, [&](bs_upoly* o) { return bs_squarefree_part(ctx, &sr[0], o); });
    if (rc) return rc;
    dl.push_back(S.u.deg);
    for (int i = 1; i < q && S.u.deg > 0; ++i) {
      HostPoly T;
      rc = fetch(&T, [&](bs_upoly* o) { return bs_gcd_z(ctx, &S.u, &sr[i], o); });
      if (rc) return rc;
      S = std::move(T);
      S.u.c = S.c.data();
      dl.push_back(S.u.deg);
    }
  } else {
    // modular: the psc's mod one prime, R* exact and reduced, the chain in Z_p[x]
    int32_t q = 0, dmax = 0;
    uint32_t p = 0;
    rc = bs_psc_modp(ctx, f, &g, var, &q, &dmax, nullptr, nullptr, &p);
    if (rc) return rc;
    std::vector<int32_t> dq(q);
    std::vector<uint32_t> coef((size_t)q * (dmax + 1));
    rc = bs_psc_modp(ctx, f, &g, var, &q, &dmax, dq.data(), coef.data(), &p);
    if (rc) return rc;
    HostPoly R;
    rc = fetch(&R, [&](bs_upoly* o) { return bs_resultant(ctx, f, &g, var, o); });
    if (rc) return rc;
    int dr = R.u.deg;
    while (dr >= 0 && limbs_zero(R.u.c + (size_t)dr * R.u.limbs, R.u.limbs)) --dr;
    if (dr < 0) return ctx_fail(ctx, BS_ERR_ZERO, "res(f, f_y) = 0: f is not square-free");
    R.u.deg = dr;
    HostPoly Rs;
    rc = fetch(&Rs, [&](bs_upoly* o) { return bs_squarefree_part(ctx, &R.u, o); });
    if (rc) return rc;
    std::vector<uint32_t> S(Rs.u.deg + 1);
    for (int i = 0; i <= Rs.u.deg; ++i) S[i] = residue_of(Rs.u.c + (size_t)i * Rs.u.limbs, Rs.u.limbs, p);
    int ds = Rs.u.deg;
    while (ds >= 0 && S[ds] == 0u) --ds;  // p divides no leading coefficient of f, f_y
    dl.push_back(ds);
    std::vector<uint32_t> G(std::max(ds, dmax) + 2);
    for (int i = 1; i < q && ds > 0; ++i) {
      int dg = -1;
      rc = bs_gcd_modp(ctx, S.data(), ds, coef.data() + (size_t)i * (dmax + 1), dq[i], p, G.data(), &dg);
      if (rc) return rc;
      S.assign(G.begin(), G.begin() + (dg + 1));
      ds = dg;
      dl.push_back(ds);
    }
    *p_out = p;
  }
  // d_i = deg S_(i-1) - deg S_i, the chain ending in a constant
  std::vector<int32_t> d;
  for (size_t i = 1; i < dl.size(); ++i) d.push_back(dl[i - 1] - dl[i]);
  if (dl.back() > 0) d.push_back(dl.back());  // S_(q-1) divides sr_(n_y - 1) = lc(f_y), a constant
  while (!d.empty() && d.back() == 0) d.pop_back();
  if ((int)d.size() > cap) return ctx_fail(ctx, BS_ERR_CAPACITY, "degree list capacity too small");
  int64_t N = 0;
  for (size_t i = 0; i < d.size(); ++i) {
    degs[i] = d[i];
    N += (int64_t)(ny - (int)(i + 1)) * d[i];
  }
  *s_out = (int32_t)d.size();
  *N_out = N;
  return BS_OK;
}

}  // namespace bs

using namespace bs;

extern "C" int bs_fiber_count(bs_ctx* ctx, const bs_bipoly* f, int var, int mode, int cap, int32_t* degs,
                              int32_t* s, int64_t* N, uint32_t* p) {
  if (!ctx) return BS_ERR_ARG;
  if (!f || (var != 0 && var != 1) || mode < 0 || mode > 2 || cap < 0 || (cap > 0 && !degs) || !s || !N ||
      !p)
    return ctx_fail(ctx, BS_ERR_ARG, "bad arguments");
  if (ctx->server) return ctx_fail(ctx, BS_ERR_ARG, "the context runs a serving loop");
  return run_fiber(ctx, f, var, mode, cap, degs, s, N, p);
}
