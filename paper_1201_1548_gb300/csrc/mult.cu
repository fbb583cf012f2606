// The multiplicity of a polynomial Q at the roots of R (Sec. 3.3: Teissier's test compares
// mult(R, alpha) with mult(Q, alpha) at the critical values alpha, Q = res(f_x*, f_y*)).
//
// With Yun's factorisation Q = c q_1 q_2^2 ... q_s^s (the q_k square-free and pairwise
// coprime), a root alpha of Q has mult(Q, alpha) = k exactly when q_k(alpha) = 0.  So the
// square-free part R* of R splits into pairwise coprime factors
//   c_k = gcd(R*, q_k)  (k >= 1),   c_0 = R* / gcd(R*, Q*)   (Q* the square-free part of Q),
// c_k vanishing exactly at the roots of R where Q has multiplicity k.  Every square-free
// part, factorisation, gcd and quotient runs on the device by the modular route; the host
// only orders the batches and packs the result.
#include <cuda_runtime.h>

#include <algorithm>
#include <vector>

#include "ctx.cuh"
#include "modpoly.cuh"
#include "owned.cuh"

namespace bs {

static bs_upoly trimmed(const bs_upoly& u) {
  bs_upoly t = u;
  t.deg = trimmed_degree(u);
  return t;
}

static int run_mult(bs_ctx* ctx, const bs_upoly* r, const bs_upoly* q, int cap, int32_t* fdeg, int32_t* nfac,
                    bs_upoly* out) {
  for (const bs_upoly* u : {r, q})
    if (u->deg < -1 || u->limbs < 1 || (u->deg >= 0 && !u->c)) return ctx_fail(ctx, BS_ERR_ARG, "bad polynomial");
  const bs_upoly R = trimmed(*r), Q = trimmed(*q);
  if (R.deg < 0) return ctx_fail(ctx, BS_ERR_ZERO, "R = 0");
  if (Q.deg < 0) return ctx_fail(ctx, BS_ERR_ZERO, "Q = 0: every multiplicity is infinite");
  if (!out->c) {  // size query: the factors of R* are factors of R, bounded as R*'s are
    bs_upoly b{0, 0, nullptr};
    int rc = bs_squarefree_part(ctx, &R, &b);
    if (rc) return rc;
    out->deg = R.deg + Q.deg;
    out->limbs = b.limbs;
    *nfac = Q.deg + 1;
    return BS_OK;
  }
  // R* and Q* in one batch
  std::vector<HostPoly> sq;
  int rc = modgcd_owned(ctx, {1, 1}, {R, Q}, {}, &sq);
  if (rc) return rc;
  const bs_upoly Rs = sq[0].u, Qs = sq[1].u;
  // Yun's factorisation of Q: q_1, ..., q_s packed one after the other
  std::vector<int32_t> qdeg;
  int32_t s = 0;
  HostPoly qf;
  if (Q.deg > 0) {
    bs_upoly b{0, 0, nullptr};
    int32_t capf = 0;
    rc = bs_squarefree_factorization(ctx, &Q, 0, nullptr, &capf, &b);
    if (rc) return rc;
    qdeg.assign(std::max(capf, 1), 0);
    qf.c.assign((size_t)(std::max(b.deg, 0) + 1) * std::max(b.limbs, 1), 0u);
    qf.u = bs_upoly{std::max(b.deg, 0), std::max(b.limbs, 1), qf.c.data()};
    rc = bs_squarefree_factorization(ctx, &Q, (int)qdeg.size(), qdeg.data(), &s, &qf.u);
    if (rc) return rc;
  }
  // c_k = gcd(R*, q_k) for the non-constant q_k, and g = gcd(R*, Q*), in one batch
  std::vector<int> kind, which;
  std::vector<bs_upoly> a, b;
  size_t off = 0;
  for (int k = 1; k <= s; ++k) {
    const bs_upoly qk{qdeg[k - 1], qf.u.limbs, qf.u.c + off * qf.u.limbs};
    off += (size_t)qdeg[k - 1] + 1;
    if (qk.deg <= 0 || Rs.deg <= 0) continue;
    kind.push_back(0);
    a.push_back(Rs);
    b.push_back(qk);
    which.push_back(k);
  }
  std::vector<HostPoly> ck;
  if (!kind.empty()) {
    kind.push_back(0);
    a.push_back(Rs);
    b.push_back(Qs);
    rc = modgcd_owned(ctx, kind, a, b, &ck);
    if (rc) return rc;
  }
  // c_0 = R* / g (exact)
  HostPoly c0;
  bs_upoly C0 = Rs;
  if (!ck.empty() && ck.back().u.deg > 0) {
    std::vector<HostPoly> qo;
    rc = modgcd_owned(ctx, {2}, {Rs}, {ck.back().u}, &qo);
    if (rc) return rc;
    c0 = std::move(qo[0]);
    C0 = c0.u;
  }
  // the factors in order c_0, c_1, ..., c_t
  std::vector<bs_upoly> fac{C0};
  for (size_t j = 0; j + 1 < ck.size(); ++j) {
    const int k = which[j];
    while ((int)fac.size() < k) fac.push_back(bs_upoly{-2, 1, nullptr});  // constant 1, filled below
    fac.push_back(ck[j].u);
  }
  while (fac.size() > 1 && fac.back().deg <= 0) fac.pop_back();
  int total = 0;
  for (size_t k = 0; k < fac.size(); ++k) {
    if (fac[k].deg == -2 || fac[k].deg == 0) fac[k].deg = 0;
    total += fac[k].deg;
  }
  if (total != Rs.deg) return ctx_fail(ctx, BS_ERR_UNLUCKY, "the factors do not multiply to R*");
  if ((int)fac.size() > cap) return ctx_fail(ctx, BS_ERR_CAPACITY, "factor capacity too small");
  const int words = total + (int)fac.size();
  if (words - 1 > out->deg) return ctx_fail(ctx, BS_ERR_CAPACITY, "output capacity too small");
  static const uint32_t one = 1u;
  int pos = 0;
  for (size_t k = 0; k < fac.size(); ++k) {
    bs_upoly view{fac[k].deg, out->limbs, out->c + (size_t)pos * out->limbs};
    // a constant factor is 1 (primitive with a positive leading coefficient)
    rc = (fac[k].deg == 0) ? put_result(ctx, &one, 1, 0, &view) : put_result(ctx, fac[k].c, fac[k].limbs, fac[k].deg, &view);
    if (rc) return rc;
    fdeg[k] = fac[k].deg;
    pos += fac[k].deg + 1;
  }
  for (int i = pos; i <= out->deg; ++i)
    for (int l = 0; l < out->limbs; ++l) out->c[(size_t)i * out->limbs + l] = 0u;
  out->deg = pos - 1;
  *nfac = (int32_t)fac.size();
  return BS_OK;
}

}  // namespace bs

using namespace bs;

extern "C" int bs_root_multiplicity(bs_ctx* ctx, const bs_upoly* r, const bs_upoly* q, int cap_factors,
                                    int32_t* fdeg, int32_t* nfac, bs_upoly* out) {
  if (!ctx) return BS_ERR_ARG;
  if (!r || !q || !out || !nfac || cap_factors < 0 || (out->c && cap_factors > 0 && !fdeg))
    return ctx_fail(ctx, BS_ERR_ARG, "bad arguments");
  if (out->c && (out->limbs < 1 || out->deg < 0)) return ctx_fail(ctx, BS_ERR_ARG, "bad output capacity");
  if (ctx->server) return ctx_fail(ctx, BS_ERR_ARG, "the context runs a serving loop");
  return run_mult(ctx, r, q, cap_factors, fdeg, nfac, out);
}
