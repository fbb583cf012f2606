// Content removal (Sec. 4, the input of the curve analysis): the content h of f with
// respect to the eliminated variable is the gcd of f's coefficients, which are polynomials
// in the other variable; a non-constant h defines vertical lines at its roots, which the
// analysis divides out first.  h is the gcd in Z[x] of the nonzero rows (a pairwise tree of
// batched modular gcds, Brown's rule), and the primitive part is f / h row by row (one
// batch of exact quotients: each row mod p divided by h mod p, lifted under Mignotte's bound
// for a factor of the row).  Every gcd and quotient runs on the device.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <vector>

#include "ctx.cuh"
#include "modpoly.cuh"
#include "owned.cuh"

namespace bs {

static int run_content(bs_ctx* ctx, const bs_bipoly* f, int var, bs_upoly* h, int cap_rows, bs_upoly* rows,
                       int32_t* nrows) {
  if (!f || f->deg_x < 0 || f->deg_y < 0 || f->limbs < 1 || f->limbs > kMaxLimbs || !f->c)
    return ctx_fail(ctx, BS_ERR_ARG, "bad bivariate polynomial");
  // the rows f_e (coefficients of the e-th power of the eliminated variable) as polynomials
  const int ne = var ? f->deg_y : f->deg_x, no = var ? f->deg_x : f->deg_y;
  const int L = f->limbs;
  std::vector<uint32_t> tbuf;
  std::vector<bs_upoly> row(ne + 1);
  if (var) {
    for (int j = 0; j <= ne; ++j) row[j] = bs_upoly{no, L, (uint32_t*)f->c + (size_t)j * (no + 1) * L};
  } else {  // columns of the grid: gather them
    tbuf.resize((size_t)(ne + 1) * (no + 1) * L);
    for (int i = 0; i <= ne; ++i) {
      for (int j = 0; j <= no; ++j)
        std::memcpy(tbuf.data() + ((size_t)i * (no + 1) + j) * L, f->c + ((size_t)j * (f->deg_x + 1) + i) * L,
                    sizeof(uint32_t) * L);
      row[i] = bs_upoly{no, L, tbuf.data() + (size_t)i * (no + 1) * L};
    }
  }
  int top = -1;
  std::vector<int> nz;
  for (int e = 0; e <= ne; ++e) {
    int d = no;
    while (d >= 0 && limbs_zero(row[e].c + (size_t)d * L, L)) --d;
    if (d >= 0) {
      nz.push_back(e);
      top = e;
    }
  }
  if (top < 0) return ctx_fail(ctx, BS_ERR_ZERO, "the content of the zero polynomial");
  *nrows = top + 1;
  const bool query = !h->c || (rows && cap_rows > 0 && !rows[0].c);
  // h and the quotients are factors of rows of degree <= no: Mignotte bounds their
  // coefficients by 2^no ||f_e||_2 < 2^(no + 32 L + 8)
  const int flimbs = L + (no + 40) / 32 + 1;
  if (query) {
    h->deg = no;
    h->limbs = flimbs;
    for (int e = 0; rows && e < std::min(cap_rows, top + 1); ++e) {
      rows[e].deg = no;
      rows[e].limbs = flimbs;
    }
    return BS_OK;
  }
  if (rows && cap_rows < top + 1) return ctx_fail(ctx, BS_ERR_CAPACITY, "fewer rows than the degree needs");
  // gcd of the nonzero rows, a pairwise tree of batched gcds
  std::vector<bs_upoly> cur;
  for (int e : nz) cur.push_back(row[e]);
  std::vector<HostPoly> keep;
  int rc;
  if (cur.size() == 1) {  // one row: gcd(row, 0) normalises its sign
    std::vector<HostPoly> o;
    rc = modgcd_owned(ctx, {0}, {cur[0]}, {bs_upoly{-1, 1, nullptr}}, &o);
    if (rc) return rc;
    keep = std::move(o);
    cur = {keep[0].u};
  }
  while (cur.size() > 1) {
    std::vector<int> kind;
    std::vector<bs_upoly> a, b;
    for (size_t i = 0; i + 1 < cur.size(); i += 2) {
      kind.push_back(0);
      a.push_back(cur[i]);
      b.push_back(cur[i + 1]);
    }
    std::vector<HostPoly> o;
    rc = modgcd_owned(ctx, kind, a, b, &o);
    if (rc) return rc;
    std::vector<bs_upoly> next;
    for (auto& p : o) next.push_back(p.u);  // moving the buffers below keeps these pointers
    if (cur.size() % 2) next.push_back(cur.back());
    for (auto& p : o) keep.push_back(std::move(p));  // alive while later levels read them
    cur = std::move(next);
  }
  const bs_upoly hz = cur[0];
  rc = put_result(ctx, hz.c, hz.limbs, hz.deg, h);
  if (rc) return rc;
  if (!rows) return BS_OK;
  // the primitive part: every row divided by h, one batch
  std::vector<int> kind(top + 1, 2);
  std::vector<bs_upoly> a(row.begin(), row.begin() + top + 1), b(top + 1, hz);
  for (int e = 0; e <= top; ++e) {
    int d = no;
    while (d >= 0 && limbs_zero(a[e].c + (size_t)d * L, L)) --d;
    a[e].deg = d;
  }
  std::vector<HostPoly> q;
  rc = modgcd_owned(ctx, kind, a, b, &q);
  if (rc) return rc;
  for (int e = 0; e <= top; ++e) {
    if (q[e].u.deg < 0) {
      for (int c = 0; c <= rows[e].deg; ++c)
        std::memset(rows[e].c + (size_t)c * rows[e].limbs, 0, sizeof(uint32_t) * rows[e].limbs);
      rows[e].deg = -1;
      continue;
    }
    rc = put_result(ctx, q[e].u.c, q[e].u.limbs, q[e].u.deg, rows + e);
    if (rc) return rc;
  }
  return BS_OK;
}

}  // namespace bs

using namespace bs;

extern "C" int bs_content(bs_ctx* ctx, const bs_bipoly* f, int var, bs_upoly* h, int cap_rows, bs_upoly* rows,
                          int32_t* nrows) {
  if (!ctx) return BS_ERR_ARG;
  if (!f || !h || !nrows || (var != 0 && var != 1) || cap_rows < 0 || (cap_rows > 0 && !rows))
    return ctx_fail(ctx, BS_ERR_ARG, "bad arguments");
  if (ctx->server) return ctx_fail(ctx, BS_ERR_ARG, "the context runs a serving loop");
  return run_content(ctx, f, var, h, cap_rows, cap_rows > 0 ? rows : nullptr, nrows);
}
