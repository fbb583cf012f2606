"""Principal subresultant coefficients and the fiber counts built on them (Sec. 3.3,
"(Exact) Computation of N" and "Computation of N^-").

Test infrastructure only: plain, slow, exact.

* The i-th subresultant of a (formal degree m) and b (formal degree n) is the
  determinant of the matrix with n - i shifted rows of a and m - i shifted rows of b, as
  in the Sylvester matrix, whose last column holds the polynomials y^k a and y^k b
  themselves (Sec. 3.3, the displayed Sres_i matrix).  Its coefficient of y^i, the
  principal subresultant coefficient sr_i, is the determinant of the square matrix that
  keeps the columns of y^(m+n-i-1), ..., y^i (`psc_matrix`); sr_0 is the resultant.
* Over a field, deg gcd(a, b) = k exactly when sr_0 = ... = sr_(k-1) = 0 and sr_k != 0
  (quoted in Sec. 3.3); this is the main pin of the construction.
* For f in Z[x, y] without vertical asymptotes, with R = res(f, f_y; y), R* its
  square-free part and sr_i = sr_i(f, f_y; y): S_0 = R*, S_i = gcd(S_(i-1), sr_i),
  R_i = S_(i-1) / S_i, and N = sum_i (n_y - i) deg R_i counts the distinct points of the
  curve over its x-critical values (Sec. 3.3).  The same chain over Z_p for one prime p
  gives the lower bound N^- = sum_i (n_y - i) deg R_i^(p).
"""

from __future__ import annotations

from fractions import Fraction

from . import gcd as G
from . import poly as P
from .resultant import degree_bound, interpolate_consecutive, y_rows
from .sylvester import IntRing, PolyRing, det_bareiss, det_modp


def psc_matrix(a, b, i, zero=0):
    """Square matrix of size m + n - 2i whose determinant is sr_i(a, b); a and b are
    ascending coefficient lists of formal degrees len - 1 (leading entries may be 0)."""
    m, n = len(a) - 1, len(b) - 1
    w = m + n - 2 * i
    rows = []
    for r in range(n - i):          # y^(n-i-1-r) a: coefficient a_(m-s) in column r + s
        row = [zero] * w
        for s in range(m + 1):
            if r + s < w:
                row[r + s] = a[m - s]
        rows.append(row)
    for r in range(m - i):          # y^(m-i-1-r) b
        row = [zero] * w
        for s in range(n + 1):
            if r + s < w:
                row[r + s] = b[n - s]
        rows.append(row)
    return rows


def subresultant_poly(a, b, i):
    """The i-th subresultant Sres_i(a, b) as an ascending list in y (over Z): the
    coefficient of y^j (j <= i) is the determinant of the first m + n - 2i - 1 columns of
    the subresultant matrix together with the column of y^j."""
    m, n = len(a) - 1, len(b) - 1
    w = m + n - 2 * i
    # rows of the subresultant matrix over all columns y^(m+n-i-1) .. y^0
    cols = m + n - i
    rows = []
    for r in range(n - i):
        row = [0] * cols
        for s in range(m + 1):
            row[r + s] = a[m - s]
        rows.append(row)
    for r in range(m - i):
        row = [0] * cols
        for s in range(n + 1):
            row[r + s] = b[n - s]
        rows.append(row)
    out = []
    for j in range(i + 1):
        cj = cols - 1 - j                      # the column of y^j
        M = [row[: w - 1] + [row[cj]] for row in rows]
        out.append(det_bareiss(M))
    return P.trim(out)


def psc_univariate(a, b):
    """[sr_0, ..., sr_(q-1)], q = min(m, n), over Z (formal degrees)."""
    q = min(len(a), len(b)) - 1
    return [det_bareiss(psc_matrix(a, b, i)) for i in range(max(q, 0))]


def psc_univariate_modp(a, b, p):
    q = min(len(a), len(b)) - 1
    a = [x % p for x in a]
    b = [x % p for x in b]
    return [det_modp(psc_matrix(a, b, i), p) for i in range(max(q, 0))]


def psc_y(f, g, route=None):
    """[sr_0(x), ..., sr_(q-1)(x)] of f and g with respect to y, q = min(m_y, n_y), each an
    ascending list in Z[x] (formal degrees in y from the actual top rows)."""
    rf, rg = y_rows(f), y_rows(g)
    if not rf or not rg:
        return []
    my, ny = len(rf) - 1, len(rg) - 1
    q = min(my, ny)
    if route is None:
        route = "zx" if my + ny <= 10 else "points"
    if route == "zx":
        return [P.trim(det_bareiss(psc_matrix(rf, rg, i, zero=[]), PolyRing)) for i in range(q)]
    if route == "points":
        D = degree_bound(f, g)      # every sr_i has degree <= D
        x0 = -(D // 2)
        xs = list(range(x0, x0 + D + 1))
        out = []
        for i in range(q):
            vals = []
            for x in xs:
                a = [P.evaluate(row, x) for row in rf]
                b = [P.evaluate(row, x) for row in rg]
                vals.append(det_bareiss(psc_matrix(a, b, i), IntRing))
            out.append(interpolate_consecutive(x0, vals))
        return out
    raise ValueError(route)


def psc_y_modp(f, g, p):
    """The psc sequence of f mod p and g mod p with respect to y, in Z_p[x]."""
    return [P.mod_p(s, p) for s in psc_y(f, g)]


def d_dy(f):
    rows = y_rows(f)
    return [[j * c for c in rows[j]] for j in range(1, len(rows))] or [[0]]


def fiber_decomposition(f):
    """[deg R_1, deg R_2, ...] of the decomposition R* = R_1 R_2 ... (Sec. 3.3) and
    N = sum_i (n_y - i) deg R_i, for f with a constant leading coefficient in y."""
    fy = d_dy(f)
    n_y = len(y_rows(f)) - 1
    sr = psc_y(f, fy)
    S_prev = G.squarefree_part(sr[0])
    degs = []
    for i in range(1, len(sr) + 1):
        if i < len(sr):
            S_i = G.gcd_z(S_prev, sr[i]) if P.trim(sr[i]) else S_prev
        else:
            S_i = [1]                    # sr_(n_y - 1) = lc(f_y) is a nonzero constant
        degs.append(P.deg(S_prev) - P.deg(S_i))
        S_prev = S_i
    while degs and degs[-1] == 0:
        degs.pop()
    N = sum((n_y - i) * d for i, d in enumerate(degs, start=1))
    return degs, N


def fiber_lower_bound_modp(f, p):
    """N^- of Sec. 3.3: the same chain over Z_p for the prime p (p must not divide the
    leading coefficients of f and f_y); S_0 = R* mod p from the exact square-free part."""
    fy = d_dy(f)
    n_y = len(y_rows(f)) - 1
    sr = psc_y_modp(f, fy, p)
    S_prev = P.monic_p(P.mod_p(G.squarefree_part(psc_y(f, fy)[0]), p), p)
    degs = []
    for i in range(1, len(sr) + 1):
        S_i = G.gcd_modp(S_prev, sr[i], p) if i < len(sr) else [1]
        degs.append(P.deg(S_prev) - P.deg(S_i))
        S_prev = S_i
    while degs and degs[-1] == 0:
        degs.pop()
    return degs, sum((n_y - i) * d for i, d in enumerate(degs, start=1))


def split_curve(branches):
    """f = prod_k (y - a_k(x)) for integer polynomials a_k (ascending lists); rows by
    powers of y (the layout of the workloads)."""
    f = [[1]]                                   # the constant 1 as a y-row list
    for a in branches:
        # multiply f (rows by y) by (y - a)
        out = [[] for _ in range(len(f) + 1)]
        for j, row in enumerate(f):
            out[j + 1] = P.add(out[j + 1], row)
            out[j] = P.sub(out[j], P.mul(row, a))
        f = out
    width = max(len(r) for r in f)
    return [list(r) + [0] * (width - len(r)) for r in f]


def split_curve_fiber_count(branches):
    """N for a split curve by direct counting: over every x-critical value alpha (where
    two branches meet; the branches are linear with rational meeting points) the number of
    distinct values a_k(alpha)."""
    lin = [(Fraction(a[0]), Fraction(a[1] if len(a) > 1 else 0)) for a in branches]
    assert all(len(a) <= 2 for a in branches)
    xs = set()
    for j in range(len(lin)):
        for k in range(j + 1, len(lin)):
            (d1, c1), (d2, c2) = lin[j], lin[k]
            if c1 == c2:
                assert d1 != d2, "coincident branches: f is not square-free"
                continue
            xs.add((d2 - d1) / (c1 - c2))
    return sum(len({d + c * x for d, c in lin}) for x in xs)
