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
* Teissier's Q = res(f_x*, f_y*; y) with f_x*, f_y* the cofactors of h = gcd(f_x, f_y) in
  Z[x, y] (the primitive pseudo-remainder sequence), and the upper bound
  N^+ = deg R* n_y - deg R + deg gcd(R^inf mod p, Q mod p) (Sec. 3.3).
* mult(Q, alpha) at the roots alpha of R (the quantity Teissier's test of Sec. 3.3 sets
  against mult(R, alpha)): over Q, Q and its first k - 1 derivatives vanish at alpha
  exactly when mult(Q, alpha) >= k, so G_1 = gcd(R*, Q), G_(k+1) = gcd(G_k, Q^(k)) holds
  the roots of multiplicity at least k and c_k = G_k / G_(k+1) those of multiplicity k.
"""

from __future__ import annotations

from fractions import Fraction
from functools import partial

from . import gcd as G
from . import poly as P
from . import resultant as R
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


def subresultant_y(f, g, d, map=map):
    """The d-th subresultant polynomial of f and g with respect to y as [s_0, ..., s_d], s_j
    the coefficient of y^j, an ascending list in Z[x] (formal degrees in y from the actual
    top rows, 0 <= d < min(m_y, n_y)).  Each s_j is a minor of the Sylvester matrix, so its
    degree is at most the resultant's bound D; the points route evaluates the univariate
    subresultant polynomial exactly at D + 1 consecutive integers and interpolates."""
    rf, rg = y_rows(f), y_rows(g)
    q = min(len(rf), len(rg)) - 1
    if not 0 <= d < q:
        raise ValueError("subresultant index out of range")
    D = degree_bound(f, g)
    x0 = -(D // 2)
    xs = list(range(x0, x0 + D + 1))
    vals = list(map(partial(_sres_at_point, rf, rg, d), xs))
    return [interpolate_consecutive(x0, [v[j] if j < len(v) else 0 for v in vals])
            for j in range(d + 1)]


def _sres_at_point(rf, rg, d, x):
    a = [P.evaluate(row, x) for row in rf]
    b = [P.evaluate(row, x) for row in rg]
    return subresultant_poly(a, b, d)


def psc_univariate(a, b):
    """[sr_0, ..., sr_(q-1)], q = min(m, n), over Z (formal degrees)."""
    q = min(len(a), len(b)) - 1
    return [det_bareiss(psc_matrix(a, b, i)) for i in range(max(q, 0))]


def psc_univariate_modp(a, b, p):
    q = min(len(a), len(b)) - 1
    a = [x % p for x in a]
    b = [x % p for x in b]
    return [det_modp(psc_matrix(a, b, i), p) for i in range(max(q, 0))]


def _psc_at_point(rf, rg, i, x):
    """sr_i(f(x, y), g(x, y)) exactly, formal degrees from the rows rf, rg."""
    a = [P.evaluate(row, x) for row in rf]
    b = [P.evaluate(row, x) for row in rg]
    return det_bareiss(psc_matrix(a, b, i), IntRing)


def psc_y(f, g, route=None, map=map):
    """[sr_0(x), ..., sr_(q-1)(x)] of f and g with respect to y, q = min(m_y, n_y), each an
    ascending list in Z[x] (formal degrees in y from the actual top rows).  ``map`` applies
    the point determinants of the points route (a process pool's map spreads them over
    cores; the arithmetic is the same)."""
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
            vals = list(map(partial(_psc_at_point, rf, rg, i), xs))
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


# ---- bivariate gcd and Teissier's Q (Sec. 3.3, computation of n_alpha^+) ---------------
# A bivariate polynomial is a list of rows in Z[x] by powers of y (trailing zero rows
# trimmed), the layout of y_rows.

def _rows(f):
    return y_rows(f)


def _content_rows(A):
    return G.content_rows(A)


def _scale_rows(A, c):
    return [P.mul(r, c) for r in A]


def _div_rows(A, c):
    return [P.exact_div_z(r, c) for r in A]


def _pprem(A, B):
    """Pseudo-remainder of A by B in Z[x][y]: lc(B)^(deg A - deg B + 1) A mod B."""
    A = [list(r) for r in A]
    db = len(B) - 1
    lb = B[-1]
    while len(A) - 1 >= db and A:
        da = len(A) - 1
        la = A[-1]
        A = [P.mul(r, lb) for r in A]                        # scale, then cancel the top
        for i in range(db + 1):
            A[da - db + i] = P.sub(A[da - db + i], P.mul(la, B[i]))
        while A and not P.trim(A[-1]):
            A.pop()
    return A


def bigcd_y(A, B):
    """gcd of A and B in Z[x][y] by the primitive pseudo-remainder sequence: the gcd of the
    contents (in Z[x]) times the primitive part of the last nonzero remainder, with a
    positive leading coefficient (the highest power of x in the top row); gcd(0, B) is B
    with that sign, gcd(0, 0) = 0 (no rows)."""
    A, B = _rows(A), _rows(B)
    if not A or not B:  # gcd(0, B) = B with a positive leading coefficient
        g = B if not A else A
        if g and g[-1][-1] < 0:
            g = _scale_rows(g, [-1])
        return g
    ca, cb = _content_rows(A), _content_rows(B)
    c = G.gcd_z(ca, cb)
    A, B = _div_rows(A, ca), _div_rows(B, cb)
    if len(A) < len(B):
        A, B = B, A
    while B and len(B) > 1:
        Rm = _pprem(A, B)
        A, B = B, (_div_rows(Rm, _content_rows(Rm)) if Rm else [])
    g = B if B else A
    if len(g) == 1:                                          # a constant in y: pp is 1
        g = [[1]]
    g = _div_rows(g, _content_rows(g))
    if g[-1][-1] < 0:
        g = _scale_rows(g, [-1])
    return _scale_rows(g, c)


def bidiv_exact(A, H):
    """A / H in Z[x][y] (exact)."""
    A, H = [list(r) for r in _rows(A)], _rows(H)
    dh = len(H) - 1
    Q = [[] for _ in range(len(A) - dh)]
    for k in range(len(A) - 1 - dh, -1, -1):
        c = P.exact_div_z(A[k + dh], H[-1])
        Q[k] = c
        for i in range(dh + 1):
            A[k + i] = P.sub(A[k + i], P.mul(c, H[i]))
    assert not any(P.trim(r) for r in A), "inexact bivariate division"
    return Q


def d_dx(f):
    rows = y_rows(f)
    return [P.derivative(r) for r in rows]


def teissier_q(f):
    """(Q, d): Q = res(f_x*, f_y*; y) with f_x* = f_x / h, f_y* = f_y / h, h = gcd(f_x, f_y),
    and d = deg_y h."""
    fx, fy = d_dx(f), d_dy(f)
    h = bigcd_y(fx, fy)
    fxs, fys = bidiv_exact(fx, h), bidiv_exact(fy, h)
    return R.res_y(fxs, fys), len(h) - 1


def fiber_upper_bound_modp(f, p):
    """N^+ of Sec. 3.3 for the prime p: deg R* n_y - deg R + deg gcd(R^inf mod p, Q mod p),
    where the last term sums the multiplicities in Q of the common roots:
    T_1 = gcd(R* mod p, Q mod p), T_k = gcd(T_(k-1), Q^(k-1) mod p)."""
    fy = d_dy(f)
    n_y = len(y_rows(f)) - 1
    Rr = R.res_y(f, fy)
    Rs = G.squarefree_part(Rr)
    Q, _ = teissier_q(f)
    Qp = P.mod_p(Q, p)
    T = G.gcd_modp(P.mod_p(Rs, p), Qp, p)
    total = 0
    dQ = Qp
    while P.deg(T) > 0:
        total += P.deg(T)
        dQ = P.mod_p(P.derivative(dQ), p)
        T = G.gcd_modp(T, dQ, p)
    return P.deg(Rs) * n_y - P.deg(Rr) + total


def multiplicity_split(r, q):
    """[c_0, c_1, ..., c_t] with R* = c_0 c_1 ... c_t, c_k the primitive factor (positive
    leading coefficient) vanishing exactly at the roots alpha of R with mult(Q, alpha) = k;
    c_t is not constant unless t = 0.  R and Q must be non-zero."""
    rs = G.squarefree_part(r)
    q = P.trim(q)
    if not q:
        raise ValueError("Q = 0")
    chain = [rs]                      # G_0 = R*, G_1, G_2, ...
    dq = q
    while P.deg(chain[-1]) > 0:
        g = G.gcd_z(chain[-1], dq)
        g = P.primitive_part(g) if P.deg(g) > 0 else [1]
        if g[-1] < 0:
            g = P.scale(g, -1)
        chain.append(g)
        if not dq:
            break
        dq = P.derivative(dq)
    out = [P.exact_div_z(chain[k], chain[k + 1]) for k in range(len(chain) - 1)]
    out = [P.primitive_part(c) if P.deg(c) > 0 else [1] for c in out]
    out = [P.scale(c, -1) if c[-1] < 0 else c for c in out]
    while len(out) > 1 and P.deg(out[-1]) <= 0:
        out.pop()
    return out or [[1]]
