"""Exact bivariate resultants in Z[x] and the quantities the modular route relies on.

Definitions followed:

* R^(y) = res(f, g; y) is the determinant of the Sylvester matrix S^(y)(f, g) whose
  entries are the coefficients f_i^(y)(x), g_i^(y)(x) in Z[x] (Sec. 2, "Resultants");
  m_y, n_y are the actual y-degrees of f and g (Sec. 2, "Notation").  res(f, g; x) is the
  same with the roles of x and y exchanged.
* deg R^(y) <= m * n for total degrees m, n (Sec. 2, below the Sylvester matrix); each
  term of the determinant also has degree <= n_y deg_x f + m_y deg_x g.
* Step (b)/(c) of the modular algorithm (Sec. 5.1): for a prime p and a point alpha,
  the value R(alpha) mod p equals the determinant of the Sylvester matrix of
  f(alpha, y), g(alpha, y) mod p with the SAME formal degrees m_y, n_y (specialisation
  commutes with the determinant of a fixed-shape matrix).

Two independent routes compute R exactly:

* ``route='zx'``: fraction-free Bareiss elimination with entries in Z[x];
* ``route='points'``: Bareiss over Z at D + 1 consecutive integer points, then exact
  Newton interpolation carried out in integers (scaled by D!).

Coefficient bound (no bound is given in the paper; this reading is recorded with the
design notes): for |x| = 1 each f-row of S has Euclidean norm at most
(sum_j ||f_j||_1**2)**(1/2), so Hadamard's inequality gives
|R(x)| <= B = (sum_j ||f_j||_1**2)**(n_y/2) * (sum_j ||g_j||_1**2)**(m_y/2), and every
coefficient of R, being a Fourier coefficient on the unit circle, is at most B in
absolute value.  Symmetric residues then need prod(p) > 2B.
"""

from __future__ import annotations

from functools import partial
from math import factorial

from . import poly as P
from .sylvester import IntRing, PolyRing, det_bareiss, det_modp, sylvester


# --------------------------------------------------------------------------------------
# shapes
# --------------------------------------------------------------------------------------

def is_zero_bivariate(f):
    return all(c == 0 for row in f for c in row)


def y_rows(f):
    """Coefficient rows f_j(x), j = 0..m_y (trailing all-zero rows removed)."""
    rows = [P.trim(row) for row in f]
    while rows and not rows[-1]:
        rows.pop()
    return rows


def transpose(f):
    """Exchange x and y in a bivariate grid."""
    if not f:
        return []
    dx = max(len(r) for r in f)
    return [[(f[j][i] if i < len(f[j]) else 0) for j in range(len(f))] for i in range(dx)]


def total_degree(f):
    d = -1
    for j, row in enumerate(f):
        for i, c in enumerate(row):
            if c:
                d = max(d, i + j)
    return d


def x_degree(f):
    d = -1
    for row in f:
        for i, c in enumerate(row):
            if c:
                d = max(d, i)
    return d


def degree_bound(f, g):
    """D = min(tdeg f * tdeg g, n_y deg_x f + m_y deg_x g) for res_y (actual degrees)."""
    my = len(y_rows(f)) - 1
    ny = len(y_rows(g)) - 1
    if my < 0 or ny < 0:
        return -1
    return min(total_degree(f) * total_degree(g), ny * x_degree(f) + my * x_degree(g))


# --------------------------------------------------------------------------------------
# univariate resultants
# --------------------------------------------------------------------------------------

def res_univariate(a, b):
    """Res_{m,n}(a, b) over Z with formal degrees len(a)-1, len(b)-1 (Sylvester determinant)."""
    return det_bareiss(sylvester(list(a), list(b)), IntRing)


def res_univariate_modp(a, b, p):
    """Res_{m,n}(a, b) mod p with formal degrees (Sylvester determinant over Z_p)."""
    return det_modp(sylvester([x % p for x in a], [x % p for x in b]), p)


# --------------------------------------------------------------------------------------
# bivariate resultant
# --------------------------------------------------------------------------------------

def _formal_rows(f):
    rows = y_rows(f)
    return rows


def res_y(f, g, route=None, map=map):
    """res(f, g; y) in Z[x] (ascending coefficients; [] is the zero polynomial).

    ``map`` applies the point determinants of the points route (the built-in by default;
    a process pool's ``map`` spreads them over cores without changing any arithmetic)."""
    rf = _formal_rows(f)
    rg = _formal_rows(g)
    if not rf or not rg:
        return []
    my, ny = len(rf) - 1, len(rg) - 1
    if my == 0 and ny == 0:
        return [1]
    if route is None:
        route = "zx" if my + ny <= 12 else "points"
    if route == "zx":
        S = sylvester(rf, rg, zero=[])
        return P.trim(det_bareiss(S, PolyRing))
    if route == "points":
        D = degree_bound(f, g)
        x0 = -(D // 2)
        xs = list(range(x0, x0 + D + 1))
        vals = list(map(partial(res_at_point, f, g), xs))
        return interpolate_consecutive(x0, vals)
    raise ValueError(route)


def res_x(f, g, route=None, map=map):
    """res(f, g; x) in Z[y]."""
    return res_y(transpose(f), transpose(g), route=route, map=map)


def resultant(f, g, var=1, route=None, map=map):
    """var = 1 eliminates y (result in Z[x]); var = 0 eliminates x (result in Z[y])."""
    return res_y(f, g, route, map) if var == 1 else res_x(f, g, route, map)


def specialise(f, x0):
    """Coefficients of f(x0, y) in y with the formal degree m_y of f (lc may vanish)."""
    return [P.evaluate(row, x0) for row in _formal_rows(f)]


def res_at_point(f, g, x0):
    """R(x0) exactly: the Sylvester determinant of f(x0, y), g(x0, y) with formal degrees."""
    a = specialise(f, x0)
    b = specialise(g, x0)
    if not a or not b:
        return 0
    return res_univariate(a, b)


def res_at_point_modp(f, g, x0, p):
    """R(x0) mod p computed from f, g reduced mod p (step (c) of Sec. 5.1)."""
    a = [P.evaluate([c % p for c in row], x0) % p for row in _formal_rows(f)]
    b = [P.evaluate([c % p for c in row], x0) % p for row in _formal_rows(g)]
    if not a or not b:
        return 0
    return res_univariate_modp(a, b, p)


def interpolate_consecutive(x0, vals):
    """Integer polynomial through (x0 + t, vals[t]), t = 0..D, by Newton's forward
    differences kept in integers: D! * R(x) = sum_k (D!/k!) Delta^k v_0 prod_{s<k}(x - x_s);
    the final division by D! must be exact (the interpolant has integer coefficients)."""
    D = len(vals) - 1
    if D < 0:
        return []
    diffs = []
    cur = list(vals)
    for _ in range(D + 1):
        diffs.append(cur[0])
        cur = [cur[i + 1] - cur[i] for i in range(len(cur) - 1)]
    Df = factorial(D)
    acc = [diffs[D] * (Df // factorial(D))]
    for k in range(D - 1, -1, -1):
        xk = x0 + k
        # acc = acc * (x - xk) + (D!/k!) * diffs[k]
        nxt = [0] * (len(acc) + 1)
        for i, c in enumerate(acc):
            nxt[i + 1] += c
            nxt[i] -= xk * c
        nxt[0] += (Df // factorial(k)) * diffs[k]
        acc = nxt
    out = []
    for c in acc:
        q, r = divmod(c, Df)
        if r:
            raise ArithmeticError("interpolant is not an integer polynomial")
        out.append(q)
    return P.trim(out)


def interpolate_consecutive_modp(x0, vals, p):
    """Polynomial of degree <= D over Z_p through (x0 + t, vals[t]), t = 0..D, for a
    prime p > D: Newton's form sum_k (Delta^k v_0 / k!) prod_{s<k} (x - x_s), with the
    forward differences and the nested products taken mod p."""
    D = len(vals) - 1
    if D < 0:
        return []
    if p <= D:
        raise ValueError("need p > D so that k! is invertible mod p")
    diffs = []
    cur = [v % p for v in vals]
    for _ in range(D + 1):
        diffs.append(cur[0])
        cur = [(cur[i + 1] - cur[i]) % p for i in range(len(cur) - 1)]
    inv_fact = [1] * (D + 1)
    f = 1
    for k in range(1, D + 1):
        f = f * k % p
        inv_fact[k] = pow(f, p - 2, p)
    acc = [diffs[D] * inv_fact[D] % p]
    for k in range(D - 1, -1, -1):
        xk = (x0 + k) % p
        nxt = [0] * (len(acc) + 1)
        for i, c in enumerate(acc):
            nxt[i + 1] = (nxt[i + 1] + c) % p
            nxt[i] = (nxt[i] - xk * c) % p
        nxt[0] = (nxt[0] + diffs[k] * inv_fact[k]) % p
        acc = nxt
    return P.trim(acc)


def res_y_modp(f, g, p, map=map):
    """res(f, g; y) with every coefficient reduced mod p (a prime above the degree bound
    D): the formal-shape Sylvester determinant over Z_p at the D + 1 consecutive integer
    points of the points route (step (c) of Sec. 5.1), interpolated over Z_p.  Same
    conventions as ``res_y`` (res(0, g) = 0, both constant in y gives 1)."""
    rf = _formal_rows(f)
    rg = _formal_rows(g)
    if not rf or not rg:
        return []
    my, ny = len(rf) - 1, len(rg) - 1
    if my == 0 and ny == 0:
        return [1 % p] if p > 1 else []
    D = degree_bound(f, g)
    x0 = -(D // 2)
    vals = list(map(partial(_res_at_point_modp_args, f, g, p), range(x0, x0 + D + 1)))
    return interpolate_consecutive_modp(x0, vals, p)


def _res_at_point_modp_args(f, g, p, x0):
    return res_at_point_modp(f, g, x0, p)


# --------------------------------------------------------------------------------------
# bound and plan
# --------------------------------------------------------------------------------------

def norm_sq_sum(f):
    """sum_j ||f_j||_1**2 over the y-rows of f."""
    return sum(sum(abs(c) for c in row) ** 2 for row in _formal_rows(f))


def bound_sq(f, g):
    """B**2 = (sum_j ||f_j||_1^2)**n_y * (sum_j ||g_j||_1^2)**m_y  (exact integer)."""
    rf, rg = _formal_rows(f), _formal_rows(g)
    my, ny = len(rf) - 1, len(rg) - 1
    return norm_sq_sum(f) ** ny * norm_sq_sum(g) ** my


def primes_needed(b2, primes):
    """Smallest k with (p_0 ... p_{k-1})**2 > 4 B**2, i.e. prod p > 2B."""
    prod = 1
    for k, p in enumerate(primes):
        if prod * prod > 4 * b2:
            return k
        prod *= p
    if prod * prod > 4 * b2:
        return len(primes)
    raise ValueError("not enough primes")


def plan(f, g, var, primes):
    """Degree bound, transform size, prime count for res(f, g; var)."""
    if var == 0:
        f, g = transpose(f), transpose(g)
    rf, rg = _formal_rows(f), _formal_rows(g)
    my, ny = len(rf) - 1, len(rg) - 1
    D = degree_bound(f, g)
    b2 = bound_sq(f, g) if my >= 0 and ny >= 0 else 0
    N = 1
    while N < D + 1:
        N *= 2
    return {"m_y": my, "n_y": ny, "D": D, "N": N, "bound_sq": b2,
            "k": primes_needed(b2, primes) if D >= 0 else 0}


def symmetric(c, m):
    c %= m
    return c - m if c > m // 2 else c
