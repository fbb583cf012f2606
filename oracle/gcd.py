"""gcds in Z_p[x] and Z[x], Yun's square-free factorisation and the square-free part.

* gcd over Z_p: Euclid's algorithm, result made monic (gcd(0, 0) = 0).
* gcd over Z_p by the theorem of Sec. 5.1 ("Computing gcds in Z[x]"): bring the
  Sylvester matrix to row-echelon form by row operations only; its last non-zero row
  holds the coefficients of the gcd.  Used as a second, independent route in the tests.
* gcd over Z: gcd(cont a, cont b) * pp(gcd over Q[x]), leading coefficient positive.
* Yun's algorithm (Sec. 2.1, BiProject): square-free, pairwise coprime r_i with
  R = c * prod r_i**i.
* square-free part R* = pp(R / gcd(R, R')) with a positive leading coefficient
  (Sec. 3.3 uses deg R* as the number of distinct roots of R).
* content of a bivariate polynomial with respect to one variable: the gcd in Z[x] of its
  coefficient rows, positive leading coefficient (Sec. 4 divides it out first).
"""

from __future__ import annotations

from fractions import Fraction
from math import gcd as igcd

from . import poly as P
from .sylvester import sylvester


def gcd_modp(a, b, p):
    """Monic gcd of a, b in Z_p[x] by Euclid."""
    a = P.mod_p(a, p)
    b = P.mod_p(b, p)
    while b:
        _, r = P.divmod_p(a, b, p)
        a, b = b, r
    return P.monic_p(a, p)


def echelon_gcd_modp(a, b, p):
    """Monic gcd in Z_p[x] from the last non-zero row of the row-echelon Sylvester matrix."""
    a = P.mod_p(a, p)
    b = P.mod_p(b, p)
    if not a:
        return P.monic_p(b, p)
    if not b:
        return P.monic_p(a, p)
    m, n = len(a) - 1, len(b) - 1
    if m == 0 or n == 0:
        return [1]
    S = sylvester(a, b)
    r = m + n
    A = [list(row) for row in S]
    # row echelon form over Z_p with row operations only
    prow = 0
    for col in range(r):
        piv = None
        for i in range(prow, r):
            if A[i][col] % p:
                piv = i
                break
        if piv is None:
            continue
        A[prow], A[piv] = A[piv], A[prow]
        inv = pow(A[prow][col], p - 2, p)
        for i in range(prow + 1, r):
            f = A[i][col] * inv % p
            if f:
                for j in range(col, r):
                    A[i][j] = (A[i][j] - f * A[prow][j]) % p
        prow += 1
    last = A[prow - 1]
    # column c holds the coefficient of x**(r - 1 - c)
    coeffs = [last[r - 1 - e] % p for e in range(r)]
    return P.monic_p(coeffs, p)


def gcd_q(a, b):
    """Monic gcd over Q[x] (Fraction coefficients)."""
    a = P.trim([Fraction(x) for x in a])
    b = P.trim([Fraction(x) for x in b])
    while b:
        _, r = P.divmod_q(a, b)
        a, b = b, r
    if not a:
        return []
    lc = a[-1]
    return [x / lc for x in a]


def gcd_z(a, b):
    """gcd in Z[x]: gcd of the contents times the primitive gcd, positive leading coefficient."""
    a, b = P.trim(a), P.trim(b)
    if not a and not b:
        return []
    if not a:
        return P.scale(P.primitive_part(b), P.content(b))
    if not b:
        return P.scale(P.primitive_part(a), P.content(a))
    c = igcd(P.content(a), P.content(b))
    g = P.fraction_to_primitive_z(gcd_q(a, b))
    return P.scale(g, c)


def squarefree_part(r):
    """R* = pp(R / gcd(R, R')) with positive leading coefficient; R must be non-zero."""
    r = P.trim(r)
    if not r:
        raise ValueError("square-free part of the zero polynomial")
    if len(r) == 1:
        return [1]
    g = gcd_q(r, P.derivative(r))
    q, rem = P.divmod_q([Fraction(x) for x in r], g)
    assert not rem
    return P.fraction_to_primitive_z(q)


def yun(r):
    """Yun's square-free factorisation over Q: primitive r_1, r_2, ... with
    pp(R) = prod r_i**i (up to sign).  Trailing factors equal to 1 are dropped."""
    r = P.trim(r)
    if not r:
        raise ValueError("square-free factorisation of the zero polynomial")
    f = [Fraction(x) for x in r]
    fp = P.derivative(f)
    a0 = gcd_q(f, fp)
    b, rem = P.divmod_q(f, a0)
    assert not rem
    c, rem = P.divmod_q(fp, a0)
    assert not rem
    d = P.sub(c, P.derivative(b))
    out = []
    while len(P.trim(b)) > 1:
        a = gcd_q(b, d)
        b_next, rem = P.divmod_q(b, a)
        assert not rem
        c_next, rem = P.divmod_q(d, a)
        assert not rem
        d = P.sub(c_next, P.derivative(b_next))
        out.append(P.fraction_to_primitive_z(a))
        b = b_next
    while out and len(out[-1]) == 1:
        out.pop()
    return out


def content_rows(rows):
    """gcd in Z[x] of the polynomials `rows` (the coefficients of f in the eliminated
    variable), with a positive leading coefficient; [] if every row is zero."""
    g = []
    for r in rows:
        g = gcd_z(g, r)
    return g


def primitive_rows(rows):
    """(h, [row / h]): the content and the rows of the primitive part."""
    h = content_rows(rows)
    return h, [P.exact_div_z(r, h) for r in rows]
