"""Pins for oracle.gcd: planted factors, the echelon theorem route, Yun's identity."""

import random

import pytest

from oracle import gcd as G
from oracle import poly as P
from oracle import resultant as R
from oracle.numtheory import prime_table


def _rand(rng, d, lo=-30, hi=30):
    a = [rng.randrange(lo, hi + 1) for _ in range(d + 1)]
    a[-1] = a[-1] or 1
    return a


def test_gcd_modp_planted_factor():
    rng = random.Random(1)
    p = prime_table(1)[0]
    for _ in range(20):
        c = _rand(rng, rng.randrange(0, 5))
        u = _rand(rng, rng.randrange(0, 6))
        v = _rand(rng, rng.randrange(0, 6))
        if R.res_univariate_modp(u, v, p) == 0:
            continue
        g = G.gcd_modp(P.mul(c, u), P.mul(c, v), p)
        assert g == P.monic_p(c, p)


def test_echelon_route_agrees_with_euclid():
    rng = random.Random(2)
    for p in (101, 65537, prime_table(1)[0]):
        for _ in range(25):
            c = _rand(rng, rng.randrange(0, 4))
            a = P.mul(c, _rand(rng, rng.randrange(0, 5)))
            b = P.mul(c, _rand(rng, rng.randrange(0, 5)))
            if not P.mod_p(a, p) or not P.mod_p(b, p):
                continue
            assert G.echelon_gcd_modp(a, b, p) == G.gcd_modp(a, b, p)


def test_gcd_modp_conventions():
    p = 97
    assert G.gcd_modp([], [], p) == []
    assert G.gcd_modp([], [3, 6], p) == P.monic_p([3, 6], p)
    assert G.gcd_modp([5], [1, 1], p) == [1]


def test_gcd_z_planted_and_content():
    rng = random.Random(3)
    for _ in range(10):
        c = _rand(rng, rng.randrange(1, 4))
        u = _rand(rng, rng.randrange(1, 4))
        v = _rand(rng, rng.randrange(1, 4))
        if R.res_univariate(u, v) == 0:
            continue
        a = P.scale(P.mul(c, u), 6)
        b = P.scale(P.mul(c, v), 4)
        g = G.gcd_z(a, b)
        # Gauss's lemma: the primitive part is pp(c), the content is gcd of the contents
        assert P.primitive_part(g) == P.primitive_part(c)
        from math import gcd
        assert P.content(g) == gcd(P.content(a), P.content(b))
        assert g[-1] > 0
        # g divides both
        P.exact_div_z(a, g)
        P.exact_div_z(b, g)


def test_yun_product_identity_and_squarefree_part():
    rng = random.Random(4)
    for _ in range(6):
        u = _rand(rng, 2, -9, 9)
        v = _rand(rng, 2, -9, 9)
        w = _rand(rng, 1, -9, 9)
        # skip unless u, v, w are square-free and pairwise coprime
        ok = all(R.res_univariate(a, b) != 0 for a, b in ((u, v), (u, w), (v, w)))
        ok = ok and all(R.res_univariate(a, P.derivative(a)) != 0 for a in (u, v, w))
        if not ok:
            continue
        r = P.mul(P.mul(u, P.mul(v, v)), P.mul(w, P.mul(w, w)))
        fac = G.yun(r)
        assert len(fac) == 3
        prod = [1]
        for i, fi in enumerate(fac, start=1):
            for _ in range(i):
                prod = P.mul(prod, fi)
        assert P.primitive_part(prod) == P.primitive_part(r)
        assert fac[0] == P.primitive_part(u)
        assert fac[1] == P.primitive_part(v)
        assert fac[2] == P.primitive_part(w)
        sq = G.squarefree_part(r)
        assert sq == P.primitive_part(P.mul(u, P.mul(v, w)))


def test_squarefree_part_conventions():
    assert G.squarefree_part([7]) == [1]
    assert G.squarefree_part([-4, 0, 2]) == [-2, 0, 1]   # 2(x^2 - 2): pp, positive lc
    with pytest.raises(ValueError):
        G.squarefree_part([])


def test_sympy_cross_check_gcd():
    sympy = pytest.importorskip("sympy")
    x = sympy.symbols("x")
    rng = random.Random(5)
    for _ in range(5):
        c = _rand(rng, 3)
        a = P.mul(c, _rand(rng, 4))
        b = P.mul(c, _rand(rng, 3))
        sa = sum(k * x ** i for i, k in enumerate(a))
        sb = sum(k * x ** i for i, k in enumerate(b))
        ref = sympy.Poly(sympy.gcd(sa, sb), x)
        coeffs = [int(t) for t in reversed(ref.all_coeffs())]
        if coeffs[-1] < 0:
            coeffs = [-t for t in coeffs]
        assert G.gcd_z(a, b) == coeffs


def test_content_rows_divides_and_leaves_a_primitive_part():
    # the content divides every row, the quotients have content 1, lc(h) > 0
    rng = random.Random(7)
    for t in range(10):
        h0 = _rand(rng, rng.randrange(0, 4))
        c = rng.choice([1, -1, 6, -35])
        rows = [P.scale(P.mul(h0, _rand(rng, rng.randrange(0, 4))), c) for _ in range(rng.randrange(1, 5))]
        if t % 3 == 0:
            rows.insert(1, [])                                   # a zero row
        h, q = G.primitive_rows(rows)
        assert h[-1] > 0
        assert all(P.mul(h, qi) == P.trim(r) for qi, r in zip(q, rows))
        assert G.content_rows(q) == [1]
        # h is a multiple of the planted factor
        assert not P.divmod_q(h, h0)[1]
