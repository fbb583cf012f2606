"""Parity of the principal subresultant coefficients (Sec. 3.3) with the oracle: small and
medium pairs in full, degenerate pairs (common factors, vertical asymptotes, leading
coefficients that vanish mod a prime), both variables, and the degree-32 pair on sampled
points, where the oracle's exact determinants at integer points check the specialisation
of every returned sr_i."""

import numpy as np
import pytest

from oracle import poly as P
from oracle import resultant as R
from oracle import subresultant as S
from workloads import cfg1_pair, cfg2_pair, cfg4_cases, dense_curve

pytestmark = pytest.mark.gpu


def _rng(seed):
    return np.random.Generator(np.random.PCG64(seed))


def test_psc_small_pairs(ctx):
    rng = _rng(51)
    for t in range(16):
        f = dense_curve(rng, int(rng.integers(1, 6)), int(rng.integers(2, 40)))
        g = dense_curve(rng, int(rng.integers(1, 6)), int(rng.integers(2, 40)))
        assert ctx.psc(f, g) == S.psc_y(f, g), t


def test_psc_degree6_pair(ctx):
    f, g = cfg1_pair(1)                          # two dense curves of total degree 6
    got = ctx.psc(f, g)
    assert len(got) == 6
    assert got == S.psc_y(f, g)
    assert got[0] == R.res_y(f, g)
    fy = S.d_dy(f)                               # a curve and its y-derivative
    assert ctx.psc(f, fy) == S.psc_y(f, fy)


def test_psc_medium_degree(ctx):
    rng = _rng(52)
    f = dense_curve(rng, 10, 24)
    g = S.d_dy(f)
    assert ctx.psc(f, g) == S.psc_y(f, g)


def test_psc_eliminating_x(ctx):
    rng = _rng(53)
    for t in range(4):
        f = dense_curve(rng, 4, 16)
        g = dense_curve(rng, 3, 16)
        assert ctx.psc(f, g, var=0) == S.psc_y(R.transpose(f), R.transpose(g)), t


def test_psc_common_factor_vanishes(ctx):
    # f = c u, g = c v with deg_y c = 2: sr_0 and sr_1 are the zero polynomial
    rng = _rng(54)
    from workloads import bimul
    c = dense_curve(rng, 2, 8)
    u = dense_curve(rng, 2, 8)
    v = dense_curve(rng, 3, 8)
    f, g = bimul(c, u), bimul(c, v)
    got = ctx.psc(f, g)
    assert got[0] == [] and got[1] == []
    assert got[2] != []
    assert got == S.psc_y(f, g)


def test_psc_degenerate_cases(ctx):
    cases = cfg4_cases(seed=2, deg=3, bits=8)
    for name in ("4a", "4b", "4c"):
        f, g = cases[name]
        assert ctx.psc(f, g) == S.psc_y(f, g), name


def test_psc_leading_row_divisible_by_a_prime(ctx):
    # the leading row of f is a multiple of the first table prime: that prime is
    # rejected and the spare primes take its place
    import paper_1201_1548_gb300 as bs
    p0 = bs.bs_prime_table(1)[0]
    rng = _rng(55)
    f = dense_curve(rng, 4, 12)
    f[-1] = [c * p0 for c in f[-1]]
    g = S.d_dy(f)
    assert ctx.psc(f, g) == S.psc_y(f, g)


def test_psc_trivial_shapes(ctx):
    f = [[1, 2, 3], [4, 5, 6]]
    assert ctx.psc(f, [[7, 1]]) == []                 # g constant in y: no index below 0
    assert ctx.psc([[0]], f) == []                    # the zero polynomial
    assert ctx.psc(f, f) == S.psc_y(f, f)             # sr_0 = 0 (identical polynomials)


def test_psc_degree32_sampled_points(ctx):
    # the degree-32 curve and its y-derivative (31 coefficients, 2500-bit sr_0): each
    # returned sr_i evaluated at integer points equals the exact determinant there
    f, g = cfg2_pair(1)
    got = ctx.psc(f, g)
    assert len(got) == 31
    assert got[0] == ctx.resultant(f, g)
    D = R.degree_bound(f, g)
    assert all(P.deg(s) <= D for s in got)
    for x0 in (-1, 2):
        a, b = R.specialise(f, x0), R.specialise(g, x0)
        for i in (0, 1, 7, 30):
            M = S.psc_matrix(a, b, i)
            from oracle.sylvester import det_bareiss
            assert P.evaluate(got[i], x0) == det_bareiss(M), (x0, i)
