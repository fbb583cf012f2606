"""Pins for oracle.resultant: closed forms, identities and two independent routes."""

import random

import pytest

from oracle import poly as P
from oracle import resultant as R
from oracle.numtheory import prime_table
from oracle.sylvester import det_leibniz, sylvester
from workloads import bimul, cfg1_pair, dense_curve, d_dy
import numpy as np


def _rng(seed):
    return np.random.Generator(np.random.PCG64(seed))


def _rand_biv(rng, dy, dx, lo=-20, hi=20):
    return [[int(rng.integers(lo, hi + 1)) for _ in range(dx + 1)] for _ in range(dy + 1)]


def test_univariate_linear_closed_form():
    # Res(y - a, y - b) = a - b with the first polynomial's rows first
    for a in range(-3, 4):
        for b in range(-3, 4):
            assert R.res_univariate([-a, 1], [-b, 1]) == a - b


def test_discriminant_of_quadratic():
    # Res(a y^2 + b y + c, 2 a y + b) = -a (b^2 - 4 a c)
    for (a, b, c) in [(1, 3, 2), (2, -5, 7), (-3, 0, 4), (5, 1, 0)]:
        assert R.res_univariate([c, b, a], [b, 2 * a]) == -a * (b * b - 4 * a * c)


def test_root_product_formula_univariate():
    rng = random.Random(2)
    for m in range(0, 5):
        for n in range(0, 5):
            roots_a = [rng.randrange(-9, 10) for _ in range(m)]
            roots_b = [rng.randrange(-9, 10) for _ in range(n)]
            ca, cb = rng.choice([-3, -2, 2, 5]), rng.choice([-2, 1, 3])
            a, b = [ca], [cb]
            for r in roots_a:
                a = P.mul(a, [-r, 1])
            for r in roots_b:
                b = P.mul(b, [-r, 1])
            expect = ca ** n * cb ** m
            for x in roots_a:
                for y in roots_b:
                    expect *= (x - y)
            assert R.res_univariate(a, b) == expect


def test_constant_conventions():
    assert R.res_univariate([5], [7]) == 1          # 0 x 0 determinant
    assert R.res_univariate([3], [1, 2, 1]) == 9    # f constant: f^n
    assert R.res_univariate([1, 2, 1], [3]) == 9    # g constant: g^m
    assert R.res_y([[0]], [[1, 2], [3]]) == []      # res(0, g) = 0


def test_degree_drop_identities():
    """Res_{m,n}(f,g) = (-1)^n g_n Res_{m-1,n}(f,g) if f_m = 0;
    Res_{m,n}(f,g) = f_m Res_{m,n-1}(f,g) if g_n = 0."""
    rng = random.Random(9)
    for _ in range(30):
        m, n = rng.randrange(1, 6), rng.randrange(1, 6)
        f = [rng.randrange(-9, 10) for _ in range(m)] + [0]
        g = [rng.randrange(-9, 10) for _ in range(n)] + [rng.randrange(1, 9)]
        assert R.res_univariate(f, g) == (-1) ** n * g[-1] * R.res_univariate(f[:-1], g)
        f2 = [rng.randrange(-9, 10) for _ in range(m)] + [rng.randrange(1, 9)]
        g2 = [rng.randrange(-9, 10) for _ in range(n)] + [0]
        assert R.res_univariate(f2, g2) == f2[-1] * R.res_univariate(f2, g2[:-1])
        # both leading coefficients zero: first column vanishes
        assert R.res_univariate(f, g2) == 0


def test_routes_agree_with_brute_force_tiny():
    rng = _rng(4)
    for _ in range(12):
        dyf, dyg = int(rng.integers(1, 4)), int(rng.integers(1, 4))
        f = _rand_biv(rng, dyf, int(rng.integers(0, 3)), -5, 5)
        g = _rand_biv(rng, dyg, int(rng.integers(0, 3)), -5, 5)
        f[-1][0] = f[-1][0] or 1
        g[-1][0] = g[-1][0] or 2
        from oracle.sylvester import PolyRing
        S = sylvester(R.y_rows(f), R.y_rows(g), zero=[])
        brute = P.trim(det_leibniz(S, PolyRing))
        assert R.res_y(f, g, route="zx") == brute
        assert R.res_y(f, g, route="points") == brute


def test_antisymmetry_and_multiplicativity():
    rng = _rng(6)
    for _ in range(6):
        f1 = dense_curve(rng, int(rng.integers(1, 4)), 6)
        f2 = dense_curve(rng, int(rng.integers(1, 4)), 6)
        g = dense_curve(rng, int(rng.integers(1, 4)), 6)
        my, ny = len(R.y_rows(f1)) - 1, len(R.y_rows(g)) - 1
        r_fg = R.res_y(f1, g)
        r_gf = R.res_y(g, f1)
        assert r_gf == P.scale(r_fg, (-1) ** (my * ny))
        assert R.res_y(bimul(f1, f2), g) == P.mul(R.res_y(f1, g), R.res_y(f2, g))


def test_closed_form_linear_in_y():
    """res_y(y - a(x), g) = g(x, a(x))."""
    rng = _rng(8)
    for _ in range(6):
        a = [int(rng.integers(-5, 6)) for _ in range(int(rng.integers(1, 4)))]
        g = dense_curve(rng, int(rng.integers(1, 5)), 5)
        f = [[-c for c in a], [1] + [0] * (len(a) - 1)]
        # g(x, a(x)) = sum_j g_j(x) a(x)^j
        expect = []
        apow = [1]
        for row in g:
            expect = P.add(expect, P.mul(row, apow))
            apow = P.mul(apow, a)
        assert R.res_y(f, g) == P.trim(expect)


def test_theorem1_common_root_and_shared_asymptote():
    rng = _rng(10)
    for _ in range(5):
        x0, y0 = int(rng.integers(-3, 4)), int(rng.integers(-3, 4))
        f = dense_curve(rng, 3, 6)
        g = dense_curve(rng, 3, 6)
        # shift constant terms so that f(x0, y0) = g(x0, y0) = 0
        fv = sum(c * x0 ** i * y0 ** j for j, row in enumerate(f) for i, c in enumerate(row))
        gv = sum(c * x0 ** i * y0 ** j for j, row in enumerate(g) for i, c in enumerate(row))
        f[0][0] -= fv
        g[0][0] -= gv
        assert P.evaluate(R.res_y(f, g), x0) == 0
    # both leading y-coefficients vanish at x = 2: R(2) = 0 even without a finite common root
    f = [[1, 0, 1], [3, 1], [-2, 1]]        # lc_y f = x - 2
    g = [[5, 1], [2 * -2, 2]]               # lc_y g = 2x - 4
    f = [row + [0] * (3 - len(row)) for row in f]
    g = [row + [0] * (2 - len(row)) for row in g]
    assert P.evaluate(R.res_y(f, g), 2) == 0


def test_degree_and_coefficient_bounds():
    rng = _rng(12)
    primes = prime_table(200)
    for _ in range(8):
        f = dense_curve(rng, int(rng.integers(1, 6)), int(rng.integers(4, 40)))
        g = dense_curve(rng, int(rng.integers(1, 6)), int(rng.integers(4, 40)))
        r = R.res_y(f, g)
        D = R.degree_bound(f, g)
        assert P.deg(r) <= D <= R.total_degree(f) * R.total_degree(g)
        b2 = R.bound_sq(f, g)
        assert all(c * c <= b2 for c in r)
        k = R.primes_needed(b2, primes)
        prod = 1
        for p in primes[:k]:
            prod *= p
        assert prod > 2 * max(abs(c) for c in r)


def test_point_values_and_modular_values():
    f, g = cfg1_pair(1)
    r = R.res_y(f, g)
    for x0 in (-3, 0, 1, 7):
        assert R.res_at_point(f, g, x0) == P.evaluate(r, x0)
    p = prime_table(1)[0]
    for x0 in (5, 123456, p - 1):
        assert R.res_at_point_modp(f, g, x0, p) == P.evaluate(r, x0) % p


def test_interpolate_consecutive_recovers_polynomial():
    rng = random.Random(1)
    for d in range(0, 12):
        poly = [rng.randrange(-10**6, 10**6) for _ in range(d + 1)]
        x0 = -(d // 2)
        vals = [P.evaluate(poly, x0 + t) for t in range(d + 1)]
        assert R.interpolate_consecutive(x0, vals) == P.trim(poly)


def test_res_x_is_res_y_of_transpose():
    f, g = cfg1_pair(2)
    assert R.res_x(f, g) == R.res_y(R.transpose(f), R.transpose(g))


def test_discriminant_type_small():
    rng = _rng(14)
    f = dense_curve(rng, 4, 8)
    g = d_dy(f)
    assert R.res_y(f, g, route="zx") == R.res_y(f, g, route="points")


def test_sympy_cross_check():
    sympy = pytest.importorskip("sympy")
    x, y = sympy.symbols("x y")
    f, g = cfg1_pair(3)

    def to_sym(h):
        return sum(c * x ** i * y ** j for j, row in enumerate(h) for i, c in enumerate(row))

    ref = sympy.Poly(sympy.resultant(to_sym(f), to_sym(g), y), x)
    ours = R.res_y(f, g)
    assert [int(c) for c in reversed(ref.all_coeffs())] == ours


def test_interpolate_consecutive_modp_recovers_polynomial():
    """Newton interpolation over Z_p against known polynomials and against the integer
    interpolant reduced mod p."""
    rng = random.Random(4)
    for p in (101, 2147483647, (1 << 61) - 1):
        for d in range(0, 14):
            poly = [rng.randrange(-10**9, 10**9) for _ in range(d + 1)]
            x0 = -(d // 2) - rng.randrange(3)
            vals = [P.evaluate(poly, x0 + t) for t in range(d + 1)]
            got = R.interpolate_consecutive_modp(x0, vals, p)
            assert got == P.mod_p(poly, p)
            assert got == P.mod_p(R.interpolate_consecutive(x0, vals), p)
    with pytest.raises(ValueError):
        R.interpolate_consecutive_modp(0, [1, 2, 3], 2)


def test_res_y_modp_against_the_zx_route():
    """res(f, g; y) mod p by point determinants over Z_p and interpolation over Z_p,
    against the exact Bareiss determinant over Z[x] reduced mod p: random pairs, a leading
    coefficient with integer roots (vertical asymptotes at some of the points), a square
    factor (R = 0) and the constant conventions."""
    from workloads import cfg4_cases
    rng = _rng(15)
    q = (1 << 61) - 1
    for t in range(10):
        f = dense_curve(rng, int(rng.integers(1, 6)), int(rng.integers(2, 40)),
                        zero_prob=0.2 if t % 2 else 0.0)
        g = dense_curve(rng, int(rng.integers(1, 6)), int(rng.integers(2, 40)))
        for p in (q, 2147483647):
            assert R.res_y_modp(f, g, p) == P.mod_p(R.res_y(f, g, route="zx"), p), t
    cases = cfg4_cases(seed=3, deg=3, bits=10)
    for name in ("4a", "4b2", "4c"):
        f, g = cases[name]
        assert R.res_y_modp(f, g, q) == P.mod_p(R.res_y(f, g, route="zx"), q), name
    assert R.res_y_modp(cases["4b2"][0], cases["4b2"][1], q) == []
    assert R.res_y_modp([[0]], [[1, 2], [3]], q) == []
    assert R.res_y_modp([[5]], [[7, 1]], q) == [1]
    assert R.res_y_modp([[3]], [[1], [2], [1]], q) == [9]
