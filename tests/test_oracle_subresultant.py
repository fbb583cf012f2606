"""Pins for oracle.subresultant: a hand-expanded determinant, the gcd-degree criterion
quoted in Sec. 3.3, the subresultant polynomial as a multiple of the gcd, specialisation
to points and primes, and the fiber count N against direct counting on split curves."""

import random

import numpy as np
import pytest

from oracle import gcd as G
from oracle import poly as P
from oracle import resultant as R
from oracle import subresultant as S
from oracle.numtheory import prime_table
from workloads import dense_curve


def _rand(rng, d, lo=-20, hi=20):
    a = [rng.randrange(lo, hi + 1) for _ in range(d + 1)]
    a[-1] = a[-1] or 1
    return a


def test_hand_expanded_examples():
    # a = y^3, b = y^2 - 1: Res = a(1) a(-1) = -1; sr_1 = det [[1,0,0],[1,0,-1],[0,1,0]] = 1
    assert S.psc_univariate([0, 0, 0, 1], [-1, 0, 1]) == [-1, 1]
    # a = (y + 1)(y + 2), b = y + 1: a common root, Res = 0
    assert S.psc_univariate([2, 3, 1], [1, 1]) == [0]
    # a = y^2 + p y + q, b = y^2 + r y + s (m = n = 2): sr_1 = det [[1, p], [1, r]] = r - p
    assert S.psc_univariate([5, 3, 1], [7, -4, 1])[1] == -4 - 3
    # m = 3, n = 2, i = 1: the 3 x 3 determinant [[a3,a2,a1],[b2,b1,b0],[0,b2,b1]]
    a, b = [4, -1, 2, 3], [5, 7, -2]
    a3, a2, a1 = 3, 2, -1
    b2, b1, b0 = -2, 7, 5
    want = a3 * (b1 * b1 - b0 * b2) - a2 * (b2 * b1 - 0) + a1 * (b2 * b2 - 0)
    assert S.psc_univariate(a, b)[1] == want


def test_psc_from_roots():
    # Sylvester's single sum (proved by D'Andrea, Hong, Krick and Szanto, 2007): for
    # a = a_m prod (y - alpha_i) with distinct alpha_i and b = b_n prod (y - beta_j),
    # sr_k = (-1)^(k(m-k)) a_m^(n-k) b_n^(m-k) sum over k-subsets A' of the alphas of
    # R(alpha \ A', beta) / R(A', alpha \ A'), with R(U, V) = prod (u - v); k = 0 is the
    # classical root product of the resultant.  No determinant is involved.
    import itertools
    from fractions import Fraction

    def rprod(U, V):
        out = 1
        for u in U:
            for v in V:
                out *= u - v
        return out

    rng = random.Random(17)
    for _ in range(150):
        m, n = rng.randrange(1, 6), rng.randrange(1, 6)
        alpha = rng.sample(range(-9, 10), m)
        beta = [rng.randrange(-9, 10) for _ in range(n)]
        am, bn = rng.choice([1, -2, 3]), rng.choice([1, 2, -3])
        a, b = [am], [bn]
        for r in alpha:
            a = P.mul(a, [-r, 1])
        for r in beta:
            b = P.mul(b, [-r, 1])
        sr = S.psc_univariate(a, b)
        assert len(sr) == min(m, n)
        for k in range(min(m, n)):
            s = Fraction(0)
            for sub in itertools.combinations(range(m), k):
                A1 = [alpha[i] for i in sub]
                A2 = [alpha[i] for i in range(m) if i not in sub]
                s += Fraction(rprod(A2, beta), rprod(A1, A2))
            assert sr[k] == (-1) ** (k * (m - k)) * am ** (n - k) * bn ** (m - k) * s, (m, n, k)


def test_sr0_is_the_resultant():
    rng = random.Random(11)
    for _ in range(20):
        a = _rand(rng, rng.randrange(1, 7))
        b = _rand(rng, rng.randrange(1, 7))
        assert S.psc_univariate(a, b)[0] == R.res_univariate(a, b)


def test_gcd_degree_criterion():
    # deg gcd(a, b) = k  <=>  sr_0 = ... = sr_(k-1) = 0 and sr_k != 0 (over Q, Sec. 3.3)
    rng = random.Random(12)
    seen = set()
    for t in range(60):
        k = t % 4
        c = _rand(rng, k) if k else [1]
        u = _rand(rng, rng.randrange(1, 5))
        v = _rand(rng, rng.randrange(1, 5))
        a, b = P.mul(c, u), P.mul(c, v)
        if P.deg(G.gcd_q(a, b)) != k:
            continue                          # u and v happened to share a factor
        sr = S.psc_univariate(a, b)
        q = min(P.deg(a), P.deg(b))
        assert all(x == 0 for x in sr[:k]), t
        if k < q:
            assert sr[k] != 0, t
        seen.add(k)
    assert seen == {0, 1, 2, 3}


def test_subresultant_polynomial_is_a_multiple_of_the_gcd():
    rng = random.Random(13)
    for t in range(24):
        k = 1 + t % 3
        c = _rand(rng, k)
        u = _rand(rng, rng.randrange(1, 4))
        v = _rand(rng, rng.randrange(1, 4))
        a, b = P.mul(c, u), P.mul(c, v)
        g = G.gcd_z(a, b)
        if P.deg(g) != k or k >= min(P.deg(a), P.deg(b)):
            continue
        for i in range(k):
            assert S.subresultant_poly(a, b, i) == [], (t, i)
        sk = S.subresultant_poly(a, b, k)
        assert P.deg(sk) == k and sk[-1] == S.psc_univariate(a, b)[k]
        assert P.primitive_part(sk) == P.primitive_part(g)


def test_specialisation_to_primes():
    rng = random.Random(14)
    p = prime_table(1)[0]
    for _ in range(12):
        a = _rand(rng, rng.randrange(1, 7), -10**12, 10**12)
        b = _rand(rng, rng.randrange(1, 7), -10**12, 10**12)
        assert S.psc_univariate_modp(a, b, p) == [x % p for x in S.psc_univariate(a, b)]


def test_bivariate_routes_and_points_agree():
    rng = np.random.Generator(np.random.PCG64(15))
    for t in range(5):
        f = dense_curve(rng, 2 + t % 3, 8)
        g = dense_curve(rng, 2 + (t + 1) % 3, 8)
        zx = S.psc_y(f, g, route="zx")
        pts = S.psc_y(f, g, route="points")
        assert zx == pts, t
        D = R.degree_bound(f, g)
        for i, s in enumerate(zx):
            assert P.deg(s) <= D
            for x0 in (-3, 0, 5):
                a, b = R.specialise(f, x0), R.specialise(g, x0)
                assert P.evaluate(s, x0) == S.psc_univariate(a, b)[i]


def test_fiber_count_on_split_curves():
    # f = prod (y - a_k(x)) with linear branches: the x-critical values are where branches
    # meet, and N counts the distinct branch values there
    cases = [
        [[0, 1], [0, -1], [0, 2]],                 # three lines through the origin
        [[0, 1], [0, -1], [2, 1], [1, 0]],
        [[1, 1], [3, -1], [0, 2], [4, -2], [-2, 3]],
    ]
    rng = random.Random(16)
    for _ in range(3):
        cases.append([[rng.randrange(-4, 5), rng.randrange(-3, 4)] for _ in range(4)])
    for branches in cases:
        # distinct branches only (f square-free)
        if len({tuple(b) for b in branches}) < len(branches):
            continue
        f = S.split_curve(branches)
        degs, N = S.fiber_decomposition(f)
        assert N == S.split_curve_fiber_count(branches), branches
        assert sum(degs) == P.deg(G.squarefree_part(R.res_y(f, S.d_dy(f))))
        p = prime_table(3)[2]
        _, lb = S.fiber_lower_bound_modp(f, p)
        assert lb == N                             # a generic prime is not unlucky here


def test_fiber_lower_bound_with_an_unlucky_prime():
    # three lines through the origin and the parallel lines y = 7, y = 0: modulo 7 the
    # last two coincide, every fiber mod 7 has fewer distinct roots and the bound drops
    branches = [[0, 1], [0, -1], [0, 2], [7, 0], [0, 0]]
    f = S.split_curve(branches)
    _, N = S.fiber_decomposition(f)
    assert N == S.split_curve_fiber_count(branches) == 14
    _, lb7 = S.fiber_lower_bound_modp(f, 7)
    assert lb7 < N


def _compose(c1d, a, b):
    """c(a x + b y) as rows by powers of y."""
    def add(A, B):
        n = max(len(A), len(B))
        return [P.add(A[i] if i < len(A) else [], B[i] if i < len(B) else []) for i in range(n)]

    def mul(A, B):
        out = [[] for _ in range(len(A) + len(B) - 1)]
        for i, r in enumerate(A):
            for j, q in enumerate(B):
                out[i + j] = P.add(out[i + j], P.mul(r, q))
        return out
    acc, pw, lin = [[]], [[1]], [[0, a], [b]]
    for c in c1d:
        acc = add(acc, [P.scale(r, c) for r in pw])
        pw = mul(pw, lin)
    return acc, add, mul


def test_bivariate_gcd_planted_factors():
    rng = np.random.Generator(np.random.PCG64(17))
    for t in range(6):
        H = dense_curve(rng, 1 + t % 2, 4)
        U = dense_curve(rng, 2, 4)
        V = dense_curve(rng, 2, 4)
        _, add, mul = _compose([1], 1, 1)
        A, B = mul(H, U), mul(H, V)
        g = S.bigcd_y(A, B)
        # g divides both, the cofactors are coprime, and g is a multiple of H
        ca, cb = S.bidiv_exact(A, g), S.bidiv_exact(B, g)
        assert S.bigcd_y(ca, cb) == [[1]]
        S.bidiv_exact(g, H)


def test_bivariate_gcd_against_sympy():
    sympy = pytest.importorskip("sympy")
    x, y = sympy.symbols("x y")
    rng = np.random.Generator(np.random.PCG64(18))

    def to_expr(F):
        return sum(c * x**i * y**j for j, r in enumerate(F) for i, c in enumerate(r))
    for t in range(4):
        H, U, V = (dense_curve(rng, 2, 4) for _ in range(3))
        _, add, mul = _compose([1], 1, 1)
        A, B = mul(H, U), mul(H, V)
        want = sympy.Poly(sympy.gcd(to_expr(A), to_expr(B)), x, y)
        got = sympy.Poly(to_expr(S.bigcd_y(A, B)), x, y)
        assert got == want or got == -want, t


def test_teissier_q_closed_form():
    # f = P(s)^2 K(t) + c with s = x + y, t = x - y: f_x = P (2 P' K + P K'),
    # f_y = P (2 P' K - P K'), so Q = res_y(2 P' K + P K', 2 P' K - P K') up to a constant
    rng = random.Random(19)
    for t in range(5):
        pc = [rng.randrange(-4, 5) or 1 for _ in range(rng.randrange(2, 4))]
        kc = [rng.randrange(-4, 5) or 1 for _ in range(rng.randrange(2, 4))]
        Pp, add, mul = _compose(pc, 1, 1)
        dP, _, _ = _compose(P.derivative(pc), 1, 1)
        Kk, _, _ = _compose(kc, 1, -1)
        dK, _, _ = _compose(P.derivative(kc), 1, -1)
        f = add(mul(mul(Pp, Pp), Kk), [[rng.randrange(1, 9)]])
        two = [[2]]
        a = add(mul(mul(two, dP), Kk), mul(Pp, dK))
        b = add(mul(mul(two, dP), Kk), [P.scale(r, -1) for r in mul(Pp, dK)])
        Q, d = S.teissier_q(f)
        assert d == len(Pp) - 1
        assert P.primitive_part(Q) == P.primitive_part(R.res_y(a, b)), t
        # the first principal subresultant coefficient of f_x, f_y that is not zero is
        # a constant multiple of Q (the cofactor property of subresultants)
        sr = S.psc_y(S.d_dx(f), S.d_dy(f))
        assert all(not P.trim(s) for s in sr[:d]) and P.primitive_part(sr[d]) == P.primitive_part(Q)


def test_fiber_bounds_bracket_N():
    p = prime_table(1)[0]
    for branches in ([[0, 1], [0, -1], [2, 1], [1, 0]], [[1, 1], [3, -1], [0, 2], [4, -2]]):
        f = S.split_curve(branches)
        _, N = S.fiber_decomposition(f)
        _, lb = S.fiber_lower_bound_modp(f, p)
        ub = S.fiber_upper_bound_modp(f, p)
        assert lb <= N <= ub
        assert ub == N          # lines in general position: f_x*, f_y* meet only on C


def _from_roots(lc, roots):
    a = [lc]
    for r in roots:
        a = P.mul(a, [-r, 1])
    return a


def test_multiplicity_split_by_counting_roots():
    # R and Q split over Z (plus an irreducible quadratic in Q): mult(Q, a) is the number
    # of times a appears among Q's roots, so c_k is the product of x - a over R's distinct
    # roots a that appear exactly k times
    rng = random.Random(21)
    for _ in range(60):
        ra = rng.sample(range(-8, 9), rng.randrange(1, 6))
        rroots = ra + [rng.choice(ra) for _ in range(rng.randrange(0, 3))]   # repeated roots
        qroots = [rng.randrange(-8, 9) for _ in range(rng.randrange(0, 7))]
        r = _from_roots(rng.choice([1, -3, 4]), rroots)
        q = P.mul(_from_roots(rng.choice([1, 2, -5]), qroots), [rng.randrange(1, 5), 0, 1])
        mult = {a: qroots.count(a) for a in ra}
        t = max(mult.values())
        want = [_from_roots(1, sorted(a for a in ra if mult[a] == k)) for k in range(t + 1)]
        assert S.multiplicity_split(r, q) == want, (rroots, qroots)


def test_multiplicity_split_against_sympy_factors():
    # a third route: the irreducible factors of R over Q (sympy), each weighed by how many
    # times it divides Q
    sympy = pytest.importorskip("sympy")
    x = sympy.symbols("x")
    rng = random.Random(22)

    def expr(c):
        return sum(int(v) * x ** i for i, v in enumerate(c))

    for _ in range(12):
        u = _rand(rng, rng.randrange(1, 3), -6, 6)
        v = _rand(rng, rng.randrange(1, 3), -6, 6)
        w = _rand(rng, rng.randrange(1, 3), -6, 6)
        r = P.mul(P.mul(u, v), w)
        q = P.mul(P.mul(P.mul(u, u), v), _rand(rng, 2, -6, 6))
        groups = {}
        for fac, _ in sympy.factor_list(expr(r))[1]:
            k, rest = 0, sympy.Poly(expr(q), x)
            fp = sympy.Poly(fac, x)
            while True:
                qq, rem = sympy.div(rest, fp)
                if not rem.is_zero:
                    break
                k, rest = k + 1, qq
            groups.setdefault(k, []).append(fac)
        t = max(groups)
        want = []
        for k in range(t + 1):
            c = sympy.Poly(sympy.Mul(*groups.get(k, [])), x)
            coeffs = [int(a) for a in reversed(c.all_coeffs())]
            want.append(P.scale(coeffs, -1) if coeffs[-1] < 0 else coeffs)
        assert S.multiplicity_split(r, q) == want


def test_bivariate_subresultant_polynomial():
    """S_d of two curves: S_0 is the resultant (Sylvester route), the top coefficient of S_d
    is sr_d (the psc route), and for a planted common factor C of degree k in y the
    S_j below k vanish and pp(S_k) = pp(C) up to sign."""
    rng = np.random.Generator(np.random.PCG64(21))
    for t in range(4):
        f = dense_curve(rng, 3 + t % 2, 8)
        g = dense_curve(rng, 2 + t % 3, 8)
        q = min(len(R.y_rows(f)), len(R.y_rows(g))) - 1
        assert S.subresultant_y(f, g, 0) == [R.res_y(f, g, route="zx")]
        sr = S.psc_y(f, g)
        for d in range(q):
            sd = S.subresultant_y(f, g, d)
            assert len(sd) == d + 1 and sd[d] == sr[d], (t, d)
    _, add, mul = _compose([1], 1, 1)
    for t in range(3):
        C = dense_curve(rng, 1 + t % 2, 5)
        U = dense_curve(rng, 2, 5)
        V = dense_curve(rng, 2, 5)
        A, B = mul(C, U), mul(C, V)
        k = len(R.y_rows(C)) - 1
        for j in range(k):
            assert all(not P.trim(s) for s in S.subresultant_y(A, B, j)), (t, j)
        Sk = S.subresultant_y(A, B, k)
        ppS = S._div_rows(Sk, S._content_rows(Sk))
        ppC = S._div_rows(R.y_rows(C), S._content_rows(R.y_rows(C)))
        assert ppS == ppC or ppS == [P.scale(r, -1) for r in ppC], t
    with pytest.raises(ValueError):
        S.subresultant_y([[1], [2], [3]], [[1], [1]], 1)


def test_bivariate_gcd_conventions():
    A = [[1, 2], [3, 0], [-5, 1]]
    rows = R.y_rows(A)
    assert S.bigcd_y([[0]], A) == S.bigcd_y(A, [[0]]) == rows
    assert S.bigcd_y([[0]], [[-c for c in r] for r in A]) == rows
    assert S.bigcd_y([[0]], [[0]]) == []
