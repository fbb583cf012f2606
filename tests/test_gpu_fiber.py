"""The fiber counts of Sec. 3.3 on the device against the oracle: the psc sequence modulo
one prime, the exact point count N with its decomposition of R*, and the lower bound N^-,
on split curves (whose fibers are counted directly) and dense curves."""

import numpy as np
import pytest

import paper_1201_1548_gb300 as bs
from oracle import resultant as R
from oracle import subresultant as S
from workloads import dense_curve

pytestmark = pytest.mark.gpu


def _rng(seed):
    return np.random.Generator(np.random.PCG64(seed))


def test_psc_modp_matches_oracle(ctx):
    rng = _rng(61)
    for t in range(8):
        f = dense_curve(rng, int(rng.integers(2, 7)), int(rng.integers(4, 60)))
        g = dense_curve(rng, int(rng.integers(2, 7)), int(rng.integers(4, 60)))
        p, res = ctx.psc_modp(f, g)
        assert p == bs.bs_prime_table(1)[0]           # no leading coefficient vanishes mod p
        assert res == S.psc_y_modp(f, g, p), t


def test_psc_modp_skips_a_rejected_prime(ctx):
    p0 = bs.bs_prime_table(1)[0]
    rng = _rng(62)
    f = dense_curve(rng, 4, 12)
    f[-1] = [c * p0 for c in f[-1]]                    # lc_y f = 0 mod the first prime
    g = S.d_dy(f)
    p, res = ctx.psc_modp(f, g)
    assert p != p0
    assert res == S.psc_y_modp(f, g, p)


SPLIT = [
    [[0, 1], [0, -1], [0, 2]],                          # three lines through the origin
    [[0, 1], [0, -1], [2, 1], [1, 0]],
    [[1, 1], [3, -1], [0, 2], [4, -2], [-2, 3]],
    [[0, 1], [0, -1], [0, 2], [0, 3], [5, 0]],          # four concurrent lines
]


@pytest.mark.parametrize("branches", SPLIT)
def test_fiber_count_split_curves(ctx, branches):
    f = S.split_curve(branches)
    want_degs, want_N = S.fiber_decomposition(f)
    assert want_N == S.split_curve_fiber_count(branches)
    degs, N, p = ctx.fiber_count(f)
    assert (degs, N, p) == (want_degs, want_N, 0)
    degs1, lb, p1 = ctx.fiber_count(f, mode=1)
    assert p1 > 0
    assert (degs1, lb) == S.fiber_lower_bound_modp(f, p1)
    assert lb <= N


def test_fiber_count_dense_curves(ctx):
    rng = _rng(63)
    for t in range(5):
        f = dense_curve(rng, 3 + t % 3, 12)           # constant leading coefficient in y
        want = S.fiber_decomposition(f)
        degs, N, _ = ctx.fiber_count(f)
        assert (degs, N) == want, t
        degs1, lb, p = ctx.fiber_count(f, mode=1)
        assert (degs1, lb) == S.fiber_lower_bound_modp(f, p), t


def test_fiber_count_in_x(ctx):
    f = S.split_curve([[0, 1], [0, -1], [3, 2]])
    ft = R.transpose(f)                                 # the same curve with x and y exchanged
    assert ctx.fiber_count(ft, var=0) == ctx.fiber_count(f, var=1)


def test_fiber_count_rejects_bad_curves(ctx):
    # a vertical asymptote: the leading coefficient in y is x
    with pytest.raises(bs.BsError) as e:
        ctx.fiber_count([[1, 0], [0, 0], [0, 1]])
    assert e.value.code == bs.BS_ERR_ARG
    # a square factor: R = res(f, f_y) = 0
    f = S.split_curve([[0, 1], [0, 1], [2, 0]])
    with pytest.raises(bs.BsError) as e:
        ctx.fiber_count(f)
    assert e.value.code == bs.BS_ERR_ZERO
    # linear in y: no critical values
    assert ctx.fiber_count([[1, 2, 3], [1, 0, 0]]) == ([], 0, 0)


def _compose(c1d, a, b):
    """c(a x + b y) as rows by powers of y, with the row helpers."""
    from oracle import poly as P

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


def _grid(rows):
    w = max(len(r) for r in rows)
    return [list(r) + [0] * (w - len(r)) for r in rows]


def _teissier_family(rng, deg_p, deg_k):
    """f = P(x+y)^2 K(x-y) + c with deg P = deg_p, deg K = deg_k (total degree
    2 deg_p + deg_k): f_x and f_y share the factor P(x+y), so d = deg_p."""
    pc = [rng.randrange(-4, 5) for _ in range(deg_p)] + [rng.choice([1, 2, -3])]
    kc = [rng.randrange(-4, 5) for _ in range(deg_k)] + [rng.choice([1, -1, 2])]
    Pp, add, mul = _compose(pc, 1, 1)
    Kk, _, _ = _compose(kc, 1, -1)
    return _grid(add(mul(mul(Pp, Pp), Kk), [[rng.randrange(1, 9)]]))


@pytest.mark.parametrize("deg_p,deg_k", [(1, 2), (2, 2), (3, 2), (3, 3), (4, 1)])
def test_teissier_q_exact_with_a_common_factor(ctx, deg_p, deg_k):
    """Q = res(f_x / h, f_y / h; y) and h = gcd(f_x, f_y) exactly (not up to a constant)
    on the family P(x+y)^2 K(x-y) + c up to total degree 10."""
    import random
    rng = random.Random(640 + 10 * deg_p + deg_k)
    f = _teissier_family(rng, deg_p, deg_k)
    want, wd = S.teissier_q(f)
    Q, d = ctx.teissier_q(f)
    assert d == wd >= deg_p                                # P(x+y) divides f_x and f_y
    assert Q == want
    fx, fy = S.d_dx(f), S.d_dy(f)
    assert ctx.gcd_bivariate(fx, fy) == S.bigcd_y(fx, fy)


def test_teissier_q_exact_dense_curves(ctx):
    """Dense curves of total degree 8 and 9, one with a vertical asymptote (a non-constant
    leading coefficient in y).  There res(f_x, f_y; y) != 0, so f_x and f_y have no common
    factor of positive degree in y, h is the gcd of their contents and
    Q = res(f_x / h, f_y / h; y) (the oracle's primitive remainder sequence is too slow at
    this degree; these are the same definitions by the resultant's zero criterion)."""
    from oracle import gcd as G
    from oracle import poly as P
    rng = _rng(65)
    for t in range(3):
        f = dense_curve(rng, 8 + t % 2, 10)
        if t == 2:
            f[-1] = [0, 3] + [0] * (len(f[-1]) - 2)       # lc_y f = 3 x
        fx, fy = S.d_dx(f), S.d_dy(f)
        assert R.res_y(fx, fy)                             # no common factor in y
        h = G.gcd_z(G.content_rows(R.y_rows(fx)), G.content_rows(R.y_rows(fy)))
        want = R.res_y([P.exact_div_z(r, h) for r in R.y_rows(fx)],
                       [P.exact_div_z(r, h) for r in R.y_rows(fy)])
        assert ctx.teissier_q(f) == (want, 0), t
        assert ctx.gcd_bivariate(fx, fy) == [h], t


def test_teissier_q_in_x(ctx):
    import random
    f = _teissier_family(random.Random(66), 2, 2)
    ft = R.transpose(f)
    assert ctx.teissier_q(ft, var=0) == ctx.teissier_q(f, var=1)


def test_gcd_bivariate_planted_factors(ctx):
    """gcd in Z[x, y] of A = C U and B = C V against the oracle's primitive PRS: C with a
    content in x, a non-constant leading coefficient in y, degrees 1..3 in y; both
    variables; coprime pairs (the gcd of the contents alone)."""
    rng = _rng(67)
    _, add, mul = _compose([1], 1, 1)
    for t in range(6):
        C = dense_curve(rng, 1 + t % 3, 6, keep_top=False)
        if t % 2:
            C = mul(C, [[1, 2]])                           # content 1 + 2x
        C[-1][-1] = C[-1][-1] or 5
        U = dense_curve(rng, 2 + t % 2, 6)
        V = dense_curve(rng, 3, 6)
        A, B = _grid(mul(C, U)), _grid(mul(C, V))
        assert ctx.gcd_bivariate(A, B) == S.bigcd_y(A, B), t
        At, Bt = R.transpose(A), R.transpose(B)
        assert ctx.gcd_bivariate(At, Bt, var=0) == S.bigcd_y(A, B), t
    for t in range(3):                                      # coprime: the gcd of the contents
        A = _grid(mul(dense_curve(rng, 4, 8), [[2, 6]]))
        B = _grid(mul(dense_curve(rng, 5, 8), [[3, 9]]))
        assert ctx.gcd_bivariate(A, B) == S.bigcd_y(A, B) == [[1, 3]], t


def test_gcd_bivariate_conventions(ctx):
    A = [[1, 2], [3, 0], [-5, 1]]
    assert ctx.gcd_bivariate([[0]], A) == S.bigcd_y([[0]], A)
    assert ctx.gcd_bivariate([[-c for c in r] for r in A], [[0]]) == S.bigcd_y(A, [[0]])
    assert ctx.gcd_bivariate([[0]], [[0]]) == []
    assert ctx.gcd_bivariate(A, A) == S.bigcd_y(A, A)         # all sr_i vanish
    Am = [[-c for c in r] for r in A]
    assert ctx.gcd_bivariate(A, _grid(Am)) == S.bigcd_y(A, Am)


def test_subresultant_polynomial(ctx):
    """S_d(f, g) for every d of random pairs and of pairs with a planted common factor,
    against the oracle's points route."""
    rng = _rng(68)
    _, add, mul = _compose([1], 1, 1)
    pairs = [(dense_curve(rng, 4, 10), dense_curve(rng, 3, 10)),
             (dense_curve(rng, 5, 6, zero_prob=0.2), dense_curve(rng, 5, 6))]
    C = dense_curve(rng, 2, 5)
    pairs.append((_grid(mul(C, dense_curve(rng, 2, 5))), _grid(mul(C, dense_curve(rng, 3, 5)))))
    for t, (f, g) in enumerate(pairs):
        q = min(len(R.y_rows(f)), len(R.y_rows(g))) - 1
        for d in range(q):
            assert ctx.subresultant(f, g, d) == S.subresultant_y(f, g, d), (t, d)
    with pytest.raises(bs.BsError) as e:
        ctx.subresultant(pairs[0][0], pairs[0][1], 3)
    assert e.value.code == bs.BS_ERR_ARG


@pytest.mark.parametrize("branches", SPLIT)
def test_fiber_upper_bound(ctx, branches):
    f = S.split_curve(branches)
    _, N, _ = ctx.fiber_count(f)
    degs, ub, p = ctx.fiber_count(f, mode=2)
    assert degs == [] and p > 0
    assert ub == S.fiber_upper_bound_modp(f, p)
    _, lb, _ = ctx.fiber_count(f, mode=1)
    assert lb <= N <= ub


def test_fiber_upper_bound_dense(ctx):
    rng = _rng(66)
    for t in range(3):
        f = dense_curve(rng, 3 + t % 2, 10)
        _, ub, p = ctx.fiber_count(f, mode=2)
        assert ub == S.fiber_upper_bound_modp(f, p), t


def _from_roots(lc, roots):
    from oracle import poly as P
    a = [lc]
    for r in roots:
        a = P.mul(a, [-r, 1])
    return a


def test_root_multiplicity_split_polynomials(ctx):
    import random
    from oracle import poly as P
    rng = random.Random(67)
    for t in range(12):
        ra = rng.sample(range(-30, 31), rng.randrange(1, 9))
        rroots = ra + [rng.choice(ra) for _ in range(rng.randrange(0, 3))]
        qroots = [rng.choice(ra) if rng.random() < 0.6 else rng.randrange(-30, 31)
                  for _ in range(rng.randrange(1, 12))]
        r = _from_roots(rng.choice([1, -3, 7]), rroots)
        q = P.mul(_from_roots(rng.choice([1, 2, -5]), qroots), [rng.randrange(1, 9), 0, 1])
        assert ctx.root_multiplicity(r, q) == S.multiplicity_split(r, q), t


def test_root_multiplicity_random_factors(ctx):
    # dense factors with wide coefficients: R = u v w (square-free in general), Q = u^3 v z
    from oracle import poly as P
    from workloads import random_univariate
    rng = _rng(68)
    for t in range(4):
        u, v, w, z = (random_univariate(rng, int(rng.integers(2, 7)), int(rng.integers(8, 70)))
                      for _ in range(4))
        r = P.mul(P.mul(u, v), w)
        q = P.mul(P.mul(P.mul(P.mul(u, u), u), v), z)
        got = ctx.root_multiplicity(r, q)
        assert got == S.multiplicity_split(r, q), t
        assert len(got) >= 4 and P.deg(got[3]) > 0, t       # the roots of u: multiplicity 3


def test_root_multiplicity_of_teissier_q(ctx):
    # the use of Sec. 3.3: R = res(f, f_y) and Teissier's Q of curves with singular points
    from oracle import resultant as Rm
    import random
    rng = random.Random(69)
    cases = [S.split_curve(b) for b in SPLIT[:3]]
    for _ in range(2):
        pc = [rng.randrange(-4, 5) or 1 for _ in range(rng.randrange(2, 4))]
        kc = [rng.randrange(-4, 5) or 1 for _ in range(rng.randrange(2, 4))]
        Pp, add, mul = _compose(pc, 1, 1)
        Kk, _, _ = _compose(kc, 1, -1)
        cases.append(_grid(add(mul(mul(Pp, Pp), Kk), [[rng.randrange(1, 9)]])))
    for t, f in enumerate(cases):
        Rr = Rm.res_y(f, S.d_dy(f))
        Q, _ = S.teissier_q(f)
        assert ctx.root_multiplicity(Rr, Q) == S.multiplicity_split(Rr, Q), t


def test_root_multiplicity_edge_cases(ctx):
    assert ctx.root_multiplicity([-6, 1, 1], [5]) == [[-6, 1, 1]]          # Q constant
    assert ctx.root_multiplicity([7], [1, 2, 1]) == [[1]]                   # R constant
    # R = 4 x^2 (R* = x), Q = x^3: the one root has multiplicity 3 in Q
    assert ctx.root_multiplicity([0, 0, 4], [0, 0, 0, 1]) == [[1], [1], [1], [0, 1]]
    for r, q in (([], [1, 1]), ([1, 1], []), ([0, 0], [1, 1])):
        with pytest.raises(bs.BsError) as e:
            ctx.root_multiplicity(r, q)
        assert e.value.code == bs.BS_ERR_ZERO
