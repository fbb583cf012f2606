"""Parity of the gcd in Z_p[x] and of the square-free part in Z[x] with the oracle."""

import numpy as np
import pytest

import paper_1201_1548_gb300 as bs
from oracle import gcd as G
from oracle import poly as P
from oracle import resultant as R
from workloads import cfg4_cases, random_univariate, unimul

pytestmark = pytest.mark.gpu


def _rng(seed):
    return np.random.Generator(np.random.PCG64(seed))


def _rand_modp(rng, deg, p):
    a = [int(x) for x in rng.integers(0, p, deg + 1)]
    while a[-1] == 0:
        a[-1] = int(rng.integers(1, p))
    return a


# ---- gcd in Z_p[x] ------------------------------------------------------------------

@pytest.mark.parametrize("which", [0, 1, 7])
def test_gcd_modp_planted_factors(ctx, which):
    p = bs.bs_prime_table(8)[which]
    rng = _rng(100 + which)
    for t in range(24):
        c = _rand_modp(rng, int(rng.integers(0, 40)), p)
        u = _rand_modp(rng, int(rng.integers(0, 60)), p)
        v = _rand_modp(rng, int(rng.integers(0, 60)), p)
        a = P.mod_p(P.mul(c, u), p)
        b = P.mod_p(P.mul(c, v), p)
        want = G.gcd_modp(a, b, p)
        assert ctx.gcd_modp(a, b, p) == want, t
        if t < 6:  # the Sylvester echelon route gives the same gcd
            assert G.echelon_gcd_modp(a, b, p) == want


def test_gcd_modp_edge_cases(ctx):
    p = bs.bs_prime_table(1)[0]
    assert ctx.gcd_modp([], [], p) == []
    assert ctx.gcd_modp([], [3, 6], p) == G.gcd_modp([], [3, 6], p)
    assert ctx.gcd_modp([3, 6], [], p) == G.gcd_modp([3, 6], [], p)
    assert ctx.gcd_modp([5], [1, 1], p) == [1]
    a = [1, 2, 3, 4, 5]
    assert ctx.gcd_modp(a, a, p) == G.gcd_modp(a, a, p)
    # small odd primes: the kernel is not limited to the table primes
    for q in (3, 5, 65537, 2147483647):
        rng = _rng(q)
        c = _rand_modp(rng, 5, q)
        a = P.mod_p(P.mul(c, _rand_modp(rng, 9, q)), q)
        b = P.mod_p(P.mul(c, _rand_modp(rng, 7, q)), q)
        assert ctx.gcd_modp(a, b, q) == G.gcd_modp(a, b, q), q


def test_gcd_modp_long(ctx):
    p = bs.bs_prime_table(3)[2]
    rng = _rng(7)
    c = _rand_modp(rng, 300, p)
    a = P.mod_p(P.mul(c, _rand_modp(rng, 900, p)), p)
    b = P.mod_p(P.mul(c, _rand_modp(rng, 700, p)), p)
    assert ctx.gcd_modp(a, b, p) == G.gcd_modp(a, b, p)


# ---- square-free part in Z[x] ---------------------------------------------------------

def _product(*fs):
    out = [1]
    for f in fs:
        out = unimul(out, f)
    return out


def test_squarefree_part_small_structured(ctx):
    rng = _rng(21)
    for t in range(30):
        u = random_univariate(rng, int(rng.integers(1, 6)), int(rng.integers(2, 40)))
        v = random_univariate(rng, int(rng.integers(1, 5)), int(rng.integers(2, 40)))
        w = random_univariate(rng, int(rng.integers(0, 4)), int(rng.integers(2, 40)))
        r = _product(u, v, v, w, w, w)
        if t % 3 == 1:
            r = [-x for x in r]
        if t % 4 == 2:
            r = [6 * x for x in r]
        assert ctx.squarefree_part(r) == G.squarefree_part(r), t


def test_squarefree_part_conventions(ctx):
    assert ctx.squarefree_part([7]) == [1]
    assert ctx.squarefree_part([-7, 0, 0]) == [1]          # leading zeros are ignored
    assert ctx.squarefree_part([3, 6]) == [1, 2]
    assert ctx.squarefree_part([-2, -4]) == [1, 2]         # positive leading coefficient
    r = _product(*([[-1, 1]] * 5))                          # (x - 1)^5
    assert ctx.squarefree_part(r) == [-1, 1]
    r = [0, 0, 0, 5]                                        # 5 x^3
    assert ctx.squarefree_part(r) == [0, 1]
    with pytest.raises(bs.BsError):
        ctx.squarefree_part([0, 0])


def test_squarefree_part_already_squarefree(ctx):
    rng = _rng(22)
    for d in (1, 2, 17, 32):
        r = random_univariate(rng, d, 30)
        assert ctx.squarefree_part(r) == G.squarefree_part(r)


def test_squarefree_part_wide_coefficients(ctx):
    rng = _rng(23)
    u = random_univariate(rng, 6, 300)
    v = random_univariate(rng, 4, 200)
    r = _product(u, v, v)
    assert ctx.squarefree_part(r) == G.squarefree_part(r)


def test_squarefree_part_rejects_prime_dividing_lc(ctx):
    # the first table prime divides lc(R): that prime is skipped and the reconstruction
    # runs on primes outside table order
    p0 = bs.bs_prime_table(1)[0]
    rng = _rng(24)
    u = random_univariate(rng, 3, 20)
    u[-1] *= p0
    v = random_univariate(rng, 4, 20)
    r = _product(u, v, v)
    assert ctx.squarefree_part(r) == G.squarefree_part(r)


def test_squarefree_part_of_resultants(ctx):
    # square-free parts of projections of degenerate curves (the resultant of f and f_y)
    cases = cfg4_cases(seed=3, deg=3, bits=8)
    for name in ("4a", "4c"):
        f, g = cases[name]
        res = R.res_y(f, g)
        assert res, name
        assert ctx.squarefree_part(res) == G.squarefree_part(res), name


def test_squarefree_part_large_degree_by_construction(ctx):
    # R = c u v^2 w^3 with random u, v, w (square-free and pairwise coprime): R* = pp(u v w)
    rng = _rng(25)
    u = random_univariate(rng, 150, 24)
    v = random_univariate(rng, 100, 24)
    w = random_univariate(rng, 60, 24)
    r = [-3 * x for x in _product(u, v, v, w, w, w)]
    want = P.primitive_part(_product(u, v, w))
    got = ctx.squarefree_part(r)
    assert got == want


# ---- gcd in Z[x] ---------------------------------------------------------------------

def test_gcd_z_planted_factors(ctx):
    rng = _rng(31)
    for t in range(30):
        c = random_univariate(rng, int(rng.integers(0, 8)), int(rng.integers(2, 60)))
        u = random_univariate(rng, int(rng.integers(0, 10)), int(rng.integers(2, 60)))
        v = random_univariate(rng, int(rng.integers(0, 10)), int(rng.integers(2, 60)))
        a, b = _product(c, u), _product(c, v)
        if t % 3 == 0:
            a = [6 * x for x in a]
            b = [-10 * x for x in b]
        assert ctx.gcd_z(a, b) == G.gcd_z(a, b), t


def test_gcd_z_conventions(ctx):
    assert ctx.gcd_z([], []) == []
    assert ctx.gcd_z([0, 0], [0]) == []
    assert ctx.gcd_z([], [-3, -6]) == [3, 6]
    assert ctx.gcd_z([4, 0, -2], []) == [-4, 0, 2]
    assert ctx.gcd_z([6], [4]) == [2]
    assert ctx.gcd_z([6], [1, 1]) == [1]
    assert ctx.gcd_z([2, 2], [4, 4]) == [2, 2]
    assert ctx.gcd_z([-2, -2], [4, 4]) == [2, 2]
    a = [3, -1, 4, 1, -5]
    assert ctx.gcd_z(a, a) == G.gcd_z(a, a)
    most_negative = [-(1 << 31)]                           # needs a wider limb when negated
    assert ctx.gcd_z(most_negative, []) == [1 << 31]


def test_gcd_z_wide_and_long(ctx):
    rng = _rng(32)
    c = random_univariate(rng, 6, 200)
    a = _product(c, random_univariate(rng, 8, 250))
    b = _product(c, random_univariate(rng, 7, 100))
    assert ctx.gcd_z(a, b) == G.gcd_z(a, b)
    # long inputs: the planted factor is the gcd with overwhelming probability
    c = random_univariate(rng, 120, 20)
    u = random_univariate(rng, 200, 20)
    v = random_univariate(rng, 150, 20)
    got = ctx.gcd_z(_product(c, u), _product(c, v))
    assert got == P.primitive_part(c)


def test_gcd_z_prime_dividing_lc(ctx):
    p0 = bs.bs_prime_table(1)[0]
    rng = _rng(33)
    c = random_univariate(rng, 3, 20)
    u = random_univariate(rng, 4, 20)
    u[-1] *= p0
    v = random_univariate(rng, 5, 20)
    a, b = _product(c, u), _product(c, v)
    assert ctx.gcd_z(a, b) == G.gcd_z(a, b)


def test_modgcd_batch_matches_single_calls(ctx):
    rng = _rng(34)
    jobs = []
    for t in range(24):
        c = random_univariate(rng, int(rng.integers(0, 6)), int(rng.integers(4, 80)))
        u = random_univariate(rng, int(rng.integers(1, 8)), int(rng.integers(4, 80)))
        v = random_univariate(rng, int(rng.integers(1, 8)), int(rng.integers(4, 80)))
        if t % 2:
            jobs.append((0, _product(c, u), _product(c, v)))
        else:
            jobs.append((1, _product(u, v, v), None))
    jobs.append((0, [], [5, 10]))
    jobs.append((1, [9], None))
    got = ctx.modgcd_batch(jobs)
    for (k, a, b), g in zip(jobs, got):
        want = G.gcd_z(a, b) if k == 0 else G.squarefree_part(a)
        assert g == want
        assert g == (ctx.gcd_z(a, b) if k == 0 else ctx.squarefree_part(a))


def test_gcd_z_partial_content_wider_than_the_result(ctx):
    # the inputs' contents are folded by several warps (one per 64 coefficients): with
    # a = 2^300 (x^200 + x) and b = 3 x^2 + 3, one warp sees a's coefficient 2^300 and no
    # coefficient of b, so its partial gcd is far wider than the one-limb result
    a = [0] * 201
    a[1] = a[200] = 1 << 300
    b = [3, 0, 3]
    assert ctx.gcd_z(a, b) == G.gcd_z(a, b) == [1]
    a2 = [6 * x for x in a]
    b2 = [4 * x for x in P.mul(b, [1, 0, 0, 1])]         # b (x^3 + 1): shares x + 1 with a
    assert ctx.gcd_z(a2, b2) == G.gcd_z(a2, b2)
