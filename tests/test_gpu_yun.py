"""Parity of the square-free factorisation (Yun's algorithm, Sec. 2.1) with the oracle.

Small and medium inputs are compared with the oracle's Yun factorisation factor by
factor.  Large inputs are checked against the properties that make the factorisation
unique: every r_i primitive with a positive leading coefficient, r_s not constant,
R = c prod r_i^i exactly, and each r_i square-free and the r_i pairwise coprime, both
certified modulo a prime that divides no leading coefficient."""

import numpy as np
import pytest

import paper_1201_1548_gb300 as bs
from oracle import gcd as G
from oracle import poly as P
from oracle import resultant as R
from workloads import cfg4_cases, random_univariate

pytestmark = pytest.mark.gpu


def _rng(seed):
    return np.random.Generator(np.random.PCG64(seed))


def _product(*fs):
    out = [1]
    for f in fs:
        out = P.mul(out, f)
    return out


def _certify(r, facs, p=2305843009213693951):
    """The factorisation properties that fix the result uniquely (p = 2^61 - 1)."""
    assert facs, "a non-constant polynomial has at least one factor"
    assert len(facs[-1]) > 1, "the last factor is not constant"
    prod = [1]
    for i, f in enumerate(facs, start=1):
        assert f == P.primitive_part(f), i
        for _ in range(i):
            prod = P.mul(prod, f)
    r = P.trim(r)
    c, rem = divmod(r[-1], prod[-1])
    assert rem == 0 and [c * x for x in prod] == r
    nonconst = [f for f in facs if len(f) > 1]
    for f in nonconst:
        assert f[-1] % p
        assert G.gcd_modp(f, P.derivative(f), p) == [1]
    for a in range(len(nonconst)):
        for b in range(a + 1, len(nonconst)):
            assert G.gcd_modp(nonconst[a], nonconst[b], p) == [1]


def test_yun_planted_multiplicities(ctx):
    rng = _rng(41)
    for t in range(24):
        u = random_univariate(rng, int(rng.integers(1, 6)), int(rng.integers(2, 40)))
        v = random_univariate(rng, int(rng.integers(1, 5)), int(rng.integers(2, 40)))
        w = random_univariate(rng, int(rng.integers(0, 4)), int(rng.integers(2, 40)))
        r = _product(u, v, v, w, w, w)
        if t % 3 == 1:
            r = [-x for x in r]
        if t % 4 == 2:
            r = [6 * x for x in r]
        assert ctx.squarefree_factorization(r) == G.yun(r), t


def test_yun_conventions(ctx):
    assert ctx.squarefree_factorization([7]) == []
    assert ctx.squarefree_factorization([-7, 0, 0]) == []           # leading zeros ignored
    assert ctx.squarefree_factorization([3, 6]) == [[1, 2]]
    assert ctx.squarefree_factorization([-2, -4]) == [[1, 2]]        # positive lc
    r = _product(*([[-1, 1]] * 5))                                    # (x - 1)^5
    assert ctx.squarefree_factorization(r) == [[1], [1], [1], [1], [-1, 1]]
    assert ctx.squarefree_factorization([0, 0, 0, 5]) == [[1], [1], [0, 1]]   # 5 x^3
    # a multiplicity that does not occur gives r_i = 1 inside the sequence
    u, w = [1, 0, 1], [-2, 1]
    assert ctx.squarefree_factorization(_product(u, w, w, w)) == [[1, 0, 1], [1], [-2, 1]]
    with pytest.raises(bs.BsError) as e:
        ctx.squarefree_factorization([0, 0])
    assert e.value.code == bs.BS_ERR_ZERO


def test_yun_high_multiplicities(ctx):
    a, b, c = [1, 1], [3, 0, 1], [-5, 2, 0, 1]
    r = _product(*([a] * 7 + [b] * 2 + [c] * 4))
    got = ctx.squarefree_factorization(r)
    assert got == G.yun(r)
    assert len(got) == 7 and got[1] == b and got[3] == c and got[6] == a


def test_yun_already_squarefree(ctx):
    rng = _rng(42)
    for d in (1, 2, 17, 32):
        r = random_univariate(rng, d, 30)
        assert ctx.squarefree_factorization(r) == [P.primitive_part(r)] == G.yun(r)


def test_yun_wide_coefficients(ctx):
    rng = _rng(43)
    u = random_univariate(rng, 6, 300)
    v = random_univariate(rng, 4, 200)
    r = [-15 * x for x in _product(u, v, v)]
    assert ctx.squarefree_factorization(r) == G.yun(r)


def test_yun_primes_dividing_lc_are_skipped(ctx):
    # lc(R) carries the squares of the first two table primes: they are skipped and the
    # reconstruction runs on primes outside table order
    p0, p1 = bs.bs_prime_table(2)
    rng = _rng(44)
    u = random_univariate(rng, 3, 20)
    u[-1] *= p0 * p1
    v = random_univariate(rng, 4, 20)
    r = _product(u, u, v)
    assert ctx.squarefree_factorization(r) == G.yun(r)


def test_yun_of_resultants(ctx):
    # projections of degenerate curves (the resultant of f and f_y), as BiProject splits them
    cases = cfg4_cases(seed=3, deg=3, bits=8)
    for name in ("4a", "4c"):
        f, g = cases[name]
        res = R.res_y(f, g)
        assert res, name
        got = ctx.squarefree_factorization(res)
        assert got == G.yun(res), name
    # 4a: R = res(f1 f2, (f1 f2)_y) carries the square factor res(f1, f2)^2
    assert len(ctx.squarefree_factorization(R.res_y(*cases["4a"]))) >= 2


def test_yun_batch_matches_single_calls(ctx):
    rng = _rng(45)
    polys = []
    for t in range(12):
        u = random_univariate(rng, int(rng.integers(1, 8)), int(rng.integers(2, 64)))
        v = random_univariate(rng, int(rng.integers(0, 5)), int(rng.integers(2, 64)))
        polys.append(_product(u, v, v) if t % 2 else _product(u, v, v, v, v))
    polys += [[5], [1, 1], _product([1, 1], [1, 1])]
    got = ctx.squarefree_factorization_batch(polys)
    assert got == [ctx.squarefree_factorization(r) for r in polys]
    assert got == [G.yun(r) for r in polys]


def test_yun_large_degree_certified(ctx):
    # R = -3 u v^2 w^3, deg R = 530: checked against the properties that fix the result
    rng = _rng(46)
    u = random_univariate(rng, 150, 24)
    v = random_univariate(rng, 100, 24)
    w = random_univariate(rng, 60, 24)
    r = [-3 * x for x in _product(u, v, v, w, w, w)]
    got = ctx.squarefree_factorization(r)
    assert got == [P.primitive_part(u), P.primitive_part(v), P.primitive_part(w)]
    _certify(r, got)


def test_yun_many_primes_certified(ctx):
    # deg R = 3150 with 1900-bit coefficients: Mignotte's bound needs more than 160 primes,
    # which the block reconstruction kernel lifts
    rng = _rng(47)
    u = random_univariate(rng, 300, 200)
    v = random_univariate(rng, 850, 500)
    r = _product(u, u, v, v, v)
    got = ctx.squarefree_factorization(r)
    assert got == [[1], P.primitive_part(u), P.primitive_part(v)]
    _certify(r, got)


def test_yun_inputs_wider_than_2048_bits(ctx):
    # 69-limb coefficients (a resultant fed back as input is this wide): compared with the
    # oracle, and with the square-free part of the same input
    rng = _rng(48)
    u = random_univariate(rng, 3, 1100)
    v = random_univariate(rng, 2, 100)
    r = _product(u, u, v)
    assert max(abs(x).bit_length() for x in r) > 2048
    want = G.yun(r)
    assert ctx.squarefree_factorization(r) == want
    assert ctx.squarefree_part(r) == G.squarefree_part(r)


def test_yun_wide_and_long_certified(ctx):
    # deg R = 250 with about 2600-bit coefficients
    rng = _rng(49)
    u = random_univariate(rng, 100, 1000)
    v = random_univariate(rng, 50, 600)
    r = [-x for x in _product(u, u, v)]
    got = ctx.squarefree_factorization(r)
    assert got == [P.primitive_part(v), P.primitive_part(u)]
    _certify(r, got)
    assert ctx.squarefree_part(r) == P.primitive_part(_product(u, v))


def test_contents_across_the_64_bit_boundary(ctx):
    # the images' contents are lc(R) / lc(r_i) times the content of R: multipliers of 20,
    # 40, 60 and 100 bits take the 32-bit, 64-bit and multi-limb paths of the warp gcd
    rng = _rng(50)
    u = random_univariate(rng, 5, 40)
    v = random_univariate(rng, 4, 40)
    base = _product(u, u, v)
    for bits in (20, 40, 60, 100):
        C = (1 << bits) - 3 * bits
        r = [C * x for x in base]
        assert ctx.squarefree_factorization(r) == G.yun(r), bits
        assert ctx.squarefree_part(r) == G.squarefree_part(r), bits
        a, b = [C * x for x in _product(u, v)], [(C + 2) * x for x in _product(u, u)]
        assert ctx.gcd_z(a, b) == G.gcd_z(a, b), bits
