"""Parity of the univariate-resultant kernel (step (c)) with the oracle's Sylvester
determinant mod p, bit-exact, across degree classes and degenerate images."""

import random

import pytest

from oracle.numtheory import prime_table
from oracle.resultant import res_univariate_modp

pytestmark = pytest.mark.gpu

PRIMES = prime_table(64)


def _mul(x, y, p):
    out = [0] * (len(x) + len(y) - 1)
    for i, u in enumerate(x):
        for j, v in enumerate(y):
            out[i + j] = (out[i + j] + u * v) % p
    return out


@pytest.mark.parametrize("da,db", [(0, 0), (0, 5), (5, 0), (1, 1), (3, 2), (6, 6), (7, 3),
                                   (12, 11), (15, 15), (20, 5), (23, 24), (32, 31), (40, 47),
                                   (47, 47), (60, 64)])
def test_random_images(ctx, da, db):
    rng = random.Random(da * 100 + db)
    n = 300
    ps, A, B = [], [], []
    for i in range(n):
        p = PRIMES[i % len(PRIMES)]
        ps.append(p)
        A.append([rng.randrange(p) for _ in range(da + 1)])
        B.append([rng.randrange(p) for _ in range(db + 1)])
    got = ctx.uni_resultant_modp(ps, A, B)
    for i in range(0, n, 7 if da + db > 40 else 1):
        assert got[i] == res_univariate_modp(A[i], B[i], ps[i]), (i, A[i], B[i])


@pytest.mark.parametrize("da,db", [(4, 4), (9, 6), (16, 16), (31, 32)])
def test_degenerate_images(ctx, da, db):
    """vanishing leading coefficients, many zeros, small values, common factors"""
    rng = random.Random(7 + da)
    ps, A, B = [], [], []
    for i in range(240):
        p = PRIMES[i % 8]
        kind = i % 6
        hi = 3 if kind in (1, 2) else p
        a = [rng.randrange(hi) for _ in range(da + 1)]
        b = [rng.randrange(hi) for _ in range(db + 1)]
        if kind == 3:
            a[-1] = 0
        if kind == 4:
            a[-1] = 0
            b[-1] = 0
        if kind == 5:
            c = [rng.randrange(p) for _ in range(3)]
            a = _mul(a[: da - 1], c, p)
            b = _mul(b[: db - 1], c, p)
        ps.append(p)
        A.append(a)
        B.append(b)
    got = ctx.uni_resultant_modp(ps, A, B)
    for i in range(len(ps)):
        assert got[i] == res_univariate_modp(A[i], B[i], ps[i]), (i, A[i], B[i])
