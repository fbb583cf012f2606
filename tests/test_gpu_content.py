"""Content removal (Sec. 4) on the device against the oracle: the gcd in Z[x] of the rows of
f with respect to either variable, and the rows of the primitive part."""

import numpy as np
import pytest

import paper_1201_1548_gb300 as bs
from oracle import gcd as G
from oracle import poly as P
from oracle import resultant as R
from workloads import dense_curve, random_univariate

pytestmark = pytest.mark.gpu


def _rng(seed):
    return np.random.Generator(np.random.PCG64(seed))


def _times_univariate(f, h):
    """f(x, y) * h(x) for a grid f (rows by powers of y)."""
    rows = [P.mul(row, h) for row in f]
    w = max(len(r) for r in rows)
    return [r + [0] * (w - len(r)) for r in rows]


def _rows(f, var):
    return [P.trim(r) for r in (f if var == 1 else R.transpose(f))]


@pytest.mark.parametrize("var", [1, 0])
def test_content_planted_factor(ctx, var):
    rng = _rng(70 + var)
    for t in range(6):
        g = dense_curve(rng, int(rng.integers(2, 6)), int(rng.integers(4, 40)))
        h0 = random_univariate(rng, int(rng.integers(0, 4)), 20)
        f = _times_univariate(g, h0) if var == 1 else R.transpose(_times_univariate(R.transpose(g), h0))
        if t % 2:
            f = [[-6 * c for c in row] for row in f]
        h, rows = ctx.content(f, var)
        want_h, want_rows = G.primitive_rows(_rows(f, var))
        assert h == want_h, t
        assert rows == [P.trim(r) for r in want_rows], t


def test_content_conventions(ctx):
    f = [[0, 0, 3], [0, 0, 0], [0, 0, -6]]            # 3 x^2 - 6 x^2 y^2
    h, rows = ctx.content(f)
    assert h == [0, 0, 3] and rows == [[1], [], [-2]]
    assert ctx.content([[5, 0], [0, 0]]) == ([5], [[1]])
    g = [[1, 2], [3, 4]]                              # trivial content
    assert ctx.content(g) == ([1], [[1, 2], [3, 4]])
    with pytest.raises(bs.BsError) as e:
        ctx.content([[0, 0], [0, 0]])
    assert e.value.code == bs.BS_ERR_ZERO


def test_content_wide_coefficients(ctx):
    rng = _rng(72)
    g = dense_curve(rng, 4, 300)
    h0 = random_univariate(rng, 3, 200)
    f = _times_univariate(g, h0)
    h, rows = ctx.content(f)
    want_h, want_rows = G.primitive_rows(_rows(f, 1))
    assert h == want_h and rows == [P.trim(r) for r in want_rows]
