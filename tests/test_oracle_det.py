"""Pins for oracle.sylvester: the paper's Sylvester layout and three determinant routes."""

import os
import random

import numpy as np

from oracle.sylvester import (IntRing, PolyRing, det_bareiss, det_leibniz, det_modp,
                              sylvester)

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "sylvester_m4_n3.txt")


def _read_golden():
    blocks, cur = {}, None
    for line in open(GOLDEN):
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        if line in ("S", "GBT"):
            cur = blocks.setdefault(line, [])
            continue
        cur.append(line.split())
    return blocks


def test_sylvester_layout_matches_paper_example():
    """Sec. 5.1 worked example (m = 4, n = 3): S printed there is the transpose of the
    Sec. 2 row layout produced by ``sylvester``."""
    f = ["f0", "f1", "f2", "f3", "f4"]
    g = ["g0", "g1", "g2", "g3"]
    S = sylvester(f, g, zero="0")
    ST = [[S[j][i] for j in range(7)] for i in range(7)]
    assert ST == _read_golden()["S"]


def test_displacement_equation_of_paper_example():
    """S - Z_r S (Z_m (+) Z_n)^T = G B^T for the printed example, with symbols replaced by
    random integers; the right-hand side must equal the printed rank-2 pattern."""
    rng = random.Random(3)
    vals = {f"f{i}": rng.randrange(-50, 50) for i in range(5)}
    vals.update({f"g{i}": rng.randrange(-50, 50) for i in range(4)})
    vals["0"] = 0
    gold = _read_golden()
    S = np.array([[vals[x] for x in row] for row in gold["S"]], dtype=np.int64)
    r, m, n = 7, 4, 3
    Zr = np.eye(r, k=-1, dtype=np.int64)
    Zm = np.eye(n, k=-1, dtype=np.int64)   # the f block has n = 3 columns
    Zn = np.eye(m, k=-1, dtype=np.int64)   # the g block has m = 4 columns
    Zk = np.zeros((r, r), dtype=np.int64)
    Zk[:n, :n] = Zm
    Zk[n:, n:] = Zn
    lhs = S - Zr @ S @ Zk.T
    rhs = np.array([[vals[x] for x in row] for row in gold["GBT"]], dtype=np.int64)
    assert (lhs == rhs).all()
    assert np.linalg.matrix_rank(rhs.astype(float)) == 2


def test_three_determinant_routes_agree():
    rng = random.Random(11)
    for n in range(0, 7):
        for _ in range(6):
            M = [[rng.randrange(-9, 10) for _ in range(n)] for _ in range(n)]
            d1 = det_leibniz(M) if n else 1
            d2 = det_bareiss(M)
            assert d1 == d2
            if n:
                assert round(np.linalg.det(np.array(M, dtype=float))) == d1
            p = 2147483647
            assert det_modp(M, p) == d1 % p


def test_bareiss_singular_and_pivoting():
    M = [[0, 1, 2], [0, 3, 4], [5, 6, 7]]
    assert det_bareiss(M) == det_leibniz(M) == 5 * (1 * 4 - 2 * 3)
    assert det_bareiss([[1, 2], [2, 4]]) == 0
    assert det_modp([[0, 0], [1, 1]], 7) == 0


def test_bareiss_over_zx_matches_leibniz():
    rng = random.Random(5)
    for n in range(1, 5):
        M = [[[rng.randrange(-5, 6) for _ in range(rng.randrange(0, 3))] for _ in range(n)]
             for _ in range(n)]
        a = det_bareiss(M, PolyRing)
        b = det_leibniz(M, PolyRing)
        from oracle.poly import trim
        assert trim(a) == trim(b)
