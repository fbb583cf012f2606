"""The seeded input generators against the recipes they state: value ranges, shapes,
degrees, zeroing rates, the degenerate constructions and the served stream's arrival
process.  Every parity test and the benchmark draw their inputs from these."""

import numpy as np
import pytest

from oracle import poly as P
from workloads import curves as W


def _rng(seed):
    return np.random.Generator(np.random.PCG64(seed))


@pytest.mark.parametrize("bits", [1, 2, 8, 10, 31, 32, 33, 64, 256])
def test_uniform_signed_range(bits):
    vals = W.uniform_signed(_rng(bits), bits, 4000)
    lo, hi = -(1 << (bits - 1)), (1 << (bits - 1)) - 1
    assert all(lo <= v <= hi for v in vals)
    if bits <= 8:                                  # small ranges: both ends are drawn
        assert min(vals) == lo and max(vals) == hi
    else:                                          # wide ranges: both signs, large values
        assert min(vals) < lo // 2 and max(vals) > hi // 2


def _check_dense(f, tdeg, bits, keep_top=True):
    assert len(f) == tdeg + 1 and all(len(r) == tdeg + 1 for r in f)
    lim = 1 << (bits - 1)
    for j, row in enumerate(f):
        for i, c in enumerate(row):
            if i + j > tdeg:
                assert c == 0
            else:
                assert -lim <= c < lim
    if keep_top:
        assert f[tdeg][0] != 0


def test_cfg1_and_cfg2_shapes():
    for seed in (1, 2, 3):
        f, g = W.cfg1_pair(seed)
        _check_dense(f, 6, 10)
        _check_dense(g, 6, 10)
        assert sum(1 for r in f for c in r if c) >= 20     # 28 terms, few zero draws
    f, g = W.cfg2_pair(1)
    _check_dense(f, 32, 32)
    assert g == W.d_dy(f) and len(g) == 32
    assert g[31][0] == 32 * f[32][0]


def test_generators_are_deterministic():
    assert W.cfg1_pair(7) == W.cfg1_pair(7) and W.cfg1_pair(7) != W.cfg1_pair(8)
    assert W.cfg3_batch(seed=5, count=20) == W.cfg3_batch(seed=5, count=20)


def test_cfg3_batch_recipe():
    pairs = W.cfg3_batch(seed=2, count=300)
    zeros = total = 0
    degs, bits_seen = set(), set()
    for f, g in pairs:
        for h in (f, g):
            t = len(h) - 1
            assert 4 <= t <= 24
            degs.add(t)
            for j, row in enumerate(h):
                for i, c in enumerate(row):
                    if i + j <= t:
                        total += 1
                        zeros += c == 0
                        if c:
                            bits_seen.add(abs(c).bit_length())
    assert degs == set(range(4, 25))
    assert 0.18 < zeros / total < 0.22                 # 20 % zeroed (plus rare zero draws)
    assert max(bits_seen) == 63 and min(bits_seen) < 8  # signed 64-bit: magnitudes < 2^63


def _eval_row(row, x):
    return sum(c * x ** i for i, c in enumerate(row))


def test_cfg4_constructions():
    p = 2147483647
    cases = W.cfg4_cases(seed=3, poison_prime=p)
    f1f2, _ = cases["4a"]
    assert len(f1f2) - 1 == 24                          # deg_y (f1 f2) = 12 + 12
    fb, gb = cases["4b"]
    assert len(fb) - 1 == 36 and gb == W.d_dy(fb)
    fc, _ = cases["4c"]
    lc = fc[-1]
    assert all(_eval_row(lc, a) == 0 for a in (-2, -1, 0, 1, 3))
    assert _eval_row(lc, 2) != 0
    fd, _ = cases["4d"]
    assert any(fd[-1]) and all(c % p == 0 for c in fd[-1])


def test_cfg5_stream_recipe():
    rate = 200.0
    jobs = W.cfg5_stream(seed=4, jobs=600, rate_hz=rate)
    t = [j["t"] for j in jobs]
    assert all(b > a for a, b in zip(t, t[1:]))
    gaps = np.diff([0.0] + t)
    assert 0.8 / rate < gaps.mean() < 1.2 / rate       # exponential gaps of mean 1 / rate
    kinds = [j["kind"] for j in jobs]
    assert 0.4 < kinds.count("gcd") / len(kinds) < 0.6
    for j in jobs:
        assert 16 <= j["bits"] <= 256
        if j["kind"] == "gcd":
            c = j["planted"]
            assert len(c) >= 2                         # a non-constant planted factor
            for x in (j["a"], j["b"]):                 # c divides a and b exactly
                assert P.exact_div_z(x, c)
        else:
            for h in (j["f"], j["g"]):
                assert 6 <= len(h) - 1 <= 64 and h[-1][0] != 0
