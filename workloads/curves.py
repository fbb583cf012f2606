"""Seeded generators for the five workload shapes (see the package docstring).

Every generator takes an explicit integer seed and uses numpy's PCG64 bit generator, so
the same seed gives the same polynomials on x86 and Arm hosts.
"""

from __future__ import annotations

import numpy as np


def _rng(seed):
    return np.random.Generator(np.random.PCG64(int(seed)))


def uniform_signed(rng, bits, size):
    """``size`` Python ints drawn uniformly from ``[-2**(bits-1), 2**(bits-1) - 1]``."""
    if bits < 1:
        raise ValueError("bits must be >= 1")
    chunks = (bits + 31) // 32
    raw = rng.integers(0, 2**32, size=(size, chunks), dtype=np.uint64)
    mask = (1 << bits) - 1
    half = 1 << (bits - 1)
    out = []
    for row in raw:
        v = 0
        for k, c in enumerate(row):
            v |= int(c) << (32 * k)
        out.append((v & mask) - half)
    return out


def grid_shape(f):
    """(deg_y, deg_x) extents of a bivariate grid."""
    return len(f) - 1, (len(f[0]) - 1 if f else -1)


def dense_curve(rng, tdeg, bits, zero_prob=0.0, keep_top=True):
    """Dense curve of total degree ``tdeg``: every term x^i y^j with i + j <= tdeg.

    Coefficients are uniform signed ``bits``-bit integers.  With ``keep_top`` the
    coefficient of ``y**tdeg`` is redrawn until it is non-zero, so deg_y f = tdeg.
    With ``zero_prob`` > 0 each coefficient is then zeroed independently with that
    probability (the batched workload), and the actual degrees may drop.
    """
    n = tdeg + 1
    f = [[0] * n for _ in range(n)]
    vals = uniform_signed(rng, bits, n * (n + 1) // 2)
    k = 0
    for j in range(n):
        for i in range(n - j):
            f[j][i] = vals[k]
            k += 1
    if keep_top:
        while f[tdeg][0] == 0:
            f[tdeg][0] = uniform_signed(rng, bits, 1)[0]
    if zero_prob > 0.0:
        mask = rng.random(size=(n, n)) < zero_prob
        for j in range(n):
            for i in range(n - j):
                if mask[j, i]:
                    f[j][i] = 0
    return f


def random_univariate(rng, deg, bits):
    """Univariate polynomial of exact degree ``deg`` with signed ``bits``-bit coefficients."""
    a = uniform_signed(rng, bits, deg + 1)
    while a[deg] == 0:
        a[deg] = uniform_signed(rng, bits, 1)[0]
    return a


def d_dy(f):
    """Partial derivative in y of a bivariate grid (same x extent, one row fewer)."""
    if len(f) <= 1:
        return [[0] * len(f[0])]
    return [[j * c for c in f[j]] for j in range(1, len(f))]


def bimul(f, g):
    """Product of two bivariate grids (input construction for the degenerate cases)."""
    dyf, dxf = grid_shape(f)
    dyg, dxg = grid_shape(g)
    h = [[0] * (dxf + dxg + 1) for _ in range(dyf + dyg + 1)]
    for j1, row1 in enumerate(f):
        for i1, c1 in enumerate(row1):
            if c1 == 0:
                continue
            for j2, row2 in enumerate(g):
                hr = h[j1 + j2]
                for i2, c2 in enumerate(row2):
                    if c2:
                        hr[i1 + i2] += c1 * c2
    return h


def unimul(a, b):
    """Product of two univariate coefficient lists."""
    out = [0] * (len(a) + len(b) - 1)
    for i, x in enumerate(a):
        if x:
            for j, y in enumerate(b):
                out[i + j] += x * y
    return out


def highbit_variant(f, k):
    """Multiply every coefficient by 2**k and add one to the constant term (Sec. 6.2)."""
    h = [[c << k for c in row] for row in f]
    h[0][0] += 1
    return h


# --------------------------------------------------------------------------------------
# The five workload shapes
# --------------------------------------------------------------------------------------

def cfg1_pair(seed=1):
    """Dense pair of total degree 6 with uniform signed 10-bit coefficients."""
    rng = _rng(seed)
    return dense_curve(rng, 6, 10), dense_curve(rng, 6, 10)


def cfg2_pair(seed=1, tdeg=32, bits=32):
    """Discriminant-type pair (f, df/dy): f dense of total degree 32, signed 32-bit."""
    rng = _rng(seed)
    f = dense_curve(rng, tdeg, bits)
    return f, d_dy(f)


def cfg3_batch(seed=1, count=4096, deg_lo=4, deg_hi=24, bits_lo=8, bits_hi=64,
               zero_prob=0.2):
    """Batch of ``count`` pairs with independent total degrees in [deg_lo, deg_hi],
    a per-pair coefficient bit length in [bits_lo, bits_hi] and 20% of the
    coefficients zeroed."""
    rng = _rng(seed)
    pairs = []
    for _ in range(count):
        m = int(rng.integers(deg_lo, deg_hi + 1))
        n = int(rng.integers(deg_lo, deg_hi + 1))
        b = int(rng.integers(bits_lo, bits_hi + 1))
        f = dense_curve(rng, m, b, zero_prob=zero_prob, keep_top=False)
        g = dense_curve(rng, n, b, zero_prob=zero_prob, keep_top=False)
        pairs.append((f, g))
    return pairs


def cfg4_cases(seed=1, deg=12, bits=16, poison_prime=None):
    """Degenerate inputs.

    Returns a dict of name -> (f, g):

    * ``4a``: f = f1*f2 with f1, f2 dense of degree ``deg``; g = df/dy.
    * ``4b``: f = f1**2 * f2, g = df/dy (f has a square factor, so res_y(f, f_y) = 0).
    * ``4b2``: f = f1**2, g = df/dy (res_y = 0).
    * ``4c``: a curve whose leading y-coefficient is c*(x+2)(x+1)x(x-1)(x-3), so the
      resultant vanishes at vertical asymptotes; g = df/dy.
    * ``4d`` (only when ``poison_prime`` is given): the leading y-coefficient row of a
      dense curve multiplied by ``poison_prime``, so that prime divides lc_y f.
    """
    rng = _rng(seed)
    f1 = dense_curve(rng, deg, bits)
    f2 = dense_curve(rng, deg, bits)
    out = {}
    fa = bimul(f1, f2)
    out["4a"] = (fa, d_dy(fa))
    fb = bimul(bimul(f1, f1), f2)
    out["4b"] = (fb, d_dy(fb))
    fb2 = bimul(f1, f1)
    out["4b2"] = (fb2, d_dy(fb2))
    # leading coefficient c * prod(x - a) for a in (-2, -1, 0, 1, 3)
    lc = [uniform_signed(rng, 8, 1)[0] or 3]
    for a in (-2, -1, 0, 1, 3):
        nxt = [0] * (len(lc) + 1)
        for i, c in enumerate(lc):
            nxt[i + 1] += c
            nxt[i] -= a * c
        lc = nxt
    base = dense_curve(rng, deg, bits)
    width = max(len(lc), len(base[0]))
    fc = [row + [0] * (width - len(row)) for row in base]
    fc[deg] = lc + [0] * (width - len(lc))
    out["4c"] = (fc, d_dy(fc))
    if poison_prime is not None:
        fd = dense_curve(rng, deg, bits)
        fd[deg] = [c * poison_prime for c in fd[deg]]
        out["4d"] = (fd, d_dy(fd))
    return out


def cfg5_stream(seed=1, jobs=256, rate_hz=200.0, deg_lo=6, deg_hi=64, bits_lo=16,
                bits_hi=256, gcd_fraction=0.5):
    """Served stream: Poisson arrivals of resultant and gcd jobs.

    Each job is a dict with ``t`` (arrival time in seconds from the start), ``kind``
    ('resultant' or 'gcd') and its operands.  A resultant job is a dense pair of total
    degrees in [deg_lo, deg_hi] (drawn independently) and ``bits`` in [bits_lo, bits_hi];
    a gcd job is ``a = c*u``, ``b = c*v`` with a planted common factor ``c``.
    """
    rng = _rng(seed)
    t = 0.0
    out = []
    for _ in range(jobs):
        t += float(rng.exponential(1.0 / rate_hz))
        bits = int(rng.integers(bits_lo, bits_hi + 1))
        if rng.random() < gcd_fraction:
            d = int(rng.integers(deg_lo, deg_hi + 1))
            dc = int(rng.integers(1, max(2, d // 2) + 1))
            cb = max(2, bits // 2)
            c = random_univariate(rng, dc, cb)
            u = random_univariate(rng, d - dc, cb)
            v = random_univariate(rng, d - dc, cb)
            out.append({"t": t, "kind": "gcd", "a": unimul(c, u), "b": unimul(c, v),
                        "planted": c, "bits": bits})
        else:
            m = int(rng.integers(deg_lo, deg_hi + 1))
            n = int(rng.integers(deg_lo, deg_hi + 1))
            out.append({"t": t, "kind": "resultant", "f": dense_curve(rng, m, bits),
                        "g": dense_curve(rng, n, bits), "bits": bits})
    return out
