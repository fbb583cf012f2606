"""Seeded synthetic inputs shared by the tests, the benchmark and the oracle's callers.

This package only draws random integer polynomials of the shapes used in the paper's
experiments (dense total-degree-m curves with uniform signed b-bit coefficients, Sec. 6
"random curves"; the high-bit variant that multiplies by 2^k and adds one to the
constant term, Sec. 6.2) and builds a few structured inputs from them (a y-derivative,
a product of two curves, a planted common factor).  It contains none of the
resultant, gcd, reduction or reconstruction arithmetic of the method itself.

Polynomial layouts used everywhere in this repository:

* bivariate ``f``: list of rows, ``f[j][i]`` is the coefficient of ``x**i * y**j``
  (a dense ``(deg_y + 1) x (deg_x + 1)`` grid of Python ints);
* univariate ``a``: list of coefficients in ascending order, ``a[i]`` of ``x**i``.
"""

from .curves import (  # noqa: F401
    uniform_signed,
    dense_curve,
    random_univariate,
    d_dy,
    bimul,
    unimul,
    grid_shape,
    cfg1_pair,
    cfg2_pair,
    cfg3_batch,
    cfg4_cases,
    cfg5_stream,
    highbit_variant,
)
