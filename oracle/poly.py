"""Dense univariate polynomial arithmetic over Z, Q (Fraction) and Z_p.

Coefficient lists are in ascending order (``a[i]`` is the coefficient of x**i); the
zero polynomial is the empty list and has degree -1.
"""

from __future__ import annotations

from fractions import Fraction
from math import gcd


def trim(a):
    a = list(a)
    while a and a[-1] == 0:
        a.pop()
    return a


def deg(a):
    return len(trim(a)) - 1


def add(a, b):
    n = max(len(a), len(b))
    return trim([(a[i] if i < len(a) else 0) + (b[i] if i < len(b) else 0) for i in range(n)])


def sub(a, b):
    n = max(len(a), len(b))
    return trim([(a[i] if i < len(a) else 0) - (b[i] if i < len(b) else 0) for i in range(n)])


def mul(a, b):
    if not a or not b:
        return []
    out = [0] * (len(a) + len(b) - 1)
    for i, x in enumerate(a):
        if x:
            for j, y in enumerate(b):
                out[i + j] += x * y
    return trim(out)


def scale(a, c):
    return trim([c * x for x in a])


def evaluate(a, x):
    acc = 0
    for c in reversed(a):
        acc = acc * x + c
    return acc


def derivative(a):
    return trim([i * a[i] for i in range(1, len(a))])


def exact_div_z(a, b):
    """Quotient a / b in Z[x]; raises if b does not divide a exactly."""
    a = trim(a)
    b = trim(b)
    if not b:
        raise ZeroDivisionError("division by the zero polynomial")
    if not a:
        return []
    da, db = len(a) - 1, len(b) - 1
    if da < db:
        raise ArithmeticError("inexact polynomial division")
    q = [0] * (da - db + 1)
    r = list(a)
    lb = b[-1]
    for k in range(da - db, -1, -1):
        c = r[k + db]
        if c % lb:
            raise ArithmeticError("inexact polynomial division")
        c //= lb
        q[k] = c
        if c:
            for i in range(db + 1):
                r[k + i] -= c * b[i]
    if any(r):
        raise ArithmeticError("inexact polynomial division")
    return trim(q)


def divmod_field(a, b, inv, reduce):
    """Division with remainder over a field; ``inv`` inverts a scalar, ``reduce`` normalises."""
    a = [reduce(x) for x in a]
    a = trim(a)
    b = trim([reduce(x) for x in b])
    if not b:
        raise ZeroDivisionError("division by the zero polynomial")
    db = len(b) - 1
    ilb = inv(b[-1])
    q = [0] * max(len(a) - db, 0)
    r = list(a)
    for k in range(len(a) - 1 - db, -1, -1):
        c = reduce(r[k + db] * ilb)
        q[k] = c
        if c:
            for i in range(db + 1):
                r[k + i] = reduce(r[k + i] - c * b[i])
    return trim(q), trim(r)


def divmod_q(a, b):
    return divmod_field([Fraction(x) for x in a], [Fraction(x) for x in b],
                        lambda x: 1 / x, lambda x: x)


def divmod_p(a, b, p):
    return divmod_field(a, b, lambda x: pow(x % p, p - 2, p), lambda x: x % p)


def content(a):
    c = 0
    for x in a:
        c = gcd(c, x)
    return c


def primitive_part(a):
    """a / content(a), with a positive leading coefficient (0 stays 0)."""
    a = trim(a)
    if not a:
        return []
    c = content(a)
    if a[-1] < 0:
        c = -c
    return [x // c for x in a]


def mod_p(a, p):
    return trim([x % p for x in a])


def monic_p(a, p):
    a = mod_p(a, p)
    if not a:
        return []
    il = pow(a[-1], p - 2, p)
    return [x * il % p for x in a]


def fraction_to_primitive_z(a):
    """Clear denominators of a Q[x] polynomial and return its primitive part."""
    a = trim(a)
    if not a:
        return []
    den = 1
    for x in a:
        den = den * Fraction(x).denominator // gcd(den, Fraction(x).denominator)
    return primitive_part([int(Fraction(x) * den) for x in a])
