"""Elementary number theory for the oracle: primality, the prime table, primitive roots.

The prime table follows this definition (the same one the CUDA planner implements on
its own): all primes p with 2**30 < p < 2**31 and p = 1 (mod 2**14), in two decreasing
runs: first those with 3p < 2**32, then the others.  The paper fixes neither the prime size
nor the evaluation points (Sec. 5.1, steps (a) and (b) leave both open); 31-bit primes with
a 2**14-th root of unity let every prime carry an evaluation set of up to 16384 points that
is a coset of the roots of unity, and the first run keeps a sum of three products of
residues below p * 2**32.
"""

from __future__ import annotations

PRIME_LOG_ORDER = 14          # p = 1 (mod 2**14)
PRIME_LO = 1 << 30
PRIME_HI = 1 << 31
PRIME_MID = (1 << 32) // 3    # the first run: p <= PRIME_MID, i.e. 3p < 2**32


def is_prime(n: int) -> bool:
    """Deterministic Miller-Rabin.

    For n < 4,759,123,141 the bases {2, 7, 61} are sufficient (Jaeschke 1993); above
    that the first twelve primes are used, which is deterministic below 3.3e24.
    """
    if n < 2:
        return False
    small = (2, 3, 5, 7, 11, 13, 17, 19, 23, 29, 31, 37)
    for q in small:
        if n == q:
            return True
        if n % q == 0:
            return False
    bases = (2, 7, 61) if n < 4_759_123_141 else small
    d, s = n - 1, 0
    while d % 2 == 0:
        d //= 2
        s += 1
    for a in bases:
        if a % n == 0:
            continue
        x = pow(a, d, n)
        if x in (1, n - 1):
            continue
        for _ in range(s - 1):
            x = x * x % n
            if x == n - 1:
                break
        else:
            return False
    return True


def prime_table(count: int, log_order: int = PRIME_LOG_ORDER):
    """First ``count`` primes of the table: p = 1 mod 2**log_order, 2**30 < p < 2**31, first
    those with p <= PRIME_MID in decreasing order, then the others in decreasing order."""
    step = 1 << log_order
    out = []
    for top, bottom in ((PRIME_MID, PRIME_LO), (PRIME_HI - 1, PRIME_MID)):
        q = (top - 1) // step
        while len(out) < count:
            p = q * step + 1
            if p <= bottom:
                break
            if p <= top and is_prime(p):
                out.append(p)
            q -= 1
    if len(out) < count:
        raise ValueError("prime table exhausted")
    return out


def factor_small(n: int):
    """Distinct prime factors of n by trial division (fine for n < 2**40)."""
    fs = []
    d = 2
    while d * d <= n:
        if n % d == 0:
            fs.append(d)
            while n % d == 0:
                n //= d
        d += 1 if d == 2 else 2
    if n > 1:
        fs.append(n)
    return fs


def primitive_root(p: int) -> int:
    """Smallest generator of the multiplicative group of Z_p (p prime)."""
    qs = factor_small(p - 1)
    g = 2
    while True:
        if all(pow(g, (p - 1) // q, p) != 1 for q in qs):
            return g
        g += 1


def root_of_unity(p: int, n: int) -> int:
    """A primitive n-th root of unity mod p (n a power of two dividing p - 1): g**((p-1)/n)."""
    if (p - 1) % n:
        raise ValueError("n does not divide p - 1")
    return pow(primitive_root(p), (p - 1) // n, p)


COSET_EXPONENT = 0x9E3779B9    # odd; the representative is a power of g with this exponent
COSET_MAX_LOG = 14            # transform sizes up to 2^14 (the primes are 1 mod 2^14)


def coset_representative(p: int) -> int:
    """c = g**e for the first e of E mod (p-1), E mod (p-1) + 2, ... with c**(2**14) != 1
    (g the smallest primitive root, E = COSET_EXPONENT): c lies outside the subgroup of
    every transform size.  It is not a small integer, unlike g (often 3), which would make
    x = g a point of every evaluation set."""
    g = primitive_root(p)
    e = COSET_EXPONENT % (p - 1)
    while True:
        c = pow(g, e, p)
        if pow(c, 1 << COSET_MAX_LOG, p) != 1:
            return c
        e = (e + 2) % (p - 1)


def coset_points(p: int, n: int):
    """The evaluation set c * w**t, t = 0..n-1, with c = coset_representative(p) and
    w = g**((p-1)/n) for the smallest primitive root g.  It avoids 0 and every n-th root of
    unity (in particular +-1), since c**n != 1."""
    g = primitive_root(p)
    c = coset_representative(p)
    w = pow(g, (p - 1) // n, p)
    pts = []
    x = c
    for _ in range(n):
        pts.append(x)
        x = x * w % p
    return pts


def inv_mod(a: int, p: int) -> int:
    a %= p
    if a == 0:
        raise ZeroDivisionError("no inverse of 0")
    return pow(a, p - 2, p)
