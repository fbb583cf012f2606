"""Pins for oracle.numtheory: Miller-Rabin, the prime table, primitive roots, cosets."""

import random

import pytest

from oracle import numtheory as nt


def _trial(n):
    if n < 2:
        return False
    d = 2
    while d * d <= n:
        if n % d == 0:
            return False
        d += 1
    return True


def test_is_prime_matches_trial_division_small():
    for n in range(0, 5000):
        assert nt.is_prime(n) == _trial(n), n


def test_is_prime_random_31_bit():
    rng = random.Random(7)
    for _ in range(300):
        n = rng.randrange(1 << 30, 1 << 31)
        assert nt.is_prime(n) == _trial(n), n


def test_strong_pseudoprimes_rejected():
    # 2047 is a base-2 strong pseudoprime; 3215031751 is one to bases 2, 3, 5 and 7;
    # 25326001 to bases 2, 3 and 5; all composite.
    for n in (2047, 3215031751, 25326001, 561, 1105, 1729):
        assert not nt.is_prime(n)


def test_prime_table_definition():
    """Two decreasing runs of primes p = 1 mod 2^14 in (2^30, 2^31): first those with
    3p < 2^32, then the rest; checked by trial division at the runs' starts, between
    consecutive entries and across the boundary, and by counting the whole table."""
    step = 1 << nt.PRIME_LOG_ORDER
    full = nt.prime_table(6213)
    with pytest.raises(ValueError):
        nt.prime_table(6214)
    n1 = sum(1 for p in full if 3 * p < (1 << 32))
    assert all(3 * p < (1 << 32) for p in full[:n1]) and all(3 * p > (1 << 32) for p in full[n1:])
    assert all((1 << 30) < p < (1 << 31) and p % step == 1 for p in full)
    assert all(full[i] > full[i + 1] for i in range(n1 - 1))
    assert all(full[i] > full[i + 1] for i in range(n1, len(full) - 1))
    assert len(set(full)) == len(full)
    for run in (full[:6], full[n1:n1 + 6]):
        for p in run[:5]:
            assert _trial(p)
        # no candidate q*2^14+1 between consecutive entries is prime
        for a, b in zip(run[:5], run[1:6]):
            c = b + step
            while c < a:
                assert not _trial(c)
                c += step
    # the candidates above each run's first entry (up to the run's bound) are composite
    for first, bound in ((full[0], (1 << 32) // 3), (full[n1], (1 << 31) - 1)):
        c = first + step
        while c <= bound:
            assert not _trial(c)
            c += step
    # the last entry of the first run and the candidates below it down to 2^30
    c = full[n1 - 1] - step
    while c > (1 << 30):
        assert not _trial(c)
        c -= step


def test_primitive_root_brute_force_small_primes():
    for p in [3, 5, 7, 17, 97, 257, 769, 7681, 12289]:
        g = nt.primitive_root(p)

        def order(x):
            k, y = 1, x % p
            while y != 1:
                y = y * x % p
                k += 1
            return k

        assert order(g) == p - 1
        for h in range(2, g):
            assert order(h) < p - 1


def test_root_of_unity_and_coset():
    for p in nt.prime_table(3):
        for n in (1, 2, 64, 1024, 1 << 14):
            w = nt.root_of_unity(p, n)
            assert pow(w, n, p) == 1
            if n > 1:
                assert pow(w, n // 2, p) == p - 1
        pts = nt.coset_points(p, 64)
        assert len(set(pts)) == 64
        assert all(pow(x, 64, p) != 1 for x in pts)
        assert 1 not in pts and p - 1 not in pts and 0 not in pts


def test_coset_avoids_small_integers():
    """The evaluation cosets c <w> of the first 300 table primes contain no integer of
    [-16, 16] for the transform sizes 2^8, 2^10 and 2^13 (so curves with vertical
    asymptotes at small integers reject no prime by a coset hit), and c lies outside the
    subgroup of order 2^14.  The smallest primitive root would not do: it is 3 for about
    half of these primes, so x = 3 would be a point of their every evaluation set."""
    primes = nt.prime_table(300)
    for p in primes:
        c = nt.coset_representative(p)
        assert pow(c, 1 << 14, p) != 1
        ci = pow(c, p - 2, p)
        for n in (1 << 8, 1 << 10, 1 << 13):
            for x in range(-16, 17):
                if x:
                    assert pow(x * ci % p, n, p) != 1, (p, n, x)
        pts = nt.coset_points(p, 256)
        assert pts[0] == c and pts[1] == c * nt.root_of_unity(p, 256) % p
    assert sum(nt.primitive_root(p) == 3 for p in primes) > 100
