"""The Sylvester matrix (Sec. 2, "Resultants") and three independent determinant routines.

Row convention, as printed in the paper: for f of formal degree m and g of formal degree
n (in the eliminated variable) the (m + n) x (m + n) matrix has n rows holding
f_m, f_{m-1}, ..., f_0 shifted one column to the right per row, followed by m rows
holding g_n, ..., g_0 shifted the same way.  Entries may be integers, residues or
polynomials in the other variable; the routines below take a small ring object.
"""

from __future__ import annotations

from itertools import permutations

from . import poly as P


class IntRing:
    zero = 0
    one = 1

    @staticmethod
    def add(a, b):
        return a + b

    @staticmethod
    def sub(a, b):
        return a - b

    @staticmethod
    def mul(a, b):
        return a * b

    @staticmethod
    def neg(a):
        return -a

    @staticmethod
    def exact_div(a, b):
        q, r = divmod(a, b)
        if r:
            raise ArithmeticError("inexact integer division in Bareiss elimination")
        return q

    @staticmethod
    def is_zero(a):
        return a == 0


class PolyRing:
    """Z[x] with ascending coefficient lists."""
    zero = []
    one = [1]

    @staticmethod
    def add(a, b):
        return P.add(a, b)

    @staticmethod
    def sub(a, b):
        return P.sub(a, b)

    @staticmethod
    def mul(a, b):
        return P.mul(a, b)

    @staticmethod
    def neg(a):
        return P.scale(a, -1)

    @staticmethod
    def exact_div(a, b):
        return P.exact_div_z(a, b)

    @staticmethod
    def is_zero(a):
        return not P.trim(a)


def sylvester(a, b, zero=0):
    """Sylvester matrix of two coefficient lists (ascending order, formal degrees
    len(a) - 1 and len(b) - 1); leading coefficients may be zero (formal shape)."""
    m = len(a) - 1
    n = len(b) - 1
    r = m + n
    rows = []
    for i in range(n):
        row = [zero] * r
        for s in range(m + 1):
            row[i + s] = a[m - s]
        rows.append(row)
    for i in range(m):
        row = [zero] * r
        for s in range(n + 1):
            row[i + s] = b[n - s]
        rows.append(row)
    return rows


def det_leibniz(M, ring=IntRing):
    """Determinant by the permutation expansion (brute force, r <= 7)."""
    n = len(M)
    total = ring.zero
    for perm in permutations(range(n)):
        # sign by counting inversions
        inv = 0
        for i in range(n):
            for j in range(i + 1, n):
                if perm[i] > perm[j]:
                    inv += 1
        term = ring.one
        for i in range(n):
            term = ring.mul(term, M[i][perm[i]])
            if ring.is_zero(term):
                break
        if inv % 2:
            total = ring.sub(total, term)
        else:
            total = ring.add(total, term)
    return total


def det_bareiss(M, ring=IntRing):
    """Fraction-free (Bareiss) elimination over an integral domain; every division is exact."""
    n = len(M)
    if n == 0:
        return ring.one
    A = [list(row) for row in M]
    sign = 1
    prev = ring.one
    for k in range(n - 1):
        if ring.is_zero(A[k][k]):
            piv = None
            for i in range(k + 1, n):
                if not ring.is_zero(A[i][k]):
                    piv = i
                    break
            if piv is None:
                return ring.zero
            A[k], A[piv] = A[piv], A[k]
            sign = -sign
        akk = A[k][k]
        for i in range(k + 1, n):
            aik = A[i][k]
            rowi = A[i]
            rowk = A[k]
            for j in range(k + 1, n):
                num = ring.sub(ring.mul(rowi[j], akk), ring.mul(aik, rowk[j]))
                rowi[j] = ring.exact_div(num, prev)
            rowi[k] = ring.zero
        prev = akk
    d = A[n - 1][n - 1]
    return d if sign > 0 else ring.neg(d)


def det_modp(M, p):
    """Determinant over the field Z_p by Gaussian elimination with row pivoting."""
    n = len(M)
    A = [[x % p for x in row] for row in M]
    det = 1
    for k in range(n):
        piv = None
        for i in range(k, n):
            if A[i][k]:
                piv = i
                break
        if piv is None:
            return 0
        if piv != k:
            A[k], A[piv] = A[piv], A[k]
            det = -det
        akk = A[k][k]
        det = det * akk % p
        inv = pow(akk, p - 2, p)
        for i in range(k + 1, n):
            f = A[i][k] * inv % p
            if f:
                rowi, rowk = A[i], A[k]
                for j in range(k, n):
                    rowi[j] = (rowi[j] - f * rowk[j]) % p
    return det % p
