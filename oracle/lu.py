"""Reference LU decompositions, solves and error measures.

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

Sec. 3.4: right-looking LU with partial pivoting (LAPACK getrf style).  The
oracle runs the unblocked form (the "unblocked naive, b = 1" of Sec. 3.4),
which computes the same factorisation as any blocking up to rounding:
  * lu_exact: exact rational arithmetic (fractions) for small n;
  * lu_bigfloat: p-bit arithmetic with one correct rounding per operation
    (the oracle uses p + 64 bits for a target precision p).
Pivot rule (a reading; the paper does not state it): the entry of largest
absolute value in the current column, compared exactly, the lowest row index
on ties.

Sec. 4.4: the Lotkin matrix (first row all ones, A_ij = 1/(i+j+1) below,
0-based), the right-hand side b = A * ones formed exactly, and the number of
correct bits min_i(-log2|x_i - 1|), taken from exact values, never through a
binary64 conversion (the Remark of Sec. 4.4).
"""
from __future__ import annotations

import itertools
import math
from fractions import Fraction

from .bigfloat import (bf_abs_cmp, bf_div, bf_fms, bf_from_fraction,
                       bf_to_fraction)


# ------------------------------------------------------------ matrices ----
def lotkin(n: int) -> list[list[Fraction]]:
    """Sec. 4.4: row 0 all ones, A_ij = 1/(i+j+1) for i >= 1 (0-based)."""
    return [[Fraction(1) if i == 0 else Fraction(1, i + j + 1) for j in range(n)]
            for i in range(n)]


def matvec(A, x):
    return [sum((a * b for a, b in zip(row, x)), Fraction(0)) for row in A]


# ---------------------------------------------------------- exact LU -----
def lu_exact(A):
    """Exact rational LU with partial pivoting: P A = L U.

    Returns (perm, L, U): perm[i] is the original row that ends up in row i.
    """
    n = len(A)
    a = [list(map(Fraction, row)) for row in A]
    perm = list(range(n))
    for k in range(n):
        piv = k
        for i in range(k + 1, n):
            if abs(a[i][k]) > abs(a[piv][k]):
                piv = i
        if a[piv][k] == 0:
            raise ZeroDivisionError(f"singular at column {k}")
        a[k], a[piv] = a[piv], a[k]
        perm[k], perm[piv] = perm[piv], perm[k]
        for i in range(k + 1, n):
            a[i][k] /= a[k][k]
            lik = a[i][k]
            if lik:
                for j in range(k + 1, n):
                    a[i][j] -= lik * a[k][j]
    L = [[a[i][j] if j < i else (Fraction(1) if i == j else Fraction(0))
          for j in range(n)] for i in range(n)]
    U = [[a[i][j] if j >= i else Fraction(0) for j in range(n)] for i in range(n)]
    return perm, L, U


def perm_sign(perm) -> int:
    sign, seen = 1, [False] * len(perm)
    for i in range(len(perm)):
        if not seen[i]:
            j, length = i, 0
            while not seen[j]:
                seen[j] = True
                j = perm[j]
                length += 1
            if length % 2 == 0:
                sign = -sign
    return sign


def det_leibniz(A) -> Fraction:
    """Brute-force determinant: the sum over all n! permutations."""
    n = len(A)
    total = Fraction(0)
    for p in itertools.permutations(range(n)):
        term = Fraction(perm_sign(list(p)))
        for i in range(n):
            term *= A[i][p[i]]
            if term == 0:
                break
        total += term
    return total


def det_bareiss(A) -> Fraction:
    """Fraction-free Bareiss elimination on the common-denominator integers."""
    n = len(A)
    den = 1
    for row in A:
        for x in row:
            den = den * Fraction(x).denominator // math.gcd(den, Fraction(x).denominator)
    M = [[int(Fraction(x) * den) for x in row] for row in A]
    sign, prev = 1, 1
    for k in range(n - 1):
        if M[k][k] == 0:
            sw = next((i for i in range(k + 1, n) if M[i][k] != 0), None)
            if sw is None:
                return Fraction(0)
            M[k], M[sw] = M[sw], M[k]
            sign = -sign
        for i in range(k + 1, n):
            for j in range(k + 1, n):
                M[i][j] = (M[i][j] * M[k][k] - M[i][k] * M[k][j]) // prev
        prev = M[k][k]
    return Fraction(sign * M[n - 1][n - 1], den ** n)


# -------------------------------------------------------- p-bit LU -------
def to_bigfloat_matrix(A, prec):
    return [[bf_from_fraction(Fraction(x), prec) for x in row] for row in A]


def lu_bigfloat(A, prec):
    """Unblocked right-looking LU with partial pivoting at prec bits.

    A: list of rows of (N, E) p-bit numbers (modified copy returned).
    Returns (a, ipiv, info): a holds L (unit, below) and U; ipiv[k] = row
    exchanged with row k at step k (0-based, LAPACK order); info = first
    column (1-based) with an exactly zero pivot, 0 if none.
    """
    n = len(A)
    a = [list(row) for row in A]
    ipiv = list(range(n))
    info = 0
    for k in range(n):
        piv = k
        for i in range(k + 1, n):
            if bf_abs_cmp(a[i][k], a[piv][k]) > 0:
                piv = i
        ipiv[k] = piv
        if piv != k:
            a[k], a[piv] = a[piv], a[k]
        if a[k][k][0] == 0:
            if info == 0:
                info = k + 1
            continue
        for i in range(k + 1, n):
            a[i][k] = bf_div(a[i][k], a[k][k], prec)
        for i in range(k + 1, n):
            lik = a[i][k]
            if lik[0] == 0:
                continue
            row_i, row_k = a[i], a[k]
            for j in range(k + 1, n):
                if row_k[j][0]:
                    row_i[j] = bf_fms(row_i[j], lik, row_k[j], prec)
    return a, ipiv, info


def getrs_bigfloat(a, ipiv, b, prec):
    """Solve A x = b from lu_bigfloat's factors: P b, forward L, backward U."""
    n = len(a)
    x = list(b)
    for k in range(n):
        if ipiv[k] != k:
            x[k], x[ipiv[k]] = x[ipiv[k]], x[k]
    for i in range(n):
        for j in range(i):
            if a[i][j][0] and x[j][0]:
                x[i] = bf_fms(x[i], a[i][j], x[j], prec)
    for i in range(n - 1, -1, -1):
        for j in range(i + 1, n):
            if a[i][j][0] and x[j][0]:
                x[i] = bf_fms(x[i], a[i][j], x[j], prec)
        x[i] = bf_div(x[i], a[i][i], prec)
    return x


# ------------------------------------------------------------ measures ----
def apply_ipiv_rows(A, ipiv):
    """P A for LAPACK-order interchanges."""
    rows = [list(r) for r in A]
    for k, p in enumerate(ipiv):
        if p != k:
            rows[k], rows[p] = rows[p], rows[k]
    return rows


def backward_error(A, LU, ipiv) -> Fraction:
    """max|P A - L U| / max|A| from exact values (A, LU as Fractions)."""
    n = len(A)
    PA = apply_ipiv_rows(A, ipiv)
    num = Fraction(0)
    for i in range(n):
        for j in range(n):
            s = Fraction(0)
            for k in range(min(i, j) + 1):
                lik = Fraction(1) if k == i else LU[i][k]
                s += lik * LU[k][j]
            num = max(num, abs(PA[i][j] - s))
    den = max(abs(x) for row in A for x in row)
    return num / den


def log2_abs(v: Fraction) -> float:
    """log2|v| from the exact numerator and denominator (no binary64 underflow)."""
    v = abs(v)
    return math.log2(v.numerator) - math.log2(v.denominator)


def correct_bits(x) -> float:
    """min_i(-log2|x_i - 1|) for exact solution ones (Sec. 4.4)."""
    worst = math.inf
    for xi in x:
        d = Fraction(xi) - 1
        if d != 0:
            worst = min(worst, -log2_abs(d))
    return worst


def to_fractions(a):
    return [[bf_to_fraction(x) for x in row] for row in a]
