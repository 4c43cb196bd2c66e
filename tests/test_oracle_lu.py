"""Pins of oracle/lu.py and oracle/bigfloat.py.

  * exact LU: P A = L U holds exactly; det(A) = sign(P) prod u_ii equals the
    brute-force Leibniz sum and the fraction-free Bareiss determinant;
  * p-bit arithmetic: each operation equals the correctly rounded exact
    result (rationals), ties to even;
  * p-bit LU agrees with the exact LU to its precision, and on the Lotkin
    matrix the solution has at least p - log2 cond - small correct bits,
    the behaviour Table lotkin prints.
"""
import math
import os
import random
from fractions import Fraction

import pytest

from oracle import bigfloat as bf
from oracle import lu

GOLD = os.path.join(os.path.dirname(__file__), "golden", "lotkin.txt")


def _rand_rational(n, seed):
    rng = random.Random(seed)
    return [[Fraction(rng.randint(-50, 50), rng.randint(1, 9)) for _ in range(n)]
            for _ in range(n)]


@pytest.mark.parametrize("n,seed", [(1, 1), (2, 2), (4, 3), (6, 4), (7, 5)])
def test_exact_lu_and_determinants(n, seed):
    A = _rand_rational(n, seed)
    perm, L, U = lu.lu_exact(A)
    PA = [A[perm[i]] for i in range(n)]
    LU = [[sum(L[i][k] * U[k][j] for k in range(n)) for j in range(n)] for i in range(n)]
    assert PA == LU
    for i in range(n):
        for j in range(i):
            assert abs(L[i][j]) <= 1  # partial pivoting
    d = Fraction(lu.perm_sign(perm))
    for i in range(n):
        d *= U[i][i]
    assert d == lu.det_leibniz(A) == lu.det_bareiss(A)


@pytest.mark.parametrize("n", [2, 3, 5, 7])
def test_lotkin_structure_and_det(n):
    A = lu.lotkin(n)
    assert all(x == 1 for x in A[0])
    assert A[1][0] == Fraction(1, 2) and A[n - 1][n - 1] == Fraction(1, 2 * n - 1)
    perm, L, U = lu.lu_exact(A)
    d = Fraction(lu.perm_sign(perm))
    for i in range(n):
        d *= U[i][i]
    assert d == lu.det_leibniz(A) == lu.det_bareiss(A) != 0


def test_lotkin_conditioning_grows_like_5n():
    ratios = []
    for n in (8, 12, 16):
        A = lu.lotkin(n)
        perm, L, U = lu.lu_exact(A)
        inv_cols = []
        for k in range(n):
            b = [Fraction(int(perm[i] == k)) for i in range(n)]
            y = [Fraction(0)] * n
            for i in range(n):
                y[i] = b[i] - sum(L[i][j] * y[j] for j in range(i))
            x = [Fraction(0)] * n
            for i in range(n - 1, -1, -1):
                x[i] = (y[i] - sum(U[i][j] * x[j] for j in range(i + 1, n))) / U[i][i]
            inv_cols.append(x)
        na = max(sum(abs(v) for v in row) for row in A)
        ni = max(sum(abs(inv_cols[k][i]) for k in range(n)) for i in range(n))
        ratios.append(lu.log2_abs(na * ni) / n)
    assert ratios == sorted(ratios) and 4.4 < ratios[0] and ratios[-1] < 5.2


def test_bigfloat_ops_correctly_rounded():
    rng = random.Random(9)
    prec = 80
    for _ in range(800):
        x = bf.bf_from_fraction(Fraction(rng.randint(-10 ** 30, 10 ** 30), rng.randint(1, 10 ** 20)), prec)
        y = bf.bf_from_fraction(Fraction(rng.randint(-10 ** 30, 10 ** 30), rng.randint(1, 10 ** 20)), prec)
        fx, fy = bf.bf_to_fraction(x), bf.bf_to_fraction(y)
        for got, exact in ((bf.bf_add(x, y, prec), fx + fy), (bf.bf_mul(x, y, prec), fx * fy),
                           (bf.bf_fms(x, x, y, prec), fx - fx * fy)):
            assert bf.bf_to_fraction(got) == bf.bf_to_fraction(bf.bf_from_fraction(exact, prec))
            err = abs(bf.bf_to_fraction(got) - exact)
            assert exact == 0 or err <= abs(exact) * Fraction(2) ** -prec
        if fy != 0:
            q = bf.bf_div(x, y, prec)
            assert abs(bf.bf_to_fraction(q) - fx / fy) <= abs(fx / fy) * Fraction(2) ** -prec
    # ties to even at 3 bits: 9 = 1001b -> 8, 11 = 1011b -> 12
    assert bf.bf_round(9, 0, 3) == (4, 1) and bf.bf_round(11, 0, 3) == (6, 1)


def test_bigfloat_lu_matches_exact():
    A = _rand_rational(6, 21)
    prec = 200
    a, ipiv, info = lu.lu_bigfloat(lu.to_bigfloat_matrix(A, prec), prec)
    perm, L, U = lu.lu_exact(A)
    assert info == 0
    F = lu.to_fractions(a)
    for i in range(6):
        for j in range(6):
            ref = L[i][j] if j < i else U[i][j]
            assert abs(F[i][j] - ref) <= (abs(ref) + 1) * Fraction(2) ** -190
    assert lu.backward_error(A, F, ipiv) < Fraction(2) ** -190


@pytest.mark.parametrize("n,prec", [(10, 128), (14, 160)])
def test_lotkin_solve_correct_bits(n, prec):
    A = lu.lotkin(n)
    b = lu.matvec(A, [Fraction(1)] * n)
    a, ipiv, info = lu.lu_bigfloat(lu.to_bigfloat_matrix(A, prec), prec)
    x = lu.getrs_bigfloat(a, ipiv, [bf.bf_from_fraction(v, prec) for v in b], prec)
    bits = lu.correct_bits([bf.bf_to_fraction(v) for v in x])
    log2cond = 5.1 * n
    # Table lotkin: correct bits slightly exceed p - log2 cond
    assert prec - log2cond - 8 < bits < prec
    rows = [list(map(int, l.split())) for l in open(GOLD) if l.strip() and not l.startswith("#")]
    for n_, p_, lower, printed in rows:
        assert printed >= lower and lower == round(p_ - 5.1 * n_)


def test_zero_pivot_info():
    A = [[Fraction(0), Fraction(1)], [Fraction(0), Fraction(2)]]
    a, ipiv, info = lu.lu_bigfloat(lu.to_bigfloat_matrix(A, 64), 64)
    assert info == 1
