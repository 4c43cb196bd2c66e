"""Pins of the p-bit Ozaki-II replay (oracle/mp.py) against independent facts."""
import random
from fractions import Fraction

import numpy as np
import pytest

from oracle.bigfloat import bf_round
from oracle.mp import frexp_exp, oz2_gemm_mp, window_bits
from oracle.oz2 import digit_group_exact, oz2_gemm
from oracle.plan import make_plan


def rand_mp(rng, rows, cols, p, emin=-2, emax=2, positive=False):
    out = []
    for _ in range(rows):
        row = []
        for _ in range(cols):
            N = rng.getrandbits(p) | (1 << (p - 1))
            if not positive and rng.random() < 0.5:
                N = -N
            row.append((N, rng.randint(emin, emax) - p))
        out.append(row)
    return out


def value(x):
    return Fraction(x[0]) * Fraction(2) ** x[1]


def exact_product(A, B):
    m, K, n = len(A), len(A[0]), len(B[0])
    return [[sum((value(A[i][h]) * value(B[h][j]) for h in range(K)), Fraction(0))
             for j in range(n)] for i in range(m)]


def ulp_p(v: Fraction, p: int) -> Fraction:
    a = abs(v)
    e = a.numerator.bit_length() - a.denominator.bit_length()
    if Fraction(2) ** e > a:
        e -= 1
    return Fraction(2) ** (e - p + 1)


@pytest.mark.parametrize("p,K", [(80, 3), (300, 4), (1100, 2)])
def test_close_to_exact_product(p, K):
    """Positive entries (no cancellation): within 2 units of 2^-p (Prop. 2 bound)."""
    rng = random.Random(p + K)
    A = rand_mp(rng, 3, K, p, positive=True)
    B = rand_mp(rng, K, 2, p, positive=True)
    got = oz2_gemm_mp(A, B, p)
    ex = exact_product(A, B)
    for i in range(3):
        for j in range(2):
            err = abs(value(got[i][j]) - ex[i][j])
            assert err <= 2 * ulp_p(ex[i][j], p), (i, j, float(err / ulp_p(ex[i][j], p)))
            assert abs(got[i][j][0]) < (1 << p)


def test_group_sums_are_exact_digit_products():
    """S_g equals the exact digit-group sum (CRT reconstructs the integer)."""
    rng = random.Random(5)
    p = 400
    A = rand_mp(rng, 2, 3, p)
    B = rand_mp(rng, 3, 2, p)
    _, (plan, mu, nu, tg, Sbar, Pint) = oz2_gemm_mp(A, B, p, debug=True)
    from oracle.mp import digits_mp
    DA = digits_mp(A, mu, 0, plan.w, plan.S)
    DB = digits_mp(B, nu, 1, plan.w, plan.S)
    for g in plan.groups:
        ex = digit_group_exact(DA, DB, g, plan.S)
        for i in range(2):
            for j in range(2):
                assert int(Sbar[g][i, j]) == int(ex[i, j])


def test_matches_expansion_replay_on_dyadic_inputs():
    """DD-valued inputs whose fixed points are exact: P_int equals oracle.oz2's."""
    rng = np.random.default_rng(3)
    K = 4
    A = np.zeros((3, K, 2))
    B = np.zeros((K, 2, 2))
    for arr in (A, B):
        hi = rng.integers(-2**20, 2**20, size=arr.shape[:2]) / 2.0**10
        lo = rng.integers(-2**20, 2**20, size=arr.shape[:2]) / 2.0**70
        arr[..., 0], arr[..., 1] = hi, lo
    p = 106
    _, dbg = oz2_gemm(A, B, p, debug=True)

    def as_mp(X):
        out = []
        for r in range(X.shape[0]):
            row = []
            for c in range(X.shape[1]):
                v = Fraction(float(X[r, c, 0])) + Fraction(float(X[r, c, 1]))
                k = v.denominator.bit_length() - 1
                row.append((v.numerator, -k))
            out.append(row)
        return out
    _, (plan, mu, nu, tg, Sbar, Pint) = oz2_gemm_mp(as_mp(A), as_mp(B), p, debug=True)
    assert mu == dbg.mu and nu == dbg.nu
    assert all(int(Pint[i, j]) == int(dbg.Pint[i, j]) for i in range(3) for j in range(2))


def test_fused_update_and_window():
    rng = random.Random(9)
    p = 200
    A = rand_mp(rng, 2, 3, p, positive=True)
    B = rand_mp(rng, 3, 2, p, positive=True)
    C = rand_mp(rng, 2, 2, p)
    got = oz2_gemm_mp(A, B, p, alpha=-1, beta=1, C=C)
    ex = exact_product(A, B)
    for i in range(2):
        for j in range(2):
            t = value(C[i][j]) - ex[i][j]
            assert abs(value(got[i][j]) - t) <= 4 * ulp_p(max(abs(t), abs(ex[i][j])), p)
    # old C far above the product window: the result is C rounded (unchanged)
    plan = make_plan(p, 3)
    big = [[(1 | (1 << (p - 1)), window_bits(plan, 3) + 50) for _ in range(2)] for _ in range(2)]
    got = oz2_gemm_mp(A, B, p, alpha=1, beta=1, C=big)
    assert got == [[bf_round(*big[i][j], p) for j in range(2)] for i in range(2)]


def test_zero_rows_and_frexp():
    assert frexp_exp((0, 5)) is None and frexp_exp((3, -2)) == 0
    A = [[(0, 0), (0, 0)], [(1, 0), (-3, -1)]]
    B = [[(1, 0)], [(1, 1)]]
    got = oz2_gemm_mp(A, B, 64)
    assert got[0][0] == (0, 0)
    assert value(got[1][0]) == Fraction(1) - Fraction(3)
