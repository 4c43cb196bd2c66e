"""Pins of the Ozaki-II replay (oracle/oz2.py) against the mathematics.

Each check is independent of the code path it checks:
  * brute-force residue products with Python integers (S4 congruence);
  * S_g equals the exact digit-group sum (the identity Eq. (11) must meet);
  * the CPU CRT procedure equals Eq. (11)'s round-to-nearest form;
  * digits rebuild the fixed-point value and respect |v_t| <= 2^(w-1);
  * exact GEMM in rationals: every output within one unit 2^-p (the single
    rounding of (S6)), and the printed error levels of Table cpu_gemm;
  * S = 1 with inputs that fit in Q bits gives the correctly rounded product;
  * extra digit groups recover about w bits under cancellation (Sec. 3.2);
  * Eq. (15) digits are exact in E4M3 and the 3-plane Karatsuba product is
    exact for every pair of residues;
  * a planted mistake in the CRT is caught by the identity check.
"""
import math
import os
from fractions import Fraction

import numpy as np
import pytest

import oracle.oz2 as oz2
from oracle.expansion import expansion_value, fl_expansion, ulp_p
from oracle.plan import make_plan
from synth import random_expansions

GOLD = os.path.join(os.path.dirname(__file__), "golden", "paper_errors.txt")


def _rand(m, k, n, nc, seed, emin=-3, emax=3):
    A = random_expansions(m, k, nc, seed, emin, emax)
    B = random_expansions(k, n, nc, seed + 1000, emin, emax)
    return A, B


def _exact(A, B):
    ex = oz2.exact_gemm(A, B)
    return [[Fraction(N) * Fraction(2) ** E for (N, E) in row] for row in ex]


@pytest.mark.parametrize("nc,p,S", [(2, 106, None), (3, 159, None), (4, 212, None),
                                    (4, 212, 3), (2, 106, 2)])
def test_residue_congruence_and_crt_identity(nc, p, S):
    A, B = _rand(3, 5, 4, nc, 10 + nc)
    out, d = oz2.oz2_gemm(A, B, p, S=S, debug=True)
    plan = d.plan
    m, K, n = 3, 5, 4
    for l, ml in enumerate(plan.moduli):
        for g in plan.groups:
            for i in range(m):
                for j in range(n):
                    # brute force: sum over pairs and h with Python ints
                    s = 0
                    for ta in range(plan.S):
                        tb = g - ta
                        if 0 <= tb < plan.S:
                            for h in range(K):
                                s += int(d.digits_A[ta][i, h]) * int(d.digits_B[tb][h, j])
                    assert (int(d.C[(l, g)][i, j]) - s) % ml == 0
                    assert (int(d.t[(l, g)][i, j]) * plan.M[l] - s) % ml == 0
    for g in plan.groups:
        exact = oz2.digit_group_exact(d.digits_A, d.digits_B, g, plan.S)
        for i in range(m):
            for j in range(n):
                assert d.Sbar[g][i, j] == exact[i, j]
                tv = [d.t[(l, g)][i, j] for l in range(plan.N)]
                assert oz2.crt_round(tv, plan) == d.Sbar[g][i, j]


def test_digits_rebuild_fixed_point():
    A, _ = _rand(4, 6, 1, 4, 3, -40, 40)
    plan = make_plan(212, 6)
    mu = oz2.shared_shifts(A, 0, plan.Q)
    for i in range(4):
        for h in range(6):
            X = oz2.fixed_point(A[i, h], mu[i])
            assert abs(X) < 2 ** (plan.Q - 1)
            v = oz2.balanced_digits(X, plan.w, plan.S)
            assert sum(vt << (plan.w * t) for t, vt in enumerate(v)) == X
            assert all(abs(vt) <= 2 ** (plan.w - 1) for vt in v)
            # Eq. (12) is within nc-1 of trunc(2^mu x)
            exact = expansion_value(A[i, h]) * Fraction(2) ** mu[i]
            assert abs(X - int(exact)) <= 3


def test_centered_residue_ranges():
    for m in (251, 128, 127, 3):
        rs = {oz2.centered_residue(v, m) for v in range(-3 * m, 3 * m)}
        assert rs == set(range(-(m // 2), (m + 1) // 2))


@pytest.mark.parametrize("nc,p", [(2, 106), (3, 159), (4, 212)])
def test_error_one_unit_and_printed_levels(nc, p):
    printed = {int(a): float(c) for a, _, c in
               (l.split() for l in open(GOLD) if l.strip() and not l.startswith("#"))}
    A, B = _rand(4, 16, 4, nc, 20 + nc, -1, 0)
    out = oz2.oz2_gemm(A, B, p)
    ex = _exact(A, B)
    worst = 0.0
    for i in range(4):
        for j in range(4):
            c = ex[i][j]
            err = abs(expansion_value(out[i, j]) - c)
            assert err <= ulp_p(c, p)
            worst = max(worst, float(err / abs(c)))
    # Table cpu_gemm prints 1.2e-32 / 1.4e-48 / 1.5e-64: the unit 2^-p
    assert worst <= 2.0 * printed[nc]
    assert abs(printed[nc] / 2.0 ** -p - 1) < 0.1


def test_s1_exact_when_inputs_fit():
    # integers stored as DD: nothing is truncated at S = 1, so the result is
    # the correctly rounded exact product (cf. "0 ulp" against MPFR, Sec. 4.2.1)
    rng = np.random.default_rng(5)
    A = np.zeros((3, 7, 2))
    B = np.zeros((7, 3, 2))
    A[..., 0] = rng.integers(-2 ** 40, 2 ** 40, size=(3, 7))
    B[..., 0] = rng.integers(-2 ** 40, 2 ** 40, size=(7, 3))
    out = oz2.oz2_gemm(A, B, 106)
    ex = oz2.exact_gemm(A, B)
    for i in range(3):
        for j in range(3):
            N, E = ex[i, j]
            assert list(out[i, j]) == fl_expansion(N, E, 2)


def test_beta_one_fused_update():
    A, B = _rand(3, 8, 3, 4, 31, -1, 0)
    C = random_expansions(3, 3, 4, 77, -1, 0)
    out = oz2.oz2_gemm(A, B, 212, alpha=-1, beta=1, C=C)
    ex = _exact(A, B)
    for i in range(3):
        for j in range(3):
            ref = expansion_value(C[i, j]) - ex[i][j]
            err = abs(expansion_value(out[i, j]) - ref)
            assert err <= ulp_p(ref, 212)


def test_extra_groups_recover_w_bits():
    # cancellation (Sec. 3.2): c = a b - a (b - eps) = a eps, Gamma = 2^150;
    # eps sits below the top digit of b so the dropped group 0 carries it
    A, _ = _rand(1, 1, 1, 4, 41, 0, 0)
    A = np.concatenate([A, A], axis=1)            # row [a, a]
    b0 = 0.8125
    B = np.zeros((2, 1, 4))
    B[0, 0, 0] = b0
    B[1, 0, 0], B[1, 0, 1] = -b0, 2.0 ** -150     # -b + 2^-150, non-overlapping
    ex = _exact(A, B)[0][0]
    assert ex == expansion_value(A[0, 0]) * Fraction(2) ** -150
    errs = []
    for extra in (0, 1):
        out = oz2.oz2_gemm(A, B, 212, extra_groups=extra)
        errs.append(abs(expansion_value(out[0, 0]) - ex) / abs(ex))
    plan = make_plan(212, 2)
    assert plan.S == 2
    # without the low group the truncation (Prop. 2) shows at about
    # 2^-(2w) Gamma relative; with it (S = 2: groups 0..2) nothing is dropped
    assert errs[0] > Fraction(2) ** -212
    assert errs[0] < Fraction(2) ** (-2 * plan.w + 150 + 8)
    assert errs[1] <= Fraction(2) ** -211
    # one extra group recovers at least w - 8 bits here
    assert errs[1] == 0 or math.log2(errs[0] / errs[1]) > min(plan.w - 8, 30)


def test_fp8_base17_digits_exact_in_e4m3():
    def e4m3_values():
        vals = set()
        for e in range(0, 16):
            for f in range(8):
                if e == 15 and f == 7:
                    continue  # NaN
                v = (f / 8) * 2.0 ** -6 if e == 0 else (1 + f / 8) * 2.0 ** (e - 7)
                vals.add(v)
                vals.add(-v)
        return vals
    E4M3 = e4m3_values()
    worst = 0
    for r in range(-127, 128):
        d0, d1 = oz2.fp8_base17_digits(r)
        assert 17 * d1 + d0 == r and abs(d0) <= 8 and abs(d1) <= 7  # Eq. (15)
        for v in (d0, d1, d0 + d1):
            assert float(v) in E4M3
        worst = max(worst, abs(d0), abs(d1), abs(d0 + d1))
    assert worst == 15
    for r in range(-127, 128, 3):
        a0, a1 = oz2.fp8_base17_digits(r)
        for s in range(-127, 128, 5):
            b0, b1 = oz2.fp8_base17_digits(s)
            p00, p11, pss = a0 * b0, a1 * b1, (a0 + a1) * (b0 + b1)
            assert p00 + 17 * (pss - p00 - p11) + 289 * p11 == r * s


def test_planted_crt_mistake_is_caught(monkeypatch):
    A, B = _rand(2, 4, 2, 2, 61)
    real = oz2.crt_cpu

    def wrong(tvals, plan):
        X = real(tvals, plan)
        return X + plan.P if X < 0 else X  # drops the sign step of Sec. 3.5.1

    monkeypatch.setattr(oz2, "crt_cpu", wrong)
    _, d = oz2.oz2_gemm(A, B, 106, debug=True)
    ok = all(d.Sbar[g][i, j] == oz2.digit_group_exact(d.digits_A, d.digits_B, g, d.plan.S)[i, j]
             for g in d.plan.groups for i in range(2) for j in range(2))
    assert not ok


def test_zero_rows_and_columns():
    A, B = _rand(3, 5, 3, 2, 71)
    A[1] = 0.0
    B[:, 2] = 0.0
    out = oz2.oz2_gemm(A, B, 106)
    assert np.all(out[1] == 0.0) and np.all(out[:, 2] == 0.0)


def test_window_raise_keeps_far_c_unchanged():
    # (S6) with beta = 1 and an old C far above the product: the grid is
    # raised (e_top - E0 > WINDOW_BITS) and the result must be C itself, since
    # the product lies below half a unit of C's last component
    A, B = _rand(3, 6, 2, 4, 501, -2, 2)
    C = random_expansions(3, 2, 4, 502, 600, 620)
    out, d = oz2.oz2_gemm(A, B, 212, alpha=-1, beta=1, C=C, debug=True)
    for i in range(3):
        for j in range(2):
            E0 = d.plan.w * d.plan.g0 - d.mu[i] - d.nu[j]
            e_top = max(E0 + abs(int(d.Pint[i, j])).bit_length(), math.frexp(C[i, j, 0])[1]) + 1
            assert e_top - E0 > oz2.WINDOW_BITS       # the raise is exercised
            assert list(out[i, j]) == list(C[i, j])


def test_window_raise_within_bound_on_sparse_c():
    # a sparse old C whose low component falls below the raised grid: the
    # single rounding stays within one unit 2^-p of the exact beta C + alpha A B
    A, B = _rand(2, 4, 2, 4, 511, -1, 1)
    C = np.zeros((2, 2, 4))
    C[..., 0] = 2.0 ** 600
    C[..., 1] = 2.0 ** 60
    out = oz2.oz2_gemm(A, B, 212, alpha=1, beta=1, C=C)
    ex = _exact(A, B)
    for i in range(2):
        for j in range(2):
            ref = expansion_value(C[i, j]) + ex[i][j]
            assert abs(expansion_value(out[i, j]) - ref) <= ulp_p(ref, 212)


def test_gamma_factor_closed_form():
    # Eq. (7): a = [1, 1], b = [1, -1 + 2^-k]: c = 2^-k, max|a| max|b| = 1,
    # so Gamma = 2^k exactly
    for k in (1, 40, 150):
        A = np.zeros((1, 2, 4))
        A[0, :, 0] = 1.0
        B = np.zeros((2, 1, 4))
        B[0, 0, 0] = 1.0
        B[1, 0, 0], B[1, 0, 1] = -1.0, 2.0 ** -k
        if k < 53:
            B[1, 0, :] = 0.0
            B[1, 0, 0] = -1.0 + 2.0 ** -k
        g = oz2.gamma_factor(A, B)
        assert g[0, 0] == 2.0 ** k


def test_gamma_guard_of_proposition2():
    # Prop. 2 / Eq. (6): the result is within the unit 2^-p of c once Q covers
    # p + log2 Gamma + log2 2K + log2 S + g0, i.e. with g_ex >= log2 Gamma; with
    # no guard the dropped digit group shows at about Gamma 2^-Q relative
    rng = np.random.default_rng(77)
    A, Bh = _rand(1, 1, 1, 4, 91, 0, 0)
    A = np.concatenate([A, A], axis=1)                    # row [a, a]
    B = np.zeros((2, 1, 4))
    B[0, 0] = Bh[0, 0]                                    # b, all four components
    neg = -Bh[0, 0]
    B[1, 0, 0], B[1, 0, 1] = neg[0], neg[1]               # -b + delta: keep the top two
    B[1, 0, 2] = 2.0 ** -120 * (1 + rng.random())         # delta far below b
    gam = float(oz2.gamma_factor(A, B)[0, 0])
    k = math.ceil(math.log2(gam))
    assert 100 <= k <= 130
    ex = _exact(A, B)[0][0]
    err = {}
    for gex in (0, k):
        plan = make_plan(212, 2, g_ex=gex)
        assert plan.S >= 2
        out = oz2.oz2_gemm(A, B, 212, g_ex=gex)
        err[gex] = abs(expansion_value(out[0, 0]) - ex)
    assert err[k] <= ulp_p(ex, 212)                     # the guarded plan meets Prop. 2
    assert err[0] > ulp_p(ex, 212)                      # without it the truncation shows
