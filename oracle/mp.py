"""Ozaki-scheme-II GEMM for p-bit multi-limb numbers, replayed exactly.

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

The arbitrary-precision LU of Sec. 3.4 / Sec. 4.4 (p = 12544 for the Lotkin
matrix of order 2048) runs the same Ozaki-II GEMM on p-bit numbers instead
of binary64 expansions.  A p-bit number here is an exact pair (N, E), value
N * 2^E with |N| < 2^p.  The steps are those of Sec. 3.1 in the paper's
order, with the p-bit number in place of the expansion:

  (S1) E_i = max_h of the frexp exponent of a_ih (|a_ih| < 2^E_i),
       mu_i = (Q - 1) - E_i (0 for an all-zero row); nu_j likewise
  (S2) a_bar = trunc(a * 2^mu_i) (toward zero: the exact counterpart of
       Eq. (12) for a single p-bit significand), S balanced w-bit digits (Eq. (2))
  (S3)-(S5) centered residues, digit-group products, t_l and the CRT of
       Eq. (11): identical to oracle.oz2 (the same functions are reused)
  (S6) P_int = sum_g S_g 2^(w (g - g0)) on the grid 2^E0, E0 = w g0 - mu_i - nu_j;
       the old C is truncated toward zero onto the grid, the exact sum
       beta C + alpha P_int is rounded once to p bits (round to nearest even).
       If the old C reaches more than window_bits(plan) above the grid, the
       grid is raised to e_top - window_bits and the product integer is
       truncated toward zero onto it (the fixed-size accumulator reading of
       the expansion case, with a window that holds the largest P_int).
"""
from __future__ import annotations

import math

import numpy as np

from .bigfloat import bf_round
from .oz2 import balanced_digits, centered_residue, crt_cpu
from .plan import Plan, make_plan


def frexp_exp(x) -> int | None:
    """e with 2^(e-1) <= |x| < 2^e for x = (N, E); None for zero."""
    N, E = x
    if N == 0:
        return None
    return abs(N).bit_length() + E


def window_bits(plan: Plan, K: int) -> int:
    """Accumulator window above the grid (bits): the largest |P_int| plus 64
    bits of headroom, in whole 32-bit words, one bit spare for the sign."""
    sbar_bits = 2 * plan.w - 1 + math.ceil(math.log2(plan.S * K) - 1e-12) + 1
    pint_bits = plan.w * (2 * plan.S - 2 - plan.g0) + sbar_bits
    words = (pint_bits + 64 + 31) // 32 + 1
    return 32 * words - 2


def shifts_mp(X, axis: int, Q: int) -> list[int]:
    """(S1) mu_i over rows (axis 0) or nu_j over columns (axis 1)."""
    rows, cols = len(X), len(X[0])
    out = []
    for a in range(rows if axis == 0 else cols):
        es = [frexp_exp(X[a][h] if axis == 0 else X[h][a])
              for h in range(cols if axis == 0 else rows)]
        es = [e for e in es if e is not None]
        out.append(0 if not es else (Q - 1) - max(es))
    return out


def trunc_scaled(x, s: int) -> int:
    """(S2) trunc(x * 2^s) toward zero for x = (N, E)."""
    N, E = x
    k = E + s
    if k >= 0:
        return N << k
    return -((-N) >> (-k)) if N < 0 else N >> (-k)


def digits_mp(X, shifts, axis: int, w: int, S: int):
    rows, cols = len(X), len(X[0])
    D = [np.empty((rows, cols), dtype=object) for _ in range(S)]
    for i in range(rows):
        for j in range(cols):
            sh = shifts[i] if axis == 0 else shifts[j]
            v = balanced_digits(trunc_scaled(X[i][j], sh), w, S)
            for t in range(S):
                D[t][i, j] = v[t]
    return D


def oz2_gemm_mp(A, B, p: int, alpha: int = 1, beta: int = 0, C=None,
                plan: Plan | None = None, debug: bool = False):
    """C = beta C + alpha A B for p-bit matrices (lists of rows of (N, E)).

    Returns the rounded p-bit results (lists of rows of (N, E)); with debug,
    also (plan, mu, nu, t values {(l, g): int64 array}, S_g {g: object array},
    P_int object array).
    """
    m, K = len(A), len(A[0])
    n = len(B[0])
    assert len(B) == K
    if plan is None:
        plan = make_plan(p, K, backend="int8")
    S, w, Q = plan.S, plan.w, plan.Q
    mu = shifts_mp(A, 0, Q)
    nu = shifts_mp(B, 1, Q)
    DA = digits_mp(A, mu, 0, w, S)
    DB = digits_mp(B, nu, 1, w, S)
    tg = {}
    for l, ml in enumerate(plan.moduli):
        RA = [np.array([[centered_residue(int(v), ml) for v in row] for row in DA[t]],
                       dtype=np.int64) for t in range(S)]
        RB = [np.array([[centered_residue(int(v), ml) for v in row] for row in DB[t]],
                       dtype=np.int64) for t in range(S)]
        for g in plan.groups:
            acc = np.zeros((m, n), dtype=np.int64)
            for ta in range(S):
                tb = g - ta
                if 0 <= tb < S:
                    acc += RA[ta] @ RB[tb]
            tg[(l, g)] = ((acc % ml) * plan.y[l]) % ml
    Sbar = {g: np.empty((m, n), dtype=object) for g in plan.groups}
    for g in plan.groups:
        for i in range(m):
            for j in range(n):
                Sbar[g][i, j] = crt_cpu([tg[(l, g)][i, j] for l in range(plan.N)], plan)
    Wb = window_bits(plan, K)
    Pint = np.empty((m, n), dtype=object)
    out = []
    for i in range(m):
        row = []
        for j in range(n):
            v = 0
            for g in plan.groups:
                v += int(Sbar[g][i, j]) << (w * (g - plan.g0))
            Pint[i, j] = v
            E = w * plan.g0 - mu[i] - nu[j]
            cold = C[i][j] if (beta and C is not None) else (0, 0)
            if cold[0] != 0:
                e_top = max(E + abs(v).bit_length(), frexp_exp(cold)) + 1
                if e_top - E > Wb:
                    E2 = e_top - Wb
                    v = -((-v) >> (E2 - E)) if v < 0 else v >> (E2 - E)
                    E = E2
                total = trunc_scaled(cold, -E) + alpha * v
            else:
                total = alpha * v
            row.append(bf_round(total, E, p))
        out.append(row)
    if debug:
        return out, (plan, mu, nu, tg, Sbar, Pint)
    return out
