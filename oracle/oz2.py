"""Ozaki-scheme-II GEMM replayed in exact integers, steps (S1)-(S6).

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

C = beta*C + alpha*A*B for expansion matrices, A: m x K, B: K x n, each entry
nc binary64 components (arrays of shape (rows, cols, nc)).  The steps follow
Sec. 3.1 (S1)-(S6), the slice splitting and CRT of Sec. 3.2 and the direct
conversion of Sec. 3.3, in the paper's order and notation:

  (S1) shared exponents mu_i, nu_j per row of A / column of B
  (S2) a_bar = trunc(2^mu_i a) as Q-bit integers, by Eq. (12)
       then S balanced w-bit digits v_t with X = sum_t v_t 2^(wt)  (Eq. (2))
  (S3) centered residues of every digit modulo every m_l
  (S4) C_g^(l) = sum_{ta+tb=g} A_ta^(l) B_tb^(l), exact integer products,
       digit groups g = S-1 .. 2S-2 retained (Eq. (3), Prop. 2)
  (S5) t_l = (C mod m_l) y_l mod m_l and the CRT of Eq. (11), here by the
       CPU procedure of Sec. 3.5.1: the representative in [0, P) first, then
       a comparison with floor(P/2) for the sign
  (S6) c_bar = sum_g S_g 2^(wg), scaled by 2^-(mu_i+nu_j), rounded once.

Readings:
  * S1: E_i = max_h of the frexp exponent of the leading component a_ih[0], so
    |a_ih| < 2^E_i; mu_i = (Q-1) - E_i, hence |a_bar| < 2^(Q-1); an all-zero
    row gets mu_i = 0.
  * S2: Eq. (12) is the definition of the conversion: each component is
    shifted as a sign and a 53-bit magnitude, a right shift truncating the
    magnitude, and the signed terms are summed.
  * Balanced digit: v = X mod 2^w taken in [-2^(w-1), 2^(w-1)).
  * Centered residue: r in [-floor(m/2), ceil(m/2)-1].
  * S6 with beta = 1: the exact sum of the old C, brought to the grid 2^E of
    the product with the same component-wise truncation as Eq. (12), and of
    alpha times the product integer, is rounded once; E is the product grid
    2^(w g0 - mu_i - nu_j) unless the old C reaches more than WINDOW_BITS
    above it, in which case the grid is raised to e_top - WINDOW_BITS and the
    product integer is truncated toward zero onto it.
  * fl_p: successive round-to-nearest of the exact integer into nc binary64
    components (oracle.expansion.fl_expansion).
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

from .expansion import double_to_dyadic, fl_expansion
from .plan import Plan, make_plan

# two's-complement window of the fused C update (16 words of 32 bits, one
# spare bit for the sign): see the S6 reading in the module docstring
WINDOW_BITS = 510


# ---------------------------------------------------------------- (S1) ----
def leading_exponent(values) -> int | None:
    """max over the given leading components of the frexp exponent (S1)."""
    best = None
    for x in values:
        x = float(x)
        if x != 0.0:
            e = math.frexp(x)[1]
            best = e if best is None else max(best, e)
    return best


def shared_shifts(X: np.ndarray, axis: int, Q: int) -> list[int]:
    """mu_i (axis=0: per row of A) or nu_j (axis=1: per column of B)."""
    lead = X[..., 0]
    count = lead.shape[axis]
    out = []
    for idx in range(count):
        vec = lead[idx, :] if axis == 0 else lead[:, idx]
        E = leading_exponent(vec)
        out.append(0 if E is None else (Q - 1) - E)
    return out


# ---------------------------------------------------------------- (S2) ----
def fixed_point(limbs, shift: int) -> int:
    """Eq. (12): sum_c +-(m_c << (e_c + shift - 53)); a negative shift count
    is a right shift of the magnitude (truncation toward zero)."""
    total = 0
    for x in limbs:
        n, e = double_to_dyadic(float(x))  # x = n 2^e, n = +-m_c
        if n == 0:
            continue
        mag = -n if n < 0 else n
        s = e + shift
        mag = mag << s if s >= 0 else mag >> (-s)
        total += -mag if n < 0 else mag
    return total


def balanced_digits(X: int, w: int, S: int) -> list[int]:
    """X = sum_{t<S} v_t 2^(wt) with |v_t| <= 2^(w-1) (Eq. (2)).

    Digits below the top one are X mod 2^w taken in [-2^(w-1), 2^(w-1));
    the top digit is what remains, which |X| < 2^(wS-1) keeps within
    2^(w-1).
    """
    digits = []
    rest = X
    base = 1 << w
    half = 1 << (w - 1)
    for _ in range(S - 1):
        v = rest % base
        if v >= half:
            v -= base
        digits.append(v)
        rest = (rest - v) >> w
    if abs(rest) > half:
        raise ValueError("value does not fit in S balanced digits")
    digits.append(rest)
    return digits


# ---------------------------------------------------------------- (S3) ----
def centered_residue(v: int, m: int) -> int:
    """Centered residue of v modulo m in [-floor(m/2), ceil(m/2) - 1] (S3)."""
    r = v % m
    if r > (m - 1) // 2:
        r -= m
    return r


def fp8_base17_digits(r: int) -> tuple[int, int]:
    """Eq. (15): r = 17 d1 + d0 with d1 = round(r/17) (never a tie: 17 is odd)."""
    d1 = (2 * r + 17) // 34  # nearest integer to r/17
    d0 = r - 17 * d1
    return d0, d1


# ------------------------------------------------------------- plumbing ----
@dataclass
class Oz2Debug:
    plan: Plan
    mu: list
    nu: list
    digits_A: list          # [t] object arrays (m, K)
    digits_B: list          # [t] object arrays (K, n)
    res_A: dict             # (l, t) -> int64 (m, K)
    res_B: dict             # (l, t) -> int64 (K, n)
    C: dict                 # (l, g) -> int64 (m, n)
    t: dict                 # (l, g) -> int64 (m, n) in [0, m_l)
    Sbar: dict              # g -> object (m, n)
    Pint: np.ndarray        # object (m, n): sum_g Sbar_g 2^(w (g-g0))


def _digit_matrices(X: np.ndarray, shifts: list, axis: int, w: int, S: int):
    rows, cols = X.shape[0], X.shape[1]
    D = [np.empty((rows, cols), dtype=object) for _ in range(S)]
    for i in range(rows):
        for j in range(cols):
            sh = shifts[i] if axis == 0 else shifts[j]
            v = balanced_digits(fixed_point(X[i, j], sh), w, S)
            for t in range(S):
                D[t][i, j] = v[t]
    return D


def _residues(D: np.ndarray, m: int) -> np.ndarray:
    flat = [centered_residue(int(v), m) for v in D.ravel()]
    return np.array(flat, dtype=np.int64).reshape(D.shape)


def crt_cpu(tvals: list, plan: Plan) -> int:
    """S_g from t_l by Eq. (11), CPU procedure of Sec. 3.5.1.

    sum_l t_l M_l taken modulo P gives the representative in [0, P); values
    above floor(P/2) stand for negatives and have P subtracted.
    """
    X = sum(int(t) * Ml for t, Ml in zip(tvals, plan.M)) % plan.P
    if X > plan.P // 2:
        X -= plan.P
    return X


def crt_round(tvals: list, plan: Plan) -> int:
    """S_g by Eq. (11) as written: sum t_l M_l - round(sum t_l/m_l) P.

    Evaluated with exact rationals; used only to pin crt_cpu against the
    round-to-nearest form the paper derives (they must agree).
    """
    from fractions import Fraction
    F = sum(Fraction(int(t), m) for t, m in zip(tvals, plan.moduli))
    R = math.floor(F + Fraction(1, 2))
    return sum(int(t) * Ml for t, Ml in zip(tvals, plan.M)) - R * plan.P


def _trunc_shift(N: int, s: int) -> int:
    """sign(N) * (|N| >> s): truncation toward zero by 2^s."""
    if s <= 0:
        return N << (-s)
    return -((-N) >> s) if N < 0 else N >> s


def grid_expansion(limbs, E: int) -> int:
    """Old C on the grid 2^E, component-wise as Eq. (12) does for inputs."""
    return fixed_point(limbs, -E)


def assemble_output(Pint: int, E0: int, alpha: int, beta: int, cold, nc: int):
    """(S6): the single rounding, fused with C <- beta C + alpha (A B)."""
    if beta == 0 or cold is None or all(float(x) == 0.0 for x in cold):
        return fl_expansion(alpha * Pint, E0, nc)
    e_top = E0 + (abs(Pint).bit_length() if Pint != 0 else 0)
    c0 = float(cold[0])
    if c0 != 0.0:
        e_top = max(e_top, math.frexp(c0)[1])
    e_top += 1
    E = E0 if e_top - E0 <= WINDOW_BITS else e_top - WINDOW_BITS
    N = grid_expansion(cold, E) + alpha * _trunc_shift(Pint, E - E0)
    return fl_expansion(N, E, nc)


def oz2_gemm(A: np.ndarray, B: np.ndarray, p: int, alpha: int = 1,
             beta: int = 0, C: np.ndarray | None = None, backend: str = "int8",
             g_ex: int = 0, extra_groups: int = 0, S: int | None = None,
             plan: Plan | None = None, debug: bool = False):
    """Ozaki-II C = beta C + alpha A B, exact replay of (S1)-(S6).

    A: (m, K, nc), B: (K, n, nc), C: (m, n, nc) float64 arrays.
    The output entries depend only on row i of A and column j of B, so a
    sampled check passes A[rows] and B[:, cols].
    """
    m, K, nc = A.shape
    K2, n, nc2 = B.shape
    assert K == K2 and nc == nc2
    if plan is None:
        plan = make_plan(p, K, backend=backend, g_ex=g_ex,
                         extra_groups=extra_groups, S=S)
    S_, w, Q = plan.S, plan.w, plan.Q
    mu = shared_shifts(A, 0, Q)                     # (S1)
    nu = shared_shifts(B, 1, Q)
    DA = _digit_matrices(A, mu, 0, w, S_)           # (S2)
    DB = _digit_matrices(B, nu, 1, w, S_)
    res_A, res_B = {}, {}
    for l, ml in enumerate(plan.moduli):            # (S3)
        for t in range(S_):
            res_A[(l, t)] = _residues(DA[t], ml)
            res_B[(l, t)] = _residues(DB[t], ml)
    Cg, tg = {}, {}
    for l, ml in enumerate(plan.moduli):            # (S4) and t_l of (S5)
        for g in plan.groups:
            acc = np.zeros((m, n), dtype=np.int64)
            for ta in range(S_):
                tb = g - ta
                if 0 <= tb < S_:
                    acc += res_A[(l, ta)] @ res_B[(l, tb)]
            Cg[(l, g)] = acc
            tg[(l, g)] = ((acc % ml) * plan.y[l]) % ml
    Sbar = {}
    for g in plan.groups:                           # (S5) CRT per group
        sg = np.empty((m, n), dtype=object)
        for i in range(m):
            for j in range(n):
                sg[i, j] = crt_cpu([tg[(l, g)][i, j] for l in range(plan.N)], plan)
        Sbar[g] = sg
    Pint = np.empty((m, n), dtype=object)           # (S6)
    out = np.zeros((m, n, nc), dtype=np.float64)
    for i in range(m):
        for j in range(n):
            v = 0
            for g in plan.groups:
                v += int(Sbar[g][i, j]) << (w * (g - plan.g0))
            Pint[i, j] = v
            E0 = w * plan.g0 - mu[i] - nu[j]
            cold = C[i, j] if (beta and C is not None) else None
            out[i, j, :] = assemble_output(v, E0, alpha, beta, cold, nc)
    if debug:
        return out, Oz2Debug(plan, mu, nu, DA, DB, res_A, res_B, Cg, tg, Sbar, Pint)
    return out


def digit_group_exact(DA: list, DB: list, g: int, S: int) -> np.ndarray:
    """sum_{ta+tb=g} V_ta U_tb in exact integers (the quantity S_g must equal)."""
    acc = None
    for ta in range(S):
        tb = g - ta
        if 0 <= tb < S:
            prod = DA[ta].dot(DB[tb])
            acc = prod if acc is None else acc + prod
    return acc


def exact_gemm(A: np.ndarray, B: np.ndarray):
    """c_ij = sum_h a_ih b_hj exactly, as an object array of (N, E) pairs."""
    m, K, _ = A.shape
    n = B.shape[1]
    dA = [[_exp_dyadic(A[i, h]) for h in range(K)] for i in range(m)]
    dB = [[_exp_dyadic(B[h, j]) for j in range(n)] for h in range(K)]
    out = np.empty((m, n), dtype=object)
    for i in range(m):
        for j in range(n):
            terms = [(dA[i][h][0] * dB[h][j][0], dA[i][h][1] + dB[h][j][1])
                     for h in range(K) if dA[i][h][0] and dB[h][j][0]]
            if not terms:
                out[i, j] = (0, 0)
                continue
            E = min(e for _, e in terms)
            out[i, j] = (sum(N << (e - E) for N, e in terms), E)
    return out


def _exp_dyadic(limbs):
    parts = [double_to_dyadic(float(x)) for x in limbs if float(x) != 0.0]
    if not parts:
        return (0, 0)
    E = min(e for _, e in parts)
    return (sum(n << (e - E) for n, e in parts), E)


def gamma_factor(A: np.ndarray, B: np.ndarray, exact=None) -> np.ndarray:
    """Eq. (7) per element: max_h|a_ih| max_h|b_hj| / |c_ij| (inf if c = 0)."""
    from .expansion import expansion_value
    m, K, _ = A.shape
    n = B.shape[1]
    amax = [max(abs(expansion_value(A[i, h])) for h in range(K)) for i in range(m)]
    bmax = [max(abs(expansion_value(B[h, j])) for h in range(K)) for j in range(n)]
    if exact is None:
        exact = exact_gemm(A, B)
    out = np.empty((m, n), dtype=float)
    for i in range(m):
        for j in range(n):
            N, E = exact[i, j]
            if N == 0:
                out[i, j] = math.inf
            else:
                from fractions import Fraction
                c = abs(Fraction(N) * Fraction(2) ** E)
                out[i, j] = float(amax[i] * bmax[j] / c)
    return out
