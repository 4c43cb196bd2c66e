"""Seeded matrix generators (no Ozaki-II or LU arithmetic here)."""
from __future__ import annotations

from fractions import Fraction

import numpy as np


def random_expansions(rows: int, cols: int, nc: int, seed: int,
                      emin: int = -30, emax: int = 30) -> np.ndarray:
    """(rows, cols, nc) float64 array of non-overlapping expansions.

    x[0] = u * 2^e with u uniform [-1, 1), e uniform in [emin, emax];
    x[c+1] = u' * 2^(E(x[c]) - 55) with u' uniform (-1, 1) and E the frexp
    exponent, so |x[c+1]| < ulp(x[c]) / 4 and x[c] = RN(x[c] + x[c+1] + ...).
    """
    rng = np.random.default_rng(seed)
    out = np.zeros((rows, cols, nc), dtype=np.float64)
    lead = rng.uniform(-1.0, 1.0, size=(rows, cols))
    expo = rng.integers(emin, emax, size=(rows, cols), endpoint=True)
    out[..., 0] = np.ldexp(lead, expo)
    for c in range(1, nc):
        _, e = np.frexp(out[..., c - 1])
        u = rng.uniform(-1.0, 1.0, size=(rows, cols))
        nxt = np.ldexp(u, e - 55)
        nxt[out[..., c - 1] == 0.0] = 0.0
        out[..., c] = nxt
    return out


def rational_to_expansion(v: Fraction, nc: int) -> list[float]:
    """Successive correctly rounded binary64 components of a rational.

    Fraction -> float is correctly rounded (ties to even), and subtracting
    the rounded component is exact in rationals.
    """
    out = []
    rem = Fraction(v)
    for _ in range(nc):
        x = float(rem)
        out.append(x)
        rem -= Fraction(x)
    return out


def lotkin_expansions(n: int, nc: int) -> np.ndarray:
    """Lotkin matrix (Sec. 4.4): row 0 all ones, 1/(i+j+1) below (0-based).

    Returned as (n, n, nc) float64: element [i, j] holds the nc components.
    """
    vals = {d: rational_to_expansion(Fraction(1, d), nc) for d in range(1, 2 * n)}
    out = np.zeros((n, n, nc), dtype=np.float64)
    out[0, :, 0] = 1.0
    for i in range(1, n):
        for j in range(n):
            out[i, j, :] = vals[i + j + 1]
    return out


def lotkin_rhs(n: int, nc: int) -> np.ndarray:
    """b = A * ones of the exact rational Lotkin matrix, rounded: (n, nc)."""
    b = np.zeros((n, nc), dtype=np.float64)
    b[0, :] = rational_to_expansion(Fraction(n), nc)
    for i in range(1, n):
        s = sum((Fraction(1, i + j + 1) for j in range(n)), Fraction(0))
        b[i, :] = rational_to_expansion(s, nc)
    return b
