"""Exact checks of LU factors returned by the GPU (test helper, host only).

The factors of an LU are not unique functions of the rounding order, so the
GPU's factors are checked by properties every correct factorisation has,
evaluated in exact integer arithmetic from the stored binary64 components
(never through the library's own GEMM):

  * entries of the backward error P A - L U at sampled positions, each an
    exact dot product of length min(i, j) + 1;
  * the probe P A z - L (U z) for a random sign vector z, exact in O(n^2);
  * |l_ij| <= 1 (partial pivoting) and the interchanges a valid sequence.

An expansion element (nc binary64 components) is the exact dyadic value
N 2^E, the sum of its components.
"""
from __future__ import annotations

import math

import numpy as np


def _dyadic_rows(X: np.ndarray):
    """(k, nc) components -> k exact (N, E) pairs (vectorised frexp)."""
    mant, ex = np.frexp(X)
    M = (mant * 2.0 ** 53).astype(np.int64)
    E = ex.astype(np.int64) - 53
    out = []
    for i in range(X.shape[0]):
        terms = [(int(M[i, c]), int(E[i, c])) for c in range(X.shape[1]) if M[i, c] != 0]
        if not terms:
            out.append((0, 0))
            continue
        e0 = min(e for _, e in terms)
        out.append((sum(m << (e - e0) for m, e in terms), e0))
    return out


def _sum(pairs):
    pairs = [(n, e) for n, e in pairs if n]
    if not pairs:
        return (0, 0)
    e0 = min(e for _, e in pairs)
    return (sum(n << (e - e0) for n, e in pairs), e0)


def _log2_abs(x) -> float:
    n, e = x
    if n == 0:
        return -math.inf
    n = abs(n)
    b = n.bit_length()
    top = n >> max(0, b - 60)
    return math.log2(top) + max(0, b - 60) + e


def permuted(A: np.ndarray, ipiv) -> np.ndarray:
    """P A for LAPACK interchanges ipiv (1-based): row k swapped with ipiv[k]."""
    PA = np.array(A, copy=True)
    for k, p in enumerate(ipiv):
        p = int(p) - 1
        if p != k:
            PA[[k, p]] = PA[[p, k]]
    return PA


class ExactLU:
    """Exact residuals of the factors LU (unit L below, U on and above) of P A."""

    def __init__(self, A: np.ndarray, LU: np.ndarray, ipiv):
        self.n = A.shape[0]
        self.PA = permuted(A, ipiv)
        self.LU = LU
        self._lrow, self._ucol = {}, {}
        lead = np.abs(A[..., 0])
        self.log2_amax = math.log2(float(lead.max())) if lead.max() > 0 else -math.inf

    def _L(self, i):
        if i not in self._lrow:
            self._lrow[i] = _dyadic_rows(self.LU[i, :i])
        return self._lrow[i]

    def _U(self, j, upto):
        col = self._ucol.get(j)
        if col is None or len(col) < upto:
            col = _dyadic_rows(self.LU[:min(j + 1, self.n), j])
            self._ucol[j] = col
        return col

    def residual(self, i: int, j: int):
        """(P A - L U)_ij exactly, as (N, E)."""
        k1 = min(i, j) + 1
        L = self._L(i)
        U = self._U(j, k1)
        terms = []
        for k in range(k1):
            u = U[k]
            if k == i:                      # unit diagonal of L
                terms.append((-u[0], u[1]))
            else:
                lv = L[k]
                terms.append((-lv[0] * u[0], lv[1] + u[1]))
        terms.append(_dyadic_rows(self.PA[i, j][None, :])[0])
        return _sum(terms)

    def sampled_bits(self, pairs) -> float:
        """log2 max |P A - L U|_ij / max |A| over the sampled (i, j)."""
        worst = max((_log2_abs(self.residual(i, j)) for i, j in pairs), default=-math.inf)
        return worst - self.log2_amax

    def probe_bits(self, seed: int = 0) -> float:
        """log2 max_i |(P A z - L (U z))_i| / (max |A| n) for a random sign vector z.

        O(n^2) exact operations: U z first, then L (U z)."""
        n = self.n
        rng = np.random.default_rng(seed)
        z = rng.choice([-1, 1], size=n)
        Ud = [_dyadic_rows(self.LU[k, k:]) for k in range(n)]
        uz = [_sum([(int(z[k + t]) * a, e) for t, (a, e) in enumerate(Ud[k])]) for k in range(n)]
        worst = -math.inf
        for i in range(n):
            Li = self._L(i)
            lhs = _sum([(int(z[j]) * a, e) for j, (a, e) in
                        enumerate(_dyadic_rows(self.PA[i]))])
            terms = [lhs, (-uz[i][0], uz[i][1])]
            terms += [(-Li[k][0] * uz[k][0], Li[k][1] + uz[k][1]) for k in range(i)]
            worst = max(worst, _log2_abs(_sum(terms)))
        return worst - self.log2_amax - math.log2(n)


def l_bounded(LU: np.ndarray) -> bool:
    """|l_ij| <= 1 below the diagonal (partial pivoting), by the leading component
    (|x| <= 1 for an expansion iff its leading component is, or it is exactly 1
    minus a tiny tail: the leading component then equals 1)."""
    n = LU.shape[0]
    low = np.tril(np.ones((n, n), dtype=bool), -1)
    return bool(np.all(np.abs(LU[..., 0])[low] <= 1.0))


def valid_interchanges(ipiv, n: int) -> bool:
    """LAPACK interchanges: row k is swapped with a row at or below it."""
    return all(k + 1 <= int(p) <= n for k, p in enumerate(ipiv))
