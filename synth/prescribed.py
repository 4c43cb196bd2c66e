"""Prescribed-condition matrices A = U diag(sigma) V^T stored as expansions.

U and V are the orthogonal factors of numpy's Householder QR of seeded
N(0, 1) matrices (binary64).  The product is formed EXACTLY so that the stored
expansion matrix keeps the prescribed spectrum: an inexact binary64 product
would perturb it by about 1e-16 and swamp singular values below that.  To
make an exact product cheap, the factors are first put on small grids:
  * U and V on the fixed-point grid 2^-22 (|u| <= 1, 22-bit integers); the
    perturbation of an orthogonal factor is below 2^-23 per entry, so the
    singular values of A stay within a relative 1e-3 of sigma;
  * sigma_k = 10^(-c k / (n - 1)) rounded to 4 significant bits,
    m_k 2^(e_k - 3) with m_k in [8, 15].
Then A = sum_e 2^(e - 47) T_e with T_e = (U_G diag(m_G)) V_G^T over the index
group G of each exponent e; every T_e is an exact integer product in
binary64 (|entries| < 2^53 with at most 32 terms per group).  The T_e are
accumulated exactly in 24-bit integer limbs (int64 tensors, torch, on the
given device), and each element is rounded into nc binary64 components by
successive round-to-nearest-even.  All of it is exact integer arithmetic,
so the result does not depend on the device or the summation order; only
numpy's QR can differ between machines.
"""
from __future__ import annotations

import numpy as np

LIMB = 24
MASK = (1 << LIMB) - 1
GRID_BITS = 22


def factors(n: int, log10_cond: float, seed: int):
    """Quantised U, V (integers on 2^-22), m_k and e_k of the construction."""
    rng = np.random.default_rng(seed)
    U = np.linalg.qr(rng.standard_normal((n, n)))[0]
    V = np.linalg.qr(rng.standard_normal((n, n)))[0]
    Ui = np.rint(U * 2.0 ** GRID_BITS)
    Vi = np.rint(V * 2.0 ** GRID_BITS)
    k = np.arange(n, dtype=np.float64)
    sig = 10.0 ** (-log10_cond * k / max(n - 1, 1))
    e = np.floor(np.log2(sig)).astype(np.int64)
    m = np.rint(sig / np.ldexp(1.0, e - 3))
    top = m >= 16
    m[top] = 8
    e[top] += 1
    return Ui, Vi, m, e


def _groups(e: np.ndarray):
    order = np.argsort(-e, kind="stable")
    groups = []
    start = 0
    while start < len(order):
        stop = start
        while stop < len(order) and e[order[stop]] == e[order[start]] and stop - start < 32:
            stop += 1
        groups.append((int(e[order[start]]), order[start:stop]))
        start = stop
    return groups


def _pow2(e):
    """Exact 2^e as float64 from its bit pattern (e an int64 tensor in [-1022, 1023]).

    torch.ldexp multiplies by pow(2, e), which a device math library need not
    return exactly; a power of two built from its exponent field always is.
    """
    import torch
    return ((e + 1023) << 52).view(torch.float64)


def _scale2(x, e):
    """x * 2^e exactly (results in the normal range), e an int64 tensor."""
    import torch
    e1 = e.clamp(-1000, 1000)
    return x * _pow2(e1) * _pow2(e - e1)


def _carry(L):
    import torch
    for q in range(L.shape[0] - 1):
        c = torch.div(L[q], 1 << LIMB, rounding_mode="floor")
        L[q] -= c << LIMB
        L[q + 1] += c
    return L


def prescribed_cond_expansions(n: int, log10_cond: float, seed: int, nc: int,
                               device: str = "cpu"):
    """(n, n, nc) float64 torch tensor on `device` holding A = U diag(sigma) V^T."""
    import torch

    Ui, Vi, m, e = factors(n, log10_cond, seed)
    groups = _groups(e)
    emin = min(g for g, _ in groups)
    nlimbs = (53 + (max(g for g, _ in groups) - emin) + 8) // LIMB + 3
    L = torch.zeros((nlimbs, n, n), dtype=torch.int64, device=device)
    # torch's CPU matmul (not numpy's BLAS, whose spinning threads would
    # fight torch's between calls): every partial sum is an integer below
    # 2^53, so the product is exact in any summation order
    Ut = torch.from_numpy(Ui * m[None, :])
    Vt = torch.from_numpy(Vi)
    for g, idx in groups:
        ix = torch.from_numpy(np.asarray(idx))
        t = (Ut[:, ix] @ Vt[:, ix].T).to(torch.int64).to(device)   # exact integers
        s = g - emin
        q, r = divmod(s, LIMB)
        parts = [t & MASK, (t >> LIMB) & MASK, t >> (2 * LIMB)]
        for j, pt in enumerate(parts):
            L[q + j] += pt << r
    L = _carry(L)
    # value = N * 2^(emin - 3 - 2 GRID_BITS)
    scale_exp = emin - 3 - 2 * GRID_BITS
    neg = L[-1] < 0
    L = torch.where(neg.unsqueeze(0), -L, L)
    L = _carry(L)
    return _round_limbs(L, neg, scale_exp, nc)


def _round_limbs(L, neg, scale_exp: int, nc: int):
    """Successive round-to-nearest-even of sign * sum_q L[q] 2^(24 q) 2^scale_exp."""
    import torch

    nl = L.shape[0]
    out = torch.zeros(L.shape[1:] + (nc,), dtype=torch.float64, device=L.device)
    sign = torch.where(neg, -1.0, 1.0).to(torch.float64)
    ar = torch.arange(nl, device=L.device).view(-1, *([1] * (L.dim() - 1)))
    for c in range(nc):
        nz = L != 0
        any_nz = nz.any(0)
        top = torch.where(nz, ar.expand_as(L), torch.full_like(L, -1)).amax(0)
        topc = top.clamp(min=0)
        tl = torch.gather(L, 0, topc.unsqueeze(0))[0]
        bl = torch.zeros_like(tl)
        for b in range(LIMB):
            bl = torch.where((tl >> b) > 0, torch.full_like(bl, b + 1), bl)
        Lbits = topc * LIMB + bl                       # bit length of |N|
        shift = (Lbits - 62).clamp(min=0)
        q = torch.div(shift, LIMB, rounding_mode="floor")
        r = shift - q * LIMB
        W = torch.zeros_like(tl)
        for k in range(4):
            idx = (q + k).clamp(max=nl - 1)
            lk = torch.gather(L, 0, idx.unsqueeze(0))[0]
            lk = torch.where(q + k < nl, lk, torch.zeros_like(lk))
            sh = LIMB * k - r
            W += torch.where(sh >= 0, lk << sh.clamp(min=0), lk >> (-sh).clamp(min=0))
        # sticky: any bit below `shift`
        below = torch.cumsum(nz.to(torch.int64), 0)       # nonzero limbs up to q
        qm1 = (q - 1).clamp(min=0)
        lower_any = torch.where(q > 0, torch.gather(below, 0, qm1.unsqueeze(0))[0] > 0,
                                torch.zeros_like(any_nz))
        lq = torch.gather(L, 0, q.clamp(max=nl - 1).unsqueeze(0))[0]
        part_any = (lq & ((torch.ones_like(r) << r) - 1)) != 0
        sticky = (lower_any | part_any) & (shift > 0)
        W = W | sticky.to(torch.int64)
        x = W.to(torch.float64)                           # round to nearest even
        out[..., c] = torch.where(any_nz, sign * _scale2(x, shift + scale_exp), torch.zeros_like(x))
        # subtract the rounded value: R = int(x) (<= 2^62) placed at bit `shift`
        R = torch.where(any_nz, x.to(torch.int64), torch.zeros_like(W))
        pieces = [R & MASK, (R >> LIMB) & MASK, R >> (2 * LIMB)]
        for j, pc in enumerate(pieces):
            idx = (q + j).clamp(max=nl - 1)
            L.scatter_add_(0, idx.unsqueeze(0), (-(pc << r)).unsqueeze(0))
        L = _carry(L)
        flip = L[-1] < 0
        L = torch.where(flip.unsqueeze(0), -L, L)
        L = _carry(L)
        sign = torch.where(flip, -sign, sign)
    return out


def exact_row_sums(A, nc: int):
    """b_i = sum_j A_ij of an expansion matrix, exactly, rounded to nc components.

    A is a (rows, cols, nc_in) float64 torch tensor with A[i, j] the
    components of element (i, j).  Every component is an integer mantissa
    M (|M| < 2^53) times 2^E; all of them are accumulated exactly in 24-bit
    integer limbs relative to the smallest E, and the sum is rounded into
    nc binary64 components by successive round-to-nearest-even.  Used for
    right-hand sides b = A * ones of the stored (already rounded) matrix.
    """
    import torch

    rows = A.shape[0]
    v = A.reshape(rows, -1)
    mant, ex = torch.frexp(v)
    M = (mant * 2.0 ** 53).to(torch.int64)                    # exact: |M| < 2^53
    nz = M != 0
    out = torch.zeros((rows, nc), dtype=torch.float64, device=A.device)
    if not bool(nz.any()):
        return out
    E = ex.to(torch.int64) - 53
    emin = int(E[nz].min())
    pos = torch.where(nz, E - emin, torch.zeros_like(E))
    q = torch.div(pos, LIMB, rounding_mode="floor")
    r = pos - q * LIMB
    # three pieces of |M| (< 2^53) shifted by r < 24: each below 2^48, and a
    # component adds at most one piece to a limb; chunks of 2^13 components
    # keep every limb below 2^62 between carries
    nl = int(q.max()) + 6
    L = torch.zeros((nl, rows), dtype=torch.int64, device=A.device)
    chunk = 1 << 13
    for c0 in range(0, M.shape[1], chunk):
        Mc, qc, rc = M[:, c0:c0 + chunk], q[:, c0:c0 + chunk], r[:, c0:c0 + chunk]
        sgn = torch.sign(Mc)
        aM = Mc.abs()
        ridx = torch.arange(rows, device=A.device).view(rows, 1).expand_as(Mc)
        for j, pc in enumerate((aM & MASK, (aM >> LIMB) & MASK, aM >> (2 * LIMB))):
            L.index_put_((qc + j, ridx), sgn * (pc << rc), accumulate=True)
        L = _carry(L)
    neg = L[-1] < 0
    L = torch.where(neg.unsqueeze(0), -L, L)
    L = _carry(L)
    return _round_limbs(L, neg, emin, nc)
