"""p-bit multi-limb path through the C ABI (ozlu_mp_gemm / ozlu_mp_getrf / ozlu_mp_getrs).

The GEMM must equal the oracle's exact replay (oracle.mp.oz2_gemm_mp) bit for
bit; the LU is checked by its pivots, its exact backward error and the
solution's correct bits against the oracle's p + 64-bit LU.
"""
import math
import random
from fractions import Fraction

import numpy as np
import pytest

from oracle import lu as olu
from oracle.bigfloat import bf_from_fraction
from oracle.mp import oz2_gemm_mp

from gpu_util import handle, ozlu, torch

pytestmark = pytest.mark.gpu


def rand_mp(rng, rows, cols, p, emin=-3, emax=3, zeros=0.0):
    out = []
    for _ in range(rows):
        row = []
        for _ in range(cols):
            if rng.random() < zeros:
                row.append((0, 0))
                continue
            N = rng.getrandbits(p) | (1 << (p - 1))
            if rng.random() < 0.5:
                N = -N
            row.append((N, rng.randint(emin, emax) - p))
        out.append(row)
    return out


def norm(pairs, L):
    """The (N, E) pairs the device format stores (N left-aligned in 32 L bits)."""
    out = []
    for row in pairs:
        r = []
        for N, E in row:
            if N == 0:
                r.append((0, 0))
                continue
            b = abs(N).bit_length()
            r.append((N << (32 * L - b), E - (32 * L - b)))
        out.append(r)
    return out


@pytest.mark.parametrize("m,n,k,p,alpha,beta", [
    (5, 7, 9, 300, 1, 0), (3, 4, 2, 1100, -1, 1), (1, 1, 1, 100, 1, 0), (6, 5, 3, 64, -1, 1),
    (130, 3, 40, 200, -1, 1)])
def test_mp_gemm_bit_exact(m, n, k, p, alpha, beta):
    rng = random.Random(m * 100 + n * 10 + k + p)
    L = (p + 31) // 32
    A = rand_mp(rng, m, k, p, zeros=0.1)
    B = rand_mp(rng, k, n, p, zeros=0.1)
    C = rand_mp(rng, m, n, p, emin=-2, emax=6, zeros=0.2)
    ref = oz2_gemm_mp(A, B, p, alpha=alpha, beta=beta, C=C if beta else None)
    h = handle()
    dA = ozlu.MPMatrix.from_pairs(A, L)
    dB = ozlu.MPMatrix.from_pairs(B, L)
    dC = ozlu.MPMatrix.from_pairs(C, L)
    ozlu.ozlu_mp_gemm(h, p, m, n, k, alpha, dA.desc(), dB.desc(), beta, dC.desc())
    torch.cuda.synchronize()
    assert dC.to_pairs() == norm(ref, L)


def test_mp_gemm_submatrix_and_chunk_views():
    """Views with offsets and leading dimensions (the LU's calls)."""
    rng = random.Random(11)
    p, L = 150, 5
    A = rand_mp(rng, 9, 8, p)
    h = handle()
    dA = ozlu.MPMatrix.from_pairs(A, L)
    # C(3:6, 5:8) -= A(3:6, 0:2) A(0:2, 5:8)
    sub = lambda M, i0, i1, j0, j1: [row[j0:j1] for row in M[i0:i1]]
    ref = oz2_gemm_mp(sub(A, 3, 6, 0, 2), sub(A, 0, 2, 5, 8), p, alpha=-1, beta=1, C=sub(A, 3, 6, 5, 8))
    ozlu.ozlu_mp_gemm(h, p, 3, 3, 2, -1, dA.desc(3, 0), dA.desc(0, 5), 1, dA.desc(3, 5))
    torch.cuda.synchronize()
    got = dA.to_pairs()
    assert sub(got, 3, 6, 5, 8) == norm(ref, L)
    assert sub(got, 0, 3, 0, 8) == norm(sub(A, 0, 3, 0, 8), L)


def lotkin_mp(n, p):
    return [[bf_from_fraction(v, p) for v in row] for row in olu.lotkin(n)]


def value(x):
    return Fraction(x[0]) * Fraction(2) ** x[1]


def factor(A, n, p, nb):
    L = (p + 31) // 32
    h = handle()
    dA = ozlu.MPMatrix.from_pairs(A, L)
    ipiv = torch.zeros(n, dtype=torch.int32, device="cuda")
    info = torch.full((1,), -5, dtype=torch.int32, device="cuda")
    ozlu.ozlu_mp_getrf(h, p, n, dA.desc(), ipiv, nb, info)
    torch.cuda.synchronize()
    return h, dA, ipiv, int(info.item())


def backward_error(A, LU, piv, n):
    Af = [[value(x) for x in row] for row in A]
    PA = olu.apply_ipiv_rows(Af, piv)
    Lf = [[value(LU[i][j]) if j < i else (Fraction(1) if i == j else Fraction(0)) for j in range(n)]
          for i in range(n)]
    Uf = [[value(LU[i][j]) if j >= i else Fraction(0) for j in range(n)] for i in range(n)]
    res = max(abs(PA[i][j] - sum(Lf[i][k] * Uf[k][j] for k in range(n))) for i in range(n) for j in range(n))
    return res / max(abs(v) for row in Af for v in row)


@pytest.mark.parametrize("n,p,nb", [(20, 160, 8), (33, 300, 16)])
def test_mp_lu_random_pivots_and_backward_error(n, p, nb):
    rng = random.Random(n + p)
    A = rand_mp(rng, n, n, p, emin=-1, emax=1)
    h, dA, ipiv, info = factor(A, n, p, nb)
    assert info == 0
    piv = [int(v) - 1 for v in ipiv.cpu().tolist()]
    _, piv_ref, _ = olu.lu_bigfloat([[bf_from_fraction(value(x), p + 64) for x in row] for row in A], p + 64)
    assert piv == piv_ref
    assert backward_error(A, dA.to_pairs(), piv, n) < Fraction(2) ** (-p + 3 * math.ceil(math.log2(n)) + 8)


@pytest.mark.parametrize("n,p,nb", [(24, 256, 8), (40, 416, 16), (17, 192, 32)])
def test_mp_lu_lotkin(n, p, nb):
    """Lotkin (Sec. 4.4): backward error at p bits, correct bits ~ p - log2 cond."""
    A = lotkin_mp(n, p)
    h, dA, ipiv, info = factor(A, n, p, nb)
    assert info == 0
    piv = [int(v) - 1 for v in ipiv.cpu().tolist()]
    assert backward_error(A, dA.to_pairs(), piv, n) < Fraction(2) ** (-p + 3 * math.ceil(math.log2(n)) + 8)
    Af = [[value(x) for x in row] for row in A]
    L = (p + 31) // 32
    b = [[bf_from_fraction(sum(row, Fraction(0)), p)] for row in Af]
    dB = ozlu.MPMatrix.from_pairs(b, L)
    ozlu.ozlu_mp_getrs(h, p, n, 1, dA.desc(), ipiv, dB.desc())
    torch.cuda.synchronize()
    x = [value(r[0]) for r in dB.to_pairs()]
    err = max(abs(v - 1) for v in x)
    bits = -math.log2(float(err)) if err else p
    assert bits > p - 5.3 * n - 16, bits


def test_mp_lu_singular():
    """A_ij = 2^(i+j) has rank 1 and the elimination is exact: info = 2."""
    p, n = 128, 6
    A = [[(1, i + j) for j in range(n)] for i in range(n)]
    h, dA, ipiv, info = factor(A, n, p, 4)
    assert info == 2


@pytest.mark.parametrize("p", [128, 1024, 1600, 3136])
def test_mp_reciprocal_through_1x1_solve(p):
    """x = 1 / a from a 1 x 1 solve: the reciprocal kernel at p + 32 bits, then one
    rounding to p bits (limb counts over one warp included)."""
    rng = random.Random(p)
    L = (p + 31) // 32
    N = rng.getrandbits(p) | (1 << (p - 1))
    A = ozlu.MPMatrix.from_pairs([[(N, -p + 3)]], L)
    B = ozlu.MPMatrix.from_pairs([[(1, 0)]], L)
    ipiv = torch.ones(1, dtype=torch.int32, device="cuda")
    ozlu.ozlu_mp_getrs(handle(), p, 1, 1, A.desc(), ipiv, B.desc())
    torch.cuda.synchronize()
    (xn, xe), = B.to_pairs()[0]
    ex = 1 / (Fraction(N) * Fraction(2) ** (-p + 3))
    err = abs(Fraction(xn) * Fraction(2) ** xe - ex) / ex
    assert err <= Fraction(2) ** (-p + 1)


@pytest.mark.parametrize("be", ["fp8", "int8", "auto"])
@pytest.mark.parametrize("m,n,k,p", [(140, 130, 40, 400), (130, 200, 300, 900), (257, 129, 9, 160)])
def test_mp_gemm_backends_same_bits(be, m, n, k, p):
    # wide p-bit products on FP8 (tcgen05, base-17 Karatsuba planes) or INT8
    # residues run the same plan, so both equal the oracle's replay bit for bit
    handle()
    rng = random.Random(m + 3 * n + 7 * k + p)
    L = (p + 31) // 32
    A = rand_mp(rng, m, k, p, zeros=0.05)
    B = rand_mp(rng, k, n, p, zeros=0.05)
    C = rand_mp(rng, m, n, p, emin=-2, emax=6, zeros=0.1)
    ref = oz2_gemm_mp(A, B, p, alpha=-1, beta=1, C=C)
    h = ozlu.ozlu_create(None)
    try:
        ozlu.ozlu_mp_set_opts(h, ozlu.make_opts(be))
        dA = ozlu.MPMatrix.from_pairs(A, L)
        dB = ozlu.MPMatrix.from_pairs(B, L)
        dC = ozlu.MPMatrix.from_pairs(C, L)
        ozlu.ozlu_mp_gemm(h, p, m, n, k, -1, dA.desc(), dB.desc(), 1, dC.desc())
        torch.cuda.synchronize()
        assert dC.to_pairs() == norm(ref, L)
        if be == "fp8":
            assert ozlu.ozlu_get_stats(h).last_backend == 2
        assert ozlu.ozlu_debug_fetch(h, 6, np.zeros(1, np.int32))[0] == 0
    finally:
        ozlu.ozlu_destroy(h)
