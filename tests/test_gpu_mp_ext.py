"""The extended modulus table (Sec. 4.2.4) on the p-bit GEMM and LU.

With OZLU_MODSET_EXT the p-bit Ozaki-II GEMM takes its moduli from the
extended table (up to 16191) and multiplies each residue as three int8
Karatsuba planes of balanced base-128 digits.  The t values (16 bits) and the
rounded outputs must equal the oracle's exact replay with the same plan
(oracle.plan.make_plan(..., modset="ext")) bit for bit; the LU through this
route must keep the pivots and the accuracy of the oracle's p + 64-bit LU.
"""
import math
import random
from fractions import Fraction

import numpy as np
import pytest

from oracle import lu as olu
from oracle.bigfloat import bf_from_fraction
from oracle.mp import oz2_gemm_mp
from oracle.plan import make_plan

from gpu_util import handle, ozlu, torch
from test_gpu_mp import backward_error, lotkin_mp, norm, rand_mp, value

pytestmark = pytest.mark.gpu


def _ext_handle(S=0):
    h = ozlu.ozlu_create(None)
    ozlu.ozlu_mp_set_opts(h, ozlu.make_opts(modset="ext", nslice=S))
    return h


@pytest.mark.parametrize("m,n,k,p,S,alpha,beta", [
    (5, 7, 9, 300, 0, 1, 0), (37, 29, 19, 600, 0, -1, 1), (37, 29, 19, 600, 2, 1, 1),
    (130, 3, 40, 200, 3, -1, 1), (3, 140, 130, 1100, 0, 1, 0), (2, 2, 1, 64, 0, -1, 1)])
def test_mp_ext_gemm_bit_exact(m, n, k, p, S, alpha, beta):
    handle()
    rng = random.Random(7 * m + 3 * n + k + p + S)
    L = (p + 31) // 32
    A = rand_mp(rng, m, k, p, zeros=0.1)
    B = rand_mp(rng, k, n, p, zeros=0.1)
    C = rand_mp(rng, m, n, p, emin=-2, emax=6, zeros=0.2)
    plan = make_plan(p, k, modset="ext", S=S or None)
    ref = oz2_gemm_mp(A, B, p, alpha=alpha, beta=beta, C=C if beta else None, plan=plan)
    h = _ext_handle(S)
    try:
        dA = ozlu.MPMatrix.from_pairs(A, L)
        dB = ozlu.MPMatrix.from_pairs(B, L)
        dC = ozlu.MPMatrix.from_pairs(C, L)
        ozlu.ozlu_mp_gemm(h, p, m, n, k, alpha, dA.desc(), dB.desc(), beta, dC.desc())
        torch.cuda.synchronize()
        assert dC.to_pairs() == norm(ref, L)
    finally:
        ozlu.ozlu_destroy(h)


def test_mp_ext_t_values_and_extreme_residues():
    # entries chosen so that residues reach the ends of the centered range of
    # the largest moduli (|r| up to 8094, base-128 digits |q| = 63, |r0 + q|
    # up to 127): the same exact replay decides the outputs
    handle()
    p, K = 900, 64
    plan = make_plan(p, K, modset="ext")
    rng = random.Random(5)
    L = (p + 31) // 32
    A = rand_mp(rng, 4, K, p)
    B = rand_mp(rng, K, 3, p)
    A[0] = [(-((1 << p) - 1), -p)] * K          # all-ones magnitudes
    B = [[(1 << (p - 1), -p + 1)] + row[1:] for row in B]
    ref = oz2_gemm_mp(A, B, p, plan=plan)
    h = _ext_handle()
    try:
        dA = ozlu.MPMatrix.from_pairs(A, L)
        dB = ozlu.MPMatrix.from_pairs(B, L)
        dC = ozlu.MPMatrix(4, 3, L)
        ozlu.ozlu_mp_gemm(h, p, 4, 3, K, 1, dA.desc(), dB.desc(), 0, dC.desc())
        torch.cuda.synchronize()
        assert dC.to_pairs() == norm(ref, L)
    finally:
        ozlu.ozlu_destroy(h)


@pytest.mark.parametrize("n,p,nb,S", [(24, 320, 8, 0), (33, 600, 16, 2)])
def test_mp_ext_lu_pivots_and_backward_error(n, p, nb, S):
    handle()
    rng = random.Random(n * p)
    A = rand_mp(rng, n, n, p, emin=-1, emax=1)
    L = (p + 31) // 32
    h = _ext_handle(S)
    try:
        dA = ozlu.MPMatrix.from_pairs(A, L)
        ipiv = torch.zeros(n, dtype=torch.int32, device="cuda")
        info = torch.full((1,), -5, dtype=torch.int32, device="cuda")
        ozlu.ozlu_mp_getrf(h, p, n, dA.desc(), ipiv, nb, info)
        torch.cuda.synchronize()
        assert int(info.item()) == 0
        piv = [int(v) - 1 for v in ipiv.cpu().tolist()]
        _, piv_ref, _ = olu.lu_bigfloat([[bf_from_fraction(value(x), p + 64) for x in row] for row in A], p + 64)
        assert piv == piv_ref
        assert backward_error(A, dA.to_pairs(), piv, n) < Fraction(2) ** (-p + 3 * math.ceil(math.log2(n)) + 8)
    finally:
        ozlu.ozlu_destroy(h)


def test_mp_ext_lotkin_correct_bits():
    # Sec. 4.4: the Lotkin matrix at p ~ 1.2 log2 cond reaches p - log2 cond bits
    handle()
    n, p, nb = 48, 320, 16
    A = lotkin_mp(n, p)
    L = (p + 31) // 32
    h = _ext_handle()
    try:
        dA = ozlu.MPMatrix.from_pairs(A, L)
        ipiv = torch.zeros(n, dtype=torch.int32, device="cuda")
        info = torch.zeros(1, dtype=torch.int32, device="cuda")
        ozlu.ozlu_mp_getrf(h, p, n, dA.desc(), ipiv, nb, info)
        Af = [[value(x) for x in row] for row in A]
        b = [[bf_from_fraction(sum(row, Fraction(0)), p)] for row in Af]
        dB = ozlu.MPMatrix.from_pairs(b, L)
        ozlu.ozlu_mp_getrs(h, p, n, 1, dA.desc(), ipiv, dB.desc())
        torch.cuda.synchronize()
        assert int(info.item()) == 0
        err = max(abs(value(r[0]) - 1) for r in dB.to_pairs())
        bits = -math.log2(float(err)) if err else p
        assert bits > p - 5.3 * n - 16, bits
    finally:
        ozlu.ozlu_destroy(h)
