"""GPU LU (ozlu_getrf / ozlu_getrs through the C ABI) against exact checks.

Factors of an LU are not unique functions of the rounding order, so the
checks are the properties that hold for any correct factorisation:
  * the backward error max|P A - L U| / max|A|, computed exactly from the
    returned factors, is a small multiple of 2^-p;
  * |l_ij| <= 1 (partial pivoting) and the interchanges match the oracle's
    p + 64-bit LU on well-conditioned matrices (no near ties);
  * the solve of A x = A * ones reaches p - log2 cond - a few correct bits
    (Sec. 4.4's measure), and its residual is small on the Lotkin matrix;
  * singular input reports the first zero pivot in info.
"""
import math
from fractions import Fraction

import numpy as np
import pytest

from oracle import lu as olu
from oracle.bigfloat import bf_from_fraction, bf_to_fraction
from oracle.expansion import double_to_dyadic
from synth import lotkin_expansions, lotkin_rhs, random_expansions

from gpu_util import dev, handle, host, ozlu, torch

pytestmark = pytest.mark.gpu


def _ints(X):
    """(rows, cols, nc) expansions -> integer matrix and common exponent."""
    rows, cols, nc = X.shape
    parts = [[[double_to_dyadic(float(v)) for v in X[i, j]] for j in range(cols)] for i in range(rows)]
    E = min(e for r in parts for c in r for (N, e) in c if N)
    M = [[sum(N << (e - E) for N, e in c if N) for c in r] for r in parts]
    return M, E


def _backward_error_bits(A, LU, ipiv):
    n = A.shape[0]
    a, ea = _ints(A)
    f, ef = _ints(LU)
    pa = [list(r) for r in a]
    for k in range(n):
        p = ipiv[k] - 1
        pa[k], pa[p] = pa[p], pa[k]
    one = 1 << (-ef) if ef < 0 else None
    worst = 0
    # (L U)_ij at exponent 2 ef; P A at ea
    E = min(ea, 2 * ef)
    for i in range(n):
        for j in range(n):
            s = 0
            for k in range(min(i, j) + 1):
                lik = one if k == i else f[i][k]
                s += lik * f[k][j]
            d = (pa[i][j] << (ea - E)) - (s << (2 * ef - E))
            worst = max(worst, abs(d))
    amax = max(abs(v) for r in a for v in r)
    if worst == 0:
        return -math.inf
    return math.log2(worst) + E - (math.log2(amax) + ea)


def _getrf(A, nb, p=0):
    h = handle()
    n, _, nc = A.shape
    dA = dev(A)
    ipiv = torch.zeros(n, dtype=torch.int32, device="cuda")
    info = torch.zeros(1, dtype=torch.int32, device="cuda")
    ozlu.ozlu_getrf(h, nc, p, n, dA, n, ipiv, nb, info)
    torch.cuda.synchronize()
    return dA, host(dA, n), ipiv.cpu().numpy(), int(info.item())


def _getrs(dA, ipiv, b, p=0):
    h = handle()
    n, nc = b.shape
    db = torch.from_numpy(np.ascontiguousarray(b[None, :, :])).cuda()
    ozlu.ozlu_getrs(h, nc, p, n, 1, dA, n, torch.from_numpy(ipiv).cuda(), db, n)
    torch.cuda.synchronize()
    return db.cpu().numpy()[0]


def _value(limbs):
    return sum((Fraction(float(v)) for v in limbs), Fraction(0))


@pytest.mark.parametrize("nc,n,nb", [(4, 100, 64), (2, 77, 32), (3, 130, 64), (4, 40, 256),
                                     (2, 1, 256), (4, 70, 16)])
def test_getrf_backward_error_and_pivots(nc, n, nb):
    A = random_expansions(n, n, nc, 500 + n, -2, 2)
    dA, LU, ipiv, info = _getrf(A, nb)
    assert info == 0
    bits = _backward_error_bits(A, LU, ipiv)
    assert bits < -53 * nc + math.log2(n) + 12, bits
    # |l_ij| <= 1
    for i in range(n):
        for j in range(i):
            assert abs(LU[i, j, 0]) <= 1.0 + 1e-15
    if n <= 80:
        prec = 53 * nc + 64
        Af = [[_value(A[i, j]) for j in range(n)] for i in range(n)]
        _, ipiv_ref, _ = olu.lu_bigfloat(olu.to_bigfloat_matrix(Af, prec), prec)
        assert [p + 1 for p in ipiv_ref] == list(ipiv)


@pytest.mark.parametrize("nc,n", [(4, 60), (2, 45)])
def test_getrs_correct_bits(nc, n):
    A = random_expansions(n, n, nc, 900 + n, -1, 1)
    Af = [[_value(A[i, j]) for j in range(n)] for i in range(n)]
    b_exact = olu.matvec(Af, [Fraction(1)] * n)
    from synth import rational_to_expansion
    b = np.array([rational_to_expansion(v, nc) for v in b_exact])
    dA, LU, ipiv, info = _getrf(A, 32)
    x = _getrs(dA, ipiv, b)
    bits = olu.correct_bits([_value(x[i]) for i in range(n)])
    # random matrices of this size have log2 cond below about 12
    assert bits > 53 * nc - 24, bits


def test_lotkin_dd_n128_nb32():
    # the small Lotkin workload: DD, n = 128, nb = 32 (log2 cond ~ 650 > 106)
    n, nc = 128, 2
    A = lotkin_expansions(n, nc)
    b = lotkin_rhs(n, nc)
    dA, LU, ipiv, info = _getrf(A, 32)
    assert info == 0
    bits = _backward_error_bits(A, LU, ipiv)
    assert bits < -106 + 16, bits
    x = _getrs(dA, ipiv, b)
    # residual of the solve, relative to |A| |x| (exact)
    Af = [[_value(A[i, j]) for j in range(n)] for i in range(n)]
    xf = [_value(x[i]) for i in range(n)]
    bf = [_value(b[i]) for i in range(n)]
    r = max(abs(sum(Af[i][j] * xf[j] for j in range(n)) - bf[i]) for i in range(n))
    scale = max(sum(abs(Af[i][j] * xf[j]) for j in range(n)) for i in range(n))
    assert r / scale < Fraction(2) ** -80


@pytest.mark.parametrize("nc,n,nb", [(2, 40, 16), (3, 40, 32), (4, 40, 256)])
def test_duplicate_rows_exact_cancellation(nc, n, nb):
    # rows 3 and 7 are equal and hold the column-0 maximum 1.0 (reciprocal
    # exactly 1): the first pivot is row 3, row 7 gets multiplier exactly 1
    # and becomes exactly zero (a - 1 a = 0 in the fused multiply-subtract of
    # the panel and in the Ozaki-II update), so every later pivot is nonzero
    # except the last, an exact zero
    A = random_expansions(n, n, nc, 9, -1, 1)
    A[:, 0, :] *= 0.5
    A[3, 0, :] = 0.0
    A[3, 0, 0] = 1.0
    A[7, :, :] = A[3, :, :]
    dA, LU, ipiv, info = _getrf(A, nb)
    assert info == n
    assert np.all(LU[n - 1, n - 1] == 0.0)
    assert np.all(np.isfinite(LU))
    bits = _backward_error_bits(A, LU, ipiv)
    assert bits < -53 * nc + 20, bits


@pytest.mark.parametrize("nc,n,nb", [(4, 96, 32), (3, 80, 16)])
def test_schur_update_replay(nc, n, nb):
    # per-step replay: from the GPU's factors, the first step's Schur update
    # S = (P A)22 - L21 U12 (rows in the final pivot order, which commutes with
    # the row-wise update) is recomputed by the GPU GEMM and by the oracle's
    # Ozaki-II replay, bit for bit; the GPU's trailing factors L22 U22 then
    # reproduce S to the backward-error bound of an LU
    from oracle import oz2
    from gpu_util import gpu_gemm
    A = random_expansions(n, n, nc, 700 + n, -2, 2)
    dA, LU, ipiv, info = _getrf(A, nb)
    assert info == 0
    PA = A.copy()
    for k in range(n):
        p = ipiv[k] - 1
        PA[[k, p]] = PA[[p, k]]
    L21 = np.ascontiguousarray(LU[nb:, :nb])
    U12 = np.ascontiguousarray(LU[:nb, nb:])
    C = np.ascontiguousarray(PA[nb:, nb:])
    ref = oz2.oz2_gemm(L21, U12, 53 * nc, alpha=-1, beta=1, C=C)
    got = gpu_gemm(L21, U12, alpha=-1, beta=1, C=C)
    assert np.array_equal(got, ref)
    m = n - nb
    bits = _backward_error_bits(ref, np.ascontiguousarray(LU[nb:, nb:]), [k + 1 for k in range(m)])
    assert bits < -53 * nc + math.log2(m) + 12, bits


def test_singular_info():
    A = random_expansions(20, 20, 2, 3, -1, 1)
    A[:, 5, :] = 0.0
    _, _, _, info = _getrf(A, 8)
    assert info == 6


def test_getrf_host_pointers():
    h = handle()
    n, nc = 50, 3
    A = random_expansions(n, n, nc, 31, -1, 1)
    Ac = ozlu.to_colmajor(A)
    ipiv = np.zeros(n, np.int32)
    info = np.zeros(1, np.int32)
    ozlu.ozlu_getrf(h, nc, 0, n, Ac, n, ipiv, 32, info)
    _, LU, ipiv_d, info_d = _getrf(A, 32)
    np.testing.assert_array_equal(ozlu.from_colmajor(Ac, n), LU)
    np.testing.assert_array_equal(ipiv, ipiv_d)
    assert info[0] == info_d == 0


@pytest.mark.parametrize("nc,n,nb", [(4, 90, 32), (2, 70, 16)])
def test_native_blocked_lu(nc, n, nb):
    # the blocked-naive comparison: same panels, trailing update in expansion arithmetic
    h = handle()
    A = random_expansions(n, n, nc, 700 + n, -2, 2)
    dA = dev(A)
    ipiv = torch.zeros(n, dtype=torch.int32, device="cuda")
    info = torch.zeros(1, dtype=torch.int32, device="cuda")
    ozlu.ozlu_getrf(h, nc, 0, n, dA, n, ipiv, nb, info, ozlu.make_opts("int8", native=1))
    torch.cuda.synchronize()
    LU = host(dA, n)
    assert int(info.item()) == 0
    bits = _backward_error_bits(A, LU, ipiv.cpu().numpy())
    assert bits < -53 * nc + math.log2(n) + 12, bits
    _, LU2, ipiv2, _ = _getrf(A, nb)
    np.testing.assert_array_equal(ipiv.cpu().numpy(), ipiv2)


@pytest.mark.parametrize("nc,n", [(4, 70), (2, 45)])
def test_native_unblocked_lu(nc, n):
    # the unblocked naive comparison (b = 1, Sec. 3.4): same pivots as the
    # oracle's p + 64-bit LU, exact backward error within the bound
    h = handle()
    A = random_expansions(n, n, nc, 1300 + n, -2, 2)
    dA = dev(A)
    ipiv = torch.zeros(n, dtype=torch.int32, device="cuda")
    info = torch.zeros(1, dtype=torch.int32, device="cuda")
    ozlu.ozlu_getrf(h, nc, 0, n, dA, n, ipiv, 64, info, ozlu.make_opts("int8", native=2))
    torch.cuda.synchronize()
    LU = host(dA, n)
    assert int(info.item()) == 0
    piv = ipiv.cpu().numpy()
    bits = _backward_error_bits(A, LU, piv)
    assert bits < -53 * nc + math.log2(n) + 12, bits
    prec = 53 * nc + 64
    Af = [[_value(A[i, j]) for j in range(n)] for i in range(n)]
    _, ipiv_ref, _ = olu.lu_bigfloat(olu.to_bigfloat_matrix(Af, prec), prec)
    assert [p + 1 for p in ipiv_ref] == list(piv)
