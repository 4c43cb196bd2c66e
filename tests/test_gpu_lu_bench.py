"""The benchmarked LU configuration under oracle parity.

The QD LU of the benchmark runs ozlu_getrf with the default (measured)
back-end choice and nb = 256: panels wider than the cooperative kernel's base
block (128 columns) are split by the recursive panel, whose inner updates are
Ozaki-II GEMMs, and the base blocks run on many co-resident thread blocks
that exchange pivot candidates through memory.  These tests drive exactly
that path (default options, nb = 256, n >= 512) and check it against:

  * the oracle's p + 64-bit LU (pivot sequence, on a matrix without near ties);
  * exact residuals P A - L U of the returned factors (host integers), on
    every row through a random probe and on sampled entries;
  * a per-step replay of the first two trailing updates (Eq. (13)) by the
    oracle's Ozaki-II GEMM, bit for bit, with the back-end the library chose;
  * the solve against x = ones on the benchmark's own matrix construction
    (A = U diag(sigma) V^T, cond 1e40) with many thread blocks per panel.
"""
import math
from fractions import Fraction

import numpy as np
import pytest

from exact_lu import ExactLU, l_bounded, permuted, valid_interchanges
from oracle import lu as olu
from oracle import oz2
from synth import exact_row_sums, prescribed_cond_expansions, random_expansions

from gpu_util import dev, gpu_gemm, handle, host, ozlu, torch

pytestmark = pytest.mark.gpu

BACKEND = {1: "int8", 2: "fp8", 3: "fp64", 4: "fp16"}


def _getrf(A, nb, opts=None):
    h = handle()
    n, _, nc = A.shape
    dA = dev(A)
    ipiv = torch.zeros(n, dtype=torch.int32, device="cuda")
    info = torch.zeros(1, dtype=torch.int32, device="cuda")
    ozlu.ozlu_getrf(h, nc, 0, n, dA, n, ipiv, nb, info, opts)
    torch.cuda.synchronize()
    return dA, host(dA, n), ipiv.cpu().numpy(), int(info.item())


def _value(limbs):
    return sum((Fraction(float(v)) for v in limbs), Fraction(0))


@pytest.mark.slow
def test_bench_path_pivots_equal_oracle_n512():
    # QD, nb = 256 (two 128-column base blocks per panel, recursion inside
    # the panel), default back-end choice: the interchanges must be those of
    # the oracle's LU in p + 64-bit arithmetic
    n, nc, nb = 512, 4, 256
    A = random_expansions(n, n, nc, 8080, -2, 2)
    dA, LU, ipiv, info = _getrf(A, nb)
    assert info == 0
    assert valid_interchanges(ipiv, n) and l_bounded(LU)
    ex = ExactLU(A, LU, ipiv)
    assert ex.probe_bits(1) < -53 * nc + math.log2(n) + 12
    rng = np.random.default_rng(3)
    pairs = [(int(i), int(j)) for i, j in rng.integers(0, n, size=(120, 2))] + [(n - 1, n - 1)]
    assert ex.sampled_bits(pairs) < -53 * nc + math.log2(n) + 12
    prec = 53 * nc + 64
    Af = [[_value(A[i, j]) for j in range(n)] for i in range(n)]
    _, piv_ref, _ = olu.lu_bigfloat(olu.to_bigfloat_matrix(Af, prec), prec)
    assert [p + 1 for p in piv_ref] == list(ipiv)


def test_bench_matrix_many_blocks_n2560():
    # the benchmark's construction (cond 1e40) at a size where each base
    # block spreads over every SM (n / 16 rows per block >= 152 blocks)
    n, nc, nb = 2560, 4, 256
    A = prescribed_cond_expansions(n, 40.0, 41, nc, device="cuda").cpu().numpy()
    dA, LU, ipiv, info = _getrf(A, nb)
    assert info == 0
    assert valid_interchanges(ipiv, n) and l_bounded(LU)
    ex = ExactLU(A, LU, ipiv)
    rng = np.random.default_rng(5)
    pairs = [(int(i), int(j)) for i, j in rng.integers(0, n, size=(60, 2))]
    pairs += [(n - 1, n - 1), (n - 1, 0), (0, n - 1), (1800, 2100), (2100, 1800)]
    assert ex.sampled_bits(pairs) < -53 * nc + math.log2(n) + 12
    # A x = A 1 with b formed exactly: p - log2 cond (212 - 133 = 79) bits at least
    At = torch.from_numpy(A).cuda()
    b = exact_row_sums(At, nc).view(1, n, nc).contiguous()
    h = handle()
    ozlu.ozlu_getrs(h, nc, 0, n, 1, dA, n, torch.from_numpy(ipiv).cuda(), b, n)
    torch.cuda.synchronize()
    x = b.cpu().numpy()[0]
    err = max(abs(_value(x[i]) - 1) for i in range(n))
    bits = math.log2(err.denominator) - math.log2(err.numerator) if err else 212.0
    assert bits > 212 - 40 * math.log2(10) - 8, bits


@pytest.mark.slow
@pytest.mark.parametrize("be", ["auto", "fp16", "int8"])
def test_schur_replay_first_two_steps(be):
    # per-step replay at r0 = 0 and r0 = 256: the trailing matrices
    #   T1 = (P A)22 - L21 U12                  (m = n = 320, K = 256)
    #   T2 = T1[256:, 256:] - L32 U23           (m = n = 64,  K = 256)
    # are recomputed by the oracle's Ozaki-II replay from the GPU's factors
    # (rows in the final pivot order, which commutes with the row-wise update)
    # and by the library's GEMM on the same handle (the same cached back-end
    # choice as inside the LU), bit for bit; the GPU's trailing factors then
    # reproduce T1 and T2 to the backward-error bound of an LU
    n, nc, nb = 576, 4, 256
    opts = ozlu.make_opts(be) if be != "auto" else None
    A = random_expansions(n, n, nc, 9191, -2, 2)
    _, LU, ipiv, info = _getrf(A, nb, opts)
    assert info == 0
    PA = permuted(A, ipiv)
    h = handle()
    T = np.ascontiguousarray(PA[nb:, nb:])
    for r0 in (0, nb):
        L21 = np.ascontiguousarray(LU[r0 + nb:, r0:r0 + nb])
        U12 = np.ascontiguousarray(LU[r0:r0 + nb, r0 + nb:])
        C = np.ascontiguousarray(T[r0:, r0:])
        got = gpu_gemm(L21, U12, alpha=-1, beta=1, C=C, opts=opts)
        used = BACKEND[ozlu.ozlu_get_stats(h).last_backend]
        if be != "auto":
            assert used == be
        ref = oz2.oz2_gemm(L21, U12, 53 * nc, alpha=-1, beta=1, C=C, backend=used)
        assert np.array_equal(got, ref), (r0, used)
        m = n - r0 - nb
        tail = np.ascontiguousarray(LU[r0 + nb:, r0 + nb:])
        bits = ExactLU(ref, tail, list(range(1, m + 1))).probe_bits(r0)
        assert bits < -53 * nc + math.log2(m) + 12, (r0, bits)
        if r0 == 0:
            T = ref          # the trailing matrix the second panel factors
