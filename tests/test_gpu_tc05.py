"""Parity of the tensor-core (tcgen05) residue GEMM back-ends with the oracle.

FP8 (balanced base-17 digits, Eq. (15), 3-plane Karatsuba) and FP16 (Eq. (14))
residue products are exact only if the fp32 tensor-core accumulation is
exact for integer sums below 2^24.  The t values of the modular epilogue and
the rounded outputs must therefore equal the oracle's bit for bit.
"""
import numpy as np
import pytest

from oracle import oz2
from synth import random_expansions

from gpu_util import gpu_gemm, handle, ozlu, torch  # noqa: F401

pytestmark = pytest.mark.gpu


def _pair(m, k, n, nc, seed, emin=-30, emax=30):
    return (random_expansions(m, k, nc, seed, emin, emax),
            random_expansions(k, n, nc, seed + 1, emin, emax))


def _t_values(h, G, N, m, n):
    return ozlu.ozlu_debug_fetch(h, 5, np.zeros((G, N, n, m), np.uint8))


@pytest.mark.parametrize("be", ["fp8", "fp16"])
@pytest.mark.parametrize("nc,m,n,k", [(4, 130, 140, 150), (2, 64, 64, 256), (4, 1, 1, 1),
                                      (3, 200, 33, 500), (4, 257, 129, 64)])
def test_tc05_bit_exact(be, nc, m, n, k):
    A, B = _pair(m, k, n, nc, 7000 + m + k + nc)
    opts = ozlu.make_opts(be)
    out = gpu_gemm(A, B, opts=opts)
    h = handle()
    err = ozlu.ozlu_debug_fetch(h, 6, np.zeros(1, np.int32))
    assert err[0] == 0
    ref_out, ref = oz2.oz2_gemm(A, B, 53 * nc, backend=be, debug=True)
    pl = ref.plan
    t = _t_values(h, len(pl.groups), pl.N, m, n)
    for l in range(pl.N):
        for gi, g in enumerate(pl.groups):
            np.testing.assert_array_equal(t[gi, l].T, ref.t[(l, g)])
    np.testing.assert_array_equal(out, ref_out)


@pytest.mark.parametrize("be", ["fp8", "fp16"])
def test_tc05_fused_update(be):
    A, B = _pair(90, 256, 70, 4, 4242, -2, 2)
    C = random_expansions(90, 70, 4, 4243, -1, 3)
    out = gpu_gemm(A, B, alpha=-1, beta=1, C=C, opts=ozlu.make_opts(be))
    ref = oz2.oz2_gemm(A, B, 212, alpha=-1, beta=1, C=C, backend=be)
    np.testing.assert_array_equal(out, ref)


@pytest.mark.parametrize("be,n", [("fp8", 2048), ("fp8", 4096)])
def test_tc05_full_size_sampled(be, n):
    A, B = _pair(n, n, n, 4, 9090 + n)
    out = gpu_gemm(A, B, opts=ozlu.make_opts(be))
    rng = np.random.default_rng(n + 1)
    rows = np.sort(rng.choice(n, 4, replace=False))
    cols = np.sort(rng.choice(n, 4, replace=False))
    ref = oz2.oz2_gemm(A[rows], B[:, cols], 212, backend=be)
    np.testing.assert_array_equal(out[np.ix_(rows, cols)], ref)


@pytest.mark.parametrize("be", ["fp16", "int8"])
def test_lu_update_shape_full_size_sampled(be):
    # the trailing update of the benchmark's first LU step: m = n = 3840,
    # K = nb = 256, C <- C - A B (Eq. (13)); sampled outputs against the oracle
    m, k = 3840, 256
    A, B = _pair(m, k, m, 4, 3840, -3, 3)
    C = random_expansions(m, m, 4, 3841, -2, 4)
    out = gpu_gemm(A, B, alpha=-1, beta=1, C=C, opts=ozlu.make_opts(be))
    h = handle()
    assert ozlu.ozlu_debug_fetch(h, 6, np.zeros(1, np.int32))[0] == 0
    rng = np.random.default_rng(7)
    rows = np.sort(np.concatenate([rng.choice(m, 5, replace=False), [0, m - 1]]))
    cols = np.sort(np.concatenate([rng.choice(m, 5, replace=False), [0, m - 1]]))
    ref = oz2.oz2_gemm(A[rows], B[:, cols], 212, alpha=-1, beta=1, C=C[np.ix_(rows, cols)],
                       backend=be)
    np.testing.assert_array_equal(out[np.ix_(rows, cols)], ref)
