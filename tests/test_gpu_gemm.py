"""Parity of the CUDA Ozaki-II GEMM (through the C ABI) with the CPU oracle.

The output of (S6) is a deterministic function of the inputs, so everything
is compared bit for bit: shared exponents, residue planes, t values of the
modular epilogue and the rounded expansion components.  Sizes span several
128 x 128 tiles with ragged edges; the full workload size is checked on
sampled rows and columns (each output depends only on its row of A and its
column of B).
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


def _compare_debug(dbg, ref, m, n, k):
    pl = ref.plan
    assert list(dbg["mu"]) == ref.mu and list(dbg["nu"]) == ref.nu
    for l in range(pl.N):
        for t in range(pl.S):
            np.testing.assert_array_equal(dbg["ra"][l, t], ref.res_A[(l, t)])
            np.testing.assert_array_equal(dbg["rb"][l, t], ref.res_B[(l, t)].T)
        for gi, g in enumerate(pl.groups):
            np.testing.assert_array_equal(dbg["t"][gi, l].T, ref.t[(l, g)])


@pytest.mark.parametrize("nc,m,n,k", [(2, 37, 29, 19), (3, 64, 64, 64), (4, 130, 140, 150),
                                      (4, 1, 1, 1), (2, 129, 3, 300)])
def test_gemm_bit_exact(nc, m, n, k):
    A, B = _pair(m, k, n, nc, 100 + m + nc)
    out, dbg = gpu_gemm(A, B, debug=True)
    ref_out, ref = oz2.oz2_gemm(A, B, 53 * nc, debug=True)
    _compare_debug(dbg, ref, m, n, k)
    np.testing.assert_array_equal(out, ref_out)


@pytest.mark.parametrize("nc,S,extra,gex", [(4, 3, 0, 0), (4, 0, 1, 0), (3, 0, 0, 40),
                                            (2, 2, 1, 0)])
def test_gemm_plan_options(nc, S, extra, gex):
    A, B = _pair(50, 70, 45, nc, 7 * nc + S)
    opts = ozlu.make_opts("int8", S, extra, gex)
    out = gpu_gemm(A, B, opts=opts)
    ref = oz2.oz2_gemm(A, B, 53 * nc, S=S or None, extra_groups=extra, g_ex=gex)
    np.testing.assert_array_equal(out, ref)


@pytest.mark.parametrize("nc", [2, 4])
def test_gemm_fused_schur_update(nc):
    # C <- C - A B, the (P4) form of Eq. (13)
    A, B = _pair(70, 40, 90, nc, 300 + nc, -2, 2)
    C = random_expansions(70, 90, nc, 999, -1, 3)
    out = gpu_gemm(A, B, alpha=-1, beta=1, C=C)
    ref = oz2.oz2_gemm(A, B, 53 * nc, alpha=-1, beta=1, C=C)
    np.testing.assert_array_equal(out, ref)


def test_gemm_huge_c_window():
    # old C far above the product: the window raises the grid (S6 reading)
    A, B = _pair(5, 8, 6, 4, 11, -3, 0)
    C = random_expansions(5, 6, 4, 12, 200, 220)
    out = gpu_gemm(A, B, alpha=1, beta=1, C=C)
    ref = oz2.oz2_gemm(A, B, 212, alpha=1, beta=1, C=C)
    np.testing.assert_array_equal(out, ref)


def test_gemm_zero_rows_cols_and_reduced_p():
    A, B = _pair(33, 17, 21, 3, 55)
    A[4] = 0.0
    B[:, 7] = 0.0
    out = gpu_gemm(A, B, p=120)
    ref = oz2.oz2_gemm(A, B, 120)
    np.testing.assert_array_equal(out, ref)
    assert np.all(out[4] == 0) and np.all(out[:, 7] == 0)


def test_gemm_host_pointers_match_device():
    h = handle()
    A, B = _pair(40, 30, 20, 4, 77)
    Ac, Bc = ozlu.to_colmajor(A), ozlu.to_colmajor(B)
    Cc = np.zeros((20, 40, 4))
    ozlu.ozlu_gemm(h, 4, 0, 40, 20, 30, 1, Ac, 40, Bc, 30, 0, Cc, 40, ozlu.make_opts("int8"))
    np.testing.assert_array_equal(ozlu.from_colmajor(Cc, 40), gpu_gemm(A, B))


def test_gemm_empty_and_k0():
    h = handle()
    C = torch.ones((3, 5, 2), dtype=torch.float64, device="cuda")
    A = torch.zeros((1, 5, 2), dtype=torch.float64, device="cuda")
    ozlu.ozlu_gemm(h, 2, 0, 5, 3, 0, 1, A, 5, A, 1, 0, C, 5)   # k = 0, beta = 0: C = 0
    torch.cuda.synchronize()
    assert float(C.abs().sum()) == 0.0
    ozlu.ozlu_gemm(h, 2, 0, 0, 3, 4, 1, A, 1, A, 4, 1, C, 1)   # m = 0: nothing


@pytest.mark.parametrize("n", [1024, 4096])
def test_gemm_full_size_sampled(n):
    # the standalone QD GEMM workload (m = n = k, exponents in [-30, 30]);
    # the oracle recomputes sampled rows x columns from A[rows], B[:, cols]
    A, B = _pair(n, n, n, 4, 2024 + n)
    out = gpu_gemm(A, B)
    rng = np.random.default_rng(n)
    rows = np.sort(rng.choice(n, 6, replace=False))
    cols = np.sort(rng.choice(n, 5, replace=False))
    ref = oz2.oz2_gemm(A[rows], B[:, cols], 212)
    np.testing.assert_array_equal(out[np.ix_(rows, cols)], ref)
