"""The allocation-free GEMM entry point (ozlu_gemm_noalloc) against ozlu_gemm.

Callers that must not allocate device memory (a host whose pool allocator
already owns the device, a latency-critical caller) use ozlu_gemm_noalloc: it
works in a fixed device array inside the library.  Its results must equal
ozlu_gemm's INT8 path bit for bit (the tolerance of every GEMM parity test
here), on consecutive calls that reuse the array, and problems too large for
the array must be rejected.  This file is collected last on purpose.
"""
import numpy as np
import pytest

from synth import random_expansions

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def oz():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2609_29554_gb300 import build, ozlu
    build.build()
    return ozlu


def _dev(x, oz):
    return torch.from_numpy(oz.to_colmajor(x)).cuda()


def _reference(oz, h, A, B, C, alpha, beta):
    m, k, nc = A.shape
    n = B.shape[1]
    dC = _dev(C, oz)
    oz.ozlu_gemm(h, nc, 0, m, n, k, alpha, _dev(A, oz), m, _dev(B, oz), k, beta, dC, m,
                 oz.make_opts("int8"))
    torch.cuda.synchronize()
    return oz.from_colmajor(dC.cpu().numpy(), m)


def _noalloc(oz, A, B, C, alpha, beta):
    m, k, nc = A.shape
    n = B.shape[1]
    dC = _dev(C, oz)
    oz.ozlu_gemm_noalloc(nc, 0, m, n, k, alpha, _dev(A, oz), m, _dev(B, oz), k, beta, dC, m)
    torch.cuda.synchronize()
    return oz.from_colmajor(dC.cpu().numpy(), m)


def test_noalloc_matches_gemm_on_consecutive_calls(oz):
    # consecutive calls share the library's array: each case runs twice in a
    # row, the cases differ in size and data, and the first case is repeated
    # at the end, after the array has held other problems' intermediates
    h = oz.ozlu_create(None)
    try:
        cases = [((100, 120, 90, 4), -1, 1, 11), ((256, 256, 256, 4), 1, 0, 12),
                 ((37, 19, 29, 2), 1, 1, 13), ((64, 300, 50, 3), -1, 1, 14),
                 ((100, 120, 90, 4), -1, 1, 11)]
        for (m, k, n, nc), alpha, beta, seed in cases:
            A = random_expansions(m, k, nc, seed, -20, 20)
            B = random_expansions(k, n, nc, seed + 100, -20, 20)
            C = random_expansions(m, n, nc, seed + 200, -20, 20)
            ref = _reference(oz, h, A, B, C, alpha, beta)
            first = _noalloc(oz, A, B, C, alpha, beta)
            second = _noalloc(oz, A, B, C, alpha, beta)
            np.testing.assert_array_equal(first, ref)
            np.testing.assert_array_equal(second, ref)
    finally:
        oz.ozlu_destroy(h)


def test_noalloc_rejects_oversize_and_host_pointers(oz):
    m = n = k = 384
    A = torch.zeros((k, m, 4), dtype=torch.float64, device="cuda")
    B = torch.zeros((n, k, 4), dtype=torch.float64, device="cuda")
    C = torch.zeros((n, m, 4), dtype=torch.float64, device="cuda")
    with pytest.raises(oz.OzluError) as e:
        oz.ozlu_gemm_noalloc(4, 0, m, n, k, 1, A, m, B, k, 0, C, m)
    assert e.value.code == oz.OZLU_ERR_CAPACITY
    Ah = np.zeros((4, 4, 2))
    with pytest.raises(oz.OzluError) as e:
        oz.ozlu_gemm_noalloc(2, 0, 4, 4, 4, 1, Ah, 4, B, 4, 0, C, 4)
    assert e.value.code == -7
