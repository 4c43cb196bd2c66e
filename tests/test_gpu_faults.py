"""Failure handling without a GPU fault.

  * The bounded device waits (the panel kernel's stamp wait, the tensor-core
    GEMM's mbarrier wait) are made to run out on a flag or barrier that
    nothing sets, with a short limit: each must give up, leave
    OZLU_ERR_TIMEOUT in its error word, and the LU's finish step must turn it
    into info = -OZLU_ERR_TIMEOUT (what a replayed CUDA graph reports).  The
    context stays usable: the next calls on the same handle are correct.
  * A device allocation failure is injected on the host: the call that needed
    the memory returns OZLU_ERR_NOMEM, and the handle works afterwards.
Nothing here traps, faults or hangs the GPU.
"""
import numpy as np
import pytest

from oracle import oz2
from synth import random_expansions

from gpu_util import dev, gpu_gemm, handle, host, ozlu, torch

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("which,limit", [(1, 2_000_000), (2, 5_000)])
def test_bounded_wait_expires_and_reports(which, limit):
    h = handle()
    rc, (gave_up, err, info) = ozlu.ozlu_debug_wait_expiry(h, which, limit)
    assert rc == ozlu.OZLU_ERR_TIMEOUT
    assert gave_up == 1 and err == ozlu.OZLU_ERR_TIMEOUT and info == -ozlu.OZLU_ERR_TIMEOUT
    if which == 2:
        assert ozlu.ozlu_debug_fetch(h, 6, np.zeros(1, np.int32))[0] == ozlu.OZLU_ERR_TIMEOUT
    # the handle and the context stay usable; both error words are cleared
    A = random_expansions(40, 30, 4, 5, -3, 3)
    B = random_expansions(30, 20, 4, 6, -3, 3)
    out = gpu_gemm(A, B, opts=ozlu.make_opts("fp16"))
    assert ozlu.ozlu_debug_fetch(h, 6, np.zeros(1, np.int32))[0] == 0
    np.testing.assert_array_equal(out, oz2.oz2_gemm(A, B, 212, backend="fp16"))
    M = random_expansions(48, 48, 4, 7, -1, 1)
    dM = dev(M)
    ipiv = torch.zeros(48, dtype=torch.int32, device="cuda")
    inf = torch.ones(1, dtype=torch.int32, device="cuda")
    ozlu.ozlu_getrf(h, 4, 0, 48, dM, 48, ipiv, 16, inf)
    torch.cuda.synchronize()
    assert int(inf.item()) == 0


def test_injected_allocation_failure_gives_nomem():
    handle()   # builds the library and sets up the device
    A = random_expansions(33, 21, 3, 8, -2, 2)
    B = random_expansions(21, 17, 3, 9, -2, 2)
    h = ozlu.ozlu_create(None)
    try:
        ozlu.ozlu_debug_fail_alloc(1)
        C = torch.zeros((17, 33, 3), dtype=torch.float64, device="cuda")
        with pytest.raises(ozlu.OzluError) as e:
            ozlu.ozlu_gemm(h, 3, 0, 33, 17, 21, 1, dev(A), 33, dev(B), 21, 0, C, 33,
                           ozlu.make_opts("int8"))
        assert e.value.code == ozlu.OZLU_ERR_NOMEM
        # the workspace tries a padded size, then the exact size: fail both
        ozlu.ozlu_debug_fail_alloc(2)
        with pytest.raises(ozlu.OzluError) as e:
            ozlu.ozlu_gemm(h, 3, 0, 33, 17, 21, 1, dev(A), 33, dev(B), 21, 0, C, 33,
                           ozlu.make_opts("int8"))
        assert e.value.code == ozlu.OZLU_ERR_NOMEM
        ozlu.ozlu_debug_fail_alloc(0)
        ozlu.ozlu_gemm(h, 3, 0, 33, 17, 21, 1, dev(A), 33, dev(B), 21, 0, C, 33,
                       ozlu.make_opts("int8"))
        torch.cuda.synchronize()
        np.testing.assert_array_equal(host(C, 33), oz2.oz2_gemm(A, B, 159))
        # the LU's scratch
        h2 = ozlu.ozlu_create(None)
        try:
            ozlu.ozlu_debug_fail_alloc(1)
            ipiv = torch.zeros(8, dtype=torch.int32, device="cuda")
            info = torch.zeros(1, dtype=torch.int32, device="cuda")
            M = dev(random_expansions(8, 8, 2, 10, -1, 1))
            with pytest.raises(ozlu.OzluError) as e:
                ozlu.ozlu_getrf(h2, 2, 0, 8, M, 8, ipiv, 4, info)
            assert e.value.code == ozlu.OZLU_ERR_NOMEM
        finally:
            ozlu.ozlu_debug_fail_alloc(0)
            ozlu.ozlu_destroy(h2)
    finally:
        ozlu.ozlu_debug_fail_alloc(0)
        ozlu.ozlu_destroy(h)
