"""Binary64 residue back-end (Eq. (17)) and the measured back-end autotuner.

The binary64 back-end uses its own plan (primes of about 23 bits), so its
output is compared with the oracle run on the same plan, bit for bit.  The
autotuned call must return exactly the result of the back-end it chose.
"""
import numpy as np
import pytest

from oracle import oz2
from synth import random_expansions

from gpu_util import gpu_gemm, handle, ozlu, torch  # noqa: F401

pytestmark = pytest.mark.gpu
NAMES = {1: "int8", 2: "fp8", 3: "fp64", 4: "fp16"}


def _pair(m, k, n, nc, seed, emin=-20, emax=20):
    return (random_expansions(m, k, nc, seed, emin, emax),
            random_expansions(k, n, nc, seed + 1, emin, emax))


@pytest.mark.parametrize("nc,m,n,k", [(2, 60, 50, 70), (4, 130, 129, 64), (3, 33, 200, 257)])
def test_fp64_backend_bit_exact(nc, m, n, k):
    A, B = _pair(m, k, n, nc, 3100 + m + nc)
    out = gpu_gemm(A, B, opts=ozlu.make_opts("fp64"))
    h = handle()
    ref_out, ref = oz2.oz2_gemm(A, B, 53 * nc, backend="fp64", debug=True)
    pl = ref.plan
    t = ozlu.ozlu_debug_fetch(h, 5, np.zeros((len(pl.groups), pl.N, n, m), np.uint32))
    for l in range(pl.N):
        for gi, g in enumerate(pl.groups):
            np.testing.assert_array_equal(t[gi, l].T, ref.t[(l, g)])
    np.testing.assert_array_equal(out, ref_out)


@pytest.mark.parametrize("nc,m,n,k", [(4, 256, 256, 256), (2, 100, 90, 40), (3, 64, 8, 300)])
def test_autotuned_equals_chosen_backend(nc, m, n, k):
    # the autotuner picks a (back-end, S) pair, S seeded by Eq. (Lhint); the
    # result must be the oracle's for exactly that pair
    A, B = _pair(m, k, n, nc, 3300 + m)
    out = gpu_gemm(A, B, opts=ozlu.make_opts("auto"))
    st = ozlu.ozlu_get_stats(handle())
    chosen = NAMES[st.last_backend]
    S = st.last_nslice
    assert S >= oz2.make_plan(53 * nc, k, backend=chosen).S
    ref = oz2.oz2_gemm(A, B, 53 * nc, backend=chosen, S=S)
    np.testing.assert_array_equal(out, ref)
    # second call hits the cache and returns the same bits
    np.testing.assert_array_equal(gpu_gemm(A, B, opts=ozlu.make_opts("auto")), out)


def test_panel_width_autotuned():
    # nb = 0: the panel width is measured on the first call for the size class
    # and cached; the factorisation equals the one with that width given
    from synth import random_expansions as rx
    from gpu_util import dev, host
    h = handle()
    n, nc = 300, 3
    M = rx(n, n, nc, 77, -1, 1)
    outs = []
    for nb in (0, None):
        dM = dev(M)
        ipiv = torch.zeros(n, dtype=torch.int32, device="cuda")
        info = torch.zeros(1, dtype=torch.int32, device="cuda")
        use = 0 if nb == 0 else ozlu.ozlu_get_stats(h).tuned_nb
        ozlu.ozlu_getrf(h, nc, 0, n, dM, n, ipiv, use, info)
        torch.cuda.synchronize()
        assert int(info.item()) == 0
        outs.append((host(dM, n), ipiv.cpu().numpy()))
        if nb == 0:
            assert ozlu.ozlu_get_stats(h).tuned_nb in (64, 128, 256)
    np.testing.assert_array_equal(outs[0][1], outs[1][1])
    np.testing.assert_array_equal(outs[0][0], outs[1][0])
