"""Batched uneven LU (ozlu_getrf_batched / ozlu_getrs_batched) through the C ABI.

Every instance must come out exactly as the single-instance ozlu_getrf would
factor it (same back-end, so the same bits), eagerly, on the call that
captures the CUDA graph, and on graph replays; the batched solve must equal
the single solve.
"""
import numpy as np
import pytest

from synth import random_expansions

from gpu_util import dev, handle, host, ozlu, torch

pytestmark = pytest.mark.gpu

SIZES = [17, 64, 100, 33, 150, 1, 80, 129]


def _single(A, nc, nb, opts):
    h = handle()
    n = A.shape[0]
    dA = dev(A)
    ipiv = torch.zeros(n, dtype=torch.int32, device="cuda")
    info = torch.zeros(1, dtype=torch.int32, device="cuda")
    ozlu.ozlu_getrf(h, nc, 0, n, dA, n, ipiv, nb, info, opts)
    torch.cuda.synchronize()
    return dA, ipiv, host(dA, n), ipiv.cpu().numpy(), int(info.item())


@pytest.mark.parametrize("graph", [0, 1])
def test_batched_equals_single(graph):
    nc, nb = 3, 32
    opts = ozlu.make_opts("int8", graph=graph)
    mats = [random_expansions(n, n, nc, 40 + i, -1, 1) for i, n in enumerate(SIZES)]
    ref = [_single(A, nc, nb, ozlu.make_opts("int8")) for A in mats]
    h = ozlu.ozlu_create(None)
    try:
        d0 = [dev(A) for A in mats]
        dA = [x.clone() for x in d0]
        piv = [torch.zeros(max(n, 1), dtype=torch.int32, device="cuda") for n in SIZES]
        info = torch.full((len(SIZES),), -7, dtype=torch.int32, device="cuda")
        for rep in range(3 if graph else 1):     # eager, capture, replay
            for x, y in zip(dA, d0):
                x.copy_(y)
            ozlu.ozlu_getrf_batched(h, nc, 0, SIZES, dA, SIZES, piv, info, nb, opts)
            torch.cuda.synchronize()
            assert ozlu.ozlu_get_stats(h).graph_status == ([0, 1, 2][rep] if graph else 0)
            assert info.cpu().tolist() == [0] * len(SIZES)
            for i, n in enumerate(SIZES):
                np.testing.assert_array_equal(host(dA[i], n), ref[i][2])
                np.testing.assert_array_equal(piv[i].cpu().numpy()[:n], ref[i][3])
        # batched solve of A_i x = b_i against the single solve
        bs = [torch.from_numpy(np.ascontiguousarray(random_expansions(n, 1, nc, 90 + i)[None, :, 0, :]))
              .cuda() for i, n in enumerate(SIZES)]
        bs1 = [b.clone() for b in bs]
        ozlu.ozlu_getrs_batched(h, nc, 0, SIZES, 1, dA, SIZES, piv, bs, SIZES, opts)
        torch.cuda.synchronize()
        hs = handle()
        for i, n in enumerate(SIZES):
            ozlu.ozlu_getrs(hs, nc, 0, n, 1, dA[i], n, piv[i], bs1[i], n, ozlu.make_opts("int8"))
        torch.cuda.synchronize()
        for b, b1 in zip(bs, bs1):
            np.testing.assert_array_equal(b.cpu().numpy(), b1.cpu().numpy())
    finally:
        ozlu.ozlu_destroy(h)


def test_single_instance_graph_replay():
    """ozlu_getrf / ozlu_getrs with opts.graph: capture on the second call, replay
    after; the same bits as the eager calls, on the caller's (default) stream."""
    nc, n, nb = 4, 200, 64
    A0 = random_expansions(n, n, nc, 77, -1, 1)
    ref = _single(A0, nc, nb, ozlu.make_opts("int8"))
    b0 = np.ascontiguousarray(random_expansions(n, 1, nc, 78)[None, :, 0, :])
    hs = handle()
    xb = torch.from_numpy(b0).cuda()
    ozlu.ozlu_getrs(hs, nc, 0, n, 1, ref[0], n, ref[1], xb, n, ozlu.make_opts("int8"))
    torch.cuda.synchronize()
    h = ozlu.ozlu_create(None)
    try:
        opts = ozlu.make_opts("int8", graph=1)
        dA0 = dev(A0)
        dA = dA0.clone()
        piv = torch.zeros(n, dtype=torch.int32, device="cuda")
        info = torch.full((1,), -7, dtype=torch.int32, device="cuda")
        x = torch.empty_like(xb)
        for rep in range(4):
            dA.copy_(dA0)
            ozlu.ozlu_getrf(h, nc, 0, n, dA, n, piv, nb, info, opts)
            x.copy_(torch.from_numpy(b0))
            ozlu.ozlu_getrs(h, nc, 0, n, 1, dA, n, piv, x, n, opts)
            torch.cuda.synchronize()
            assert ozlu.ozlu_get_stats(h).graph_status == min(rep, 2)
            assert int(info.item()) == 0
            np.testing.assert_array_equal(host(dA, n), ref[2])
            np.testing.assert_array_equal(piv.cpu().numpy(), ref[3])
            np.testing.assert_array_equal(x.cpu().numpy(), xb.cpu().numpy())
    finally:
        ozlu.ozlu_destroy(h)


def test_batched_against_oracle():
    # the batched LU (default back-end choice, library panel widths, CUDA
    # graph replay) against the oracle: every instance's pivots equal those of
    # the oracle's p + 64-bit LU and its exact backward error P A - L U is
    # within the bound; each solution of A x = A 1 (b formed exactly) reaches
    # the accuracy the condition allows
    import math
    from fractions import Fraction

    from exact_lu import ExactLU, l_bounded
    from oracle import lu as olu
    from synth import exact_row_sums, prescribed_cond_expansions

    nc = 3
    sizes = [40, 72, 17, 96]
    conds = [20.0, 30.0, 25.0, 35.0]
    mats = [prescribed_cond_expansions(n, c, 500 + i, nc).numpy() for i, (n, c) in enumerate(zip(sizes, conds))]
    h = ozlu.ozlu_create(None)
    try:
        opts = ozlu.make_opts("auto", graph=1)
        d0 = [dev(A) for A in mats]
        dA = [x.clone() for x in d0]
        piv = [torch.zeros(n, dtype=torch.int32, device="cuda") for n in sizes]
        info = torch.full((len(sizes),), -7, dtype=torch.int32, device="cuda")
        for _ in range(3):                        # eager, capture, replay
            for x, y in zip(dA, d0):
                x.copy_(y)
            ozlu.ozlu_getrf_batched(h, nc, 0, sizes, dA, sizes, piv, info, 0, opts)
        rhs = [exact_row_sums(torch.from_numpy(A), nc).view(1, n, nc).contiguous().cuda()
               for A, n in zip(mats, sizes)]
        ozlu.ozlu_getrs_batched(h, nc, 0, sizes, 1, dA, sizes, piv, rhs, sizes, ozlu.make_opts("auto"))
        torch.cuda.synchronize()
        assert ozlu.ozlu_get_stats(h).graph_status == 2
        assert info.cpu().tolist() == [0] * len(sizes)
        prec = 53 * nc + 64
        for i, (A, n, c) in enumerate(zip(mats, sizes, conds)):
            LU = host(dA[i], n)
            ip = piv[i].cpu().numpy()
            assert l_bounded(LU)
            assert ExactLU(A, LU, ip).probe_bits(i) < -53 * nc + math.log2(n) + 12
            Af = [[sum((Fraction(float(v)) for v in A[r, j]), Fraction(0)) for j in range(n)] for r in range(n)]
            _, piv_ref, _ = olu.lu_bigfloat(olu.to_bigfloat_matrix(Af, prec), prec)
            assert [p + 1 for p in piv_ref] == list(ip), i
            x = rhs[i].cpu().numpy()[0]
            err = max(abs(sum((Fraction(float(v)) for v in x[r]), Fraction(0)) - 1) for r in range(n))
            bits = math.log2(err.denominator) - math.log2(err.numerator) if err else 159.0
            assert bits > 159 - c * math.log2(10) - 10, (i, bits)
    finally:
        ozlu.ozlu_destroy(h)
