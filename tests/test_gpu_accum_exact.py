"""Worst-case exactness of the fp32 tensor-core accumulation (FP8 and FP16 back-ends).

The FP8 (balanced base-17 digits, Eq. (15), three Karatsuba planes) and FP16
(Eq. (14)) residue GEMMs rely on the fp32 accumulator of tcgen05.mma being
exact for integer sums below 2^24; the plan admits K_pad S 15^2 < 2^24 (FP8)
and K_pad S 127^2 < 2^24 (FP16).  Random residues leave the sums far below
that bound, so these tests use constant matrices: every term of an
accumulation then has the same sign and magnitude, and the sums reach the
largest values the plan admits (above 2^23) at the largest inner dimension it
admits.  An output depends only on its row of A and column of B, so the
oracle replays one 1 x K by K x 1 product and every output and t value of the
GPU must equal it bit for bit.
"""
import numpy as np
import pytest

from oracle import oz2
from oracle.plan import make_plan

from gpu_util import gpu_gemm, handle, ozlu, torch  # noqa: F401

pytestmark = pytest.mark.gpu


def _const(rows, cols, nc, x):
    M = np.zeros((rows, cols, nc))
    M[..., :len(x)] = x
    return M


def _plane_sums(plan, ra, rb, K, fp8):
    """Largest |accumulated plane sum| over moduli and digit groups for constant
    rows/columns with residues ra[(l, t)], rb[(l, t)] (one value each)."""
    worst = 0
    for l in range(plan.N):
        for g in plan.groups:
            acc = [0, 0, 0]
            for ta in range(plan.S):
                tb = g - ta
                if not 0 <= tb < plan.S:
                    continue
                a, b = int(ra[(l, ta)]), int(rb[(l, tb)])
                if fp8:
                    a0, a1 = oz2.fp8_base17_digits(a)
                    b0, b1 = oz2.fp8_base17_digits(b)
                    prods = (a0 * b0, a1 * b1, (a0 + a1) * (b0 + b1))
                else:
                    prods = (a * b, 0, 0)
                for q in range(3):
                    acc[q] += K * prods[q]
            worst = max(worst, *map(abs, acc))
    return worst


def _pick(nc, p, K, be, seed, tries):
    """Constant values a, b whose accumulations come closest to 2^24."""
    plan = make_plan(p, K, backend=be)
    rng = np.random.default_rng(seed)
    best = None
    for _ in range(tries):
        a = [rng.uniform(0.5, 1.0)] + [rng.uniform(-1, 1) * 2.0 ** (-55 * (c + 1)) for c in range(nc - 1)]
        b = [rng.uniform(0.5, 1.0)] + [rng.uniform(-1, 1) * 2.0 ** (-55 * (c + 1)) for c in range(nc - 1)]
        A1 = _const(1, 1, nc, a)
        B1 = _const(1, 1, nc, b)
        _, d = oz2.oz2_gemm(A1, B1, p, plan=plan, debug=True)
        ra = {k: v[0, 0] for k, v in d.res_A.items()}
        rb = {k: v[0, 0] for k, v in d.res_B.items()}
        s = _plane_sums(plan, ra, rb, K, be == "fp8")
        if best is None or s > best[0]:
            best = (s, a, b)
    return plan, best


@pytest.mark.parametrize("be,nc,p,K", [("fp16", 2, 106, 1024), ("fp8", 4, 212, 37248)])
def test_worst_case_accumulation_exact(be, nc, p, K):
    plan, (worst, a, b) = _pick(nc, p, K, be, 11 + K, 400 if be == "fp16" else 1500)
    kpad = -(-K // 128) * 128
    bound = kpad * plan.S * (15 * 15 if be == "fp8" else 127 * 127)
    assert bound < 2 ** 24                           # the largest K the plan admits ...
    assert (kpad + 128) * plan.S * (15 * 15 if be == "fp8" else 127 * 127) >= 2 ** 24
    assert worst > 2 ** 23                           # ... and sums above 2^23
    m = n = 130
    A = _const(m, K, nc, a)
    B = _const(K, n, nc, b)
    out = gpu_gemm(A, B, opts=ozlu.make_opts(be))
    h = handle()
    assert ozlu.ozlu_debug_fetch(h, 6, np.zeros(1, np.int32))[0] == 0
    ref_out, ref = oz2.oz2_gemm(A[:1], B[:, :1], p, backend=be, debug=True)
    t = ozlu.ozlu_debug_fetch(h, 5, np.zeros((len(plan.groups), plan.N, n, m), np.uint8))
    for l in range(plan.N):
        for gi, g in enumerate(plan.groups):
            assert np.all(t[gi, l] == ref.t[(l, g)][0, 0]), (l, g)
    assert np.all(out == ref_out[0, 0])
