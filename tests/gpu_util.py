"""Helpers for the GPU tests: device setup and oracle comparisons."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2609_29554_gb300 import build, ozlu  # noqa: E402


def need_gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


_H = None


def handle():
    global _H
    need_gpu()
    if _H is None:
        build.build()
        torch.cuda.init()
        _H = ozlu.ozlu_create(None)
    return _H


def dev(x: np.ndarray):
    """(rows, cols, nc) numpy -> column-major device tensor (cols, rows, nc)."""
    return torch.from_numpy(ozlu.to_colmajor(x)).cuda()


def host(t, rows):
    return ozlu.from_colmajor(t.cpu().numpy(), rows)


def gpu_gemm(A, B, p=0, alpha=1, beta=0, C=None, opts=None, debug=False):
    """ozlu_gemm through the C ABI; the INT8 back-end unless opts says otherwise."""
    h = handle()
    if opts is None:
        opts = ozlu.make_opts("int8")
    m, k, nc = A.shape
    n = B.shape[1]
    dA, dB = dev(A), dev(B)
    dC = dev(C) if C is not None else torch.zeros((n, m, nc), dtype=torch.float64, device="cuda")
    ozlu.ozlu_gemm(h, nc, p, m, n, k, alpha, dA, max(1, m), dB, max(1, k), beta, dC, max(1, m),
                   opts)
    torch.cuda.synchronize()
    out = host(dC, m)
    if not debug:
        return out
    info = ozlu.ozlu_plan(p or 53 * nc, k, opts)
    N, S, G = info.n_mod, info.S, info.n_groups
    dbg = {
        "mu": ozlu.ozlu_debug_fetch(h, 1, np.zeros(m, np.int32)),
        "nu": ozlu.ozlu_debug_fetch(h, 2, np.zeros(n, np.int32)),
        "ra": ozlu.ozlu_debug_fetch(h, 3, np.zeros((N, S, m, k), np.int8)),
        "rb": ozlu.ozlu_debug_fetch(h, 4, np.zeros((N, S, n, k), np.int8)),
        "t": ozlu.ozlu_debug_fetch(h, 5, np.zeros((G, N, n, m), np.uint8)),
        "info": info,
    }
    return out, dbg
