"""Command-line runs of single library calls on seeded inputs.

    python -m paper_2609_29554_gb300.cli gemm  --n 2048 --nc 4 --backend fp8 [--schur]
    python -m paper_2609_29554_gb300.cli getrf --n 4096 --nc 4 --nb 256 [--matrix cond|random]

Each run builds the library if needed, generates its input with synth/,
makes one warm-up and one timed call through the C ABI and prints the time;
it is the command the profiles under profiles/ were captured with.
"""
from __future__ import annotations

import argparse
import os
import sys
import time

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("op", choices=["gemm", "getrf"])
    ap.add_argument("--n", type=int, default=2048)
    ap.add_argument("--k", type=int, default=0)
    ap.add_argument("--nc", type=int, default=4)
    ap.add_argument("--nb", type=int, default=256)
    ap.add_argument("--backend", default="auto")
    ap.add_argument("--matrix", default="random", choices=["random", "cond"])
    ap.add_argument("--reps", type=int, default=1)
    ap.add_argument("--schur", action="store_true",
                    help="gemm as the LU's trailing update: C <- C - A B on a random C")
    a = ap.parse_args(argv)
    import torch

    from paper_2609_29554_gb300 import build, ozlu
    from synth import prescribed_cond_expansions, random_expansions
    build.build()
    h = ozlu.ozlu_create(None)
    opts = ozlu.make_opts(a.backend)
    n, nc = a.n, a.nc
    if a.op == "gemm":
        k = a.k or n
        A = torch.from_numpy(ozlu.to_colmajor(random_expansions(n, k, nc, 1))).cuda()
        B = torch.from_numpy(ozlu.to_colmajor(random_expansions(k, n, nc, 2))).cuda()
        if a.schur:
            C0 = torch.from_numpy(ozlu.to_colmajor(random_expansions(n, n, nc, 3, -1, 1))).cuda()
        else:
            C0 = torch.zeros((n, n, nc), dtype=torch.float64, device="cuda")
        C = torch.empty_like(C0)
        alpha, beta = (-1, 1) if a.schur else (1, 0)

        def call():
            C.copy_(C0)
            ozlu.ozlu_gemm(h, nc, 0, n, n, k, alpha, A, n, B, k, beta, C, n, opts)
        flops = 2.0 * n * n * k
    else:
        if a.matrix == "cond":
            A0 = prescribed_cond_expansions(n, 40.0, 4, nc, device="cuda").permute(1, 0, 2).contiguous()
        else:
            A0 = torch.from_numpy(ozlu.to_colmajor(random_expansions(n, n, nc, 1, -1, 1))).cuda()
        A = torch.empty_like(A0)
        ipiv = torch.zeros(n, dtype=torch.int32, device="cuda")
        info = torch.zeros(1, dtype=torch.int32, device="cuda")

        def call():
            A.copy_(A0)
            ozlu.ozlu_getrf(h, nc, 0, n, A, n, ipiv, a.nb, info, opts)
        flops = 2.0 * n ** 3 / 3.0
    call()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(a.reps):
        call()
    torch.cuda.synchronize()
    dt = (time.perf_counter() - t0) / a.reps
    print(f"{a.op} n={n} nc={nc}: {1e3 * dt:.2f} ms, {flops / dt / 1e9:.1f} Gflop/s")
    ozlu.ozlu_destroy(h)


if __name__ == "__main__":
    main()
