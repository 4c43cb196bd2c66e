"""The roofline entry of bench.py's JSON line, from fake phase statistics (CPU).

For each phase made dominant in turn, the entry names a kernel, a bound, the
achieved figure (algorithmic work over the phase time), the peak and their
ratio; the panel of the default QD workload carries the DRAM traffic per launch
from its ncu capture.
"""
from types import SimpleNamespace

import pytest

import bench

PEAKS = {"hbm_gbs": 6774.6, "bf16_tflops": 1870.7}


def _stats(dom, backend=4):
    ms = {"gemm": 1.0, "crt": 1.0, "convert": 1.0, "panel": 1.0, "trsm": 1.0}
    ms[dom] = 10.0
    return SimpleNamespace(gemm_ms=ms["gemm"], crt_ms=ms["crt"], convert_ms=ms["convert"],
                           panel_ms=ms["panel"], trsm_ms=ms["trsm"], last_backend=backend,
                           gemm_ops=2.0e12, crt_bytes=3.0e9, convert_bytes=4.0e9)


def _args(n=4096, nc=4, nb=256, panel_width=0, workload="lu"):
    return SimpleNamespace(n=n, nc=nc, nb=nb, panel_width=panel_width, workload=workload, steps=1)


@pytest.mark.parametrize("dom,kernel,bound,unit", [
    ("gemm", "gemm_tc05_kernel", "tensor", "TFLOP/s"),
    ("crt", "crt_kernel", "hbm", "GB/s"),
    ("convert", "convert_kernel", "hbm", "GB/s"),
    ("panel", "base_block_coop_kernel", "alu", "T IMAD/s"),
    ("trsm", "trsm_base_kernel", "alu", "T IMAD/s")])
def test_roofline_entry(dom, kernel, bound, unit):
    r = bench.roofline(_stats(dom), _args(), PEAKS, "measured", steps=1)
    assert (r["kernel"], r["bound"], r["unit"]) == (kernel, bound, unit)
    for key in ("achieved", "peak", "frac", "traffic", "phase_ms_per_step"):
        assert key in r
    assert r["peak"] > 0 and r["achieved"] > 0
    assert abs(r["frac"] - r["achieved"] / r["peak"]) < 1e-12
    if dom == "gemm":
        assert r["peak"] == PEAKS["bf16_tflops"] and abs(r["achieved"] - 200.0) < 1e-9
    if dom in ("crt", "convert"):
        assert r["peak"] == PEAKS["hbm_gbs"]
    if dom == "panel":
        # the capture's traffic only while the kernel source is the captured one
        bytes_, digest = bench.PANEL_TRAFFIC[(4096, 4, 256, 0)]
        want = bytes_ if digest == bench.panel_source_digest() else None
        assert r["traffic"] == want
        assert r["work"]["limb_products"] == bench.panel_products(4096, 256)
    else:
        assert r["traffic"] is None


def test_panel_products_count():
    # base blocks of the recursive panel: 128-column leaves; column kc of a leaf
    # (c0, w) costs (n - c0 - kc - 1) (w - kc) limb products; brute force
    assert bench.panel_leaves(0, 256) == [(0, 128), (128, 128)]
    assert bench.panel_leaves(0, 100) == [(0, 100)]
    n, nb = 300, 256
    total = 0
    for r0 in range(0, n, nb):
        b = min(nb, n - r0)
        leaves = [(r0, b)] if b <= 128 else [(r0, b // 2), (r0 + b // 2, b - b // 2)]
        for c0, w in leaves:
            for kc in range(w):
                rows = n - c0 - kc - 1
                total += rows * 1 + rows * (w - kc - 1)
    assert bench.panel_products(n, nb) == total


def test_panel_traffic_only_for_the_captured_workload():
    r = bench.roofline(_stats("panel"), _args(n=2048), PEAKS, "measured", steps=1)
    assert r["traffic"] is None
    r = bench.roofline(_stats("panel"), _args(panel_width=64), PEAKS, "measured", steps=1)
    assert r["traffic"] is None


def test_fp8_gemm_peak_is_twice_bf16():
    r = bench.roofline(_stats("gemm", backend=2), _args(), PEAKS, "measured", steps=1)
    assert r["peak"] == 2 * PEAKS["bf16_tflops"]
