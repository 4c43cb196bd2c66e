"""The constant table every kernel reads, against the oracle's integers (CPU).

`tests/plan_host/plan_host.cpp` builds plans with the library's planner
(`csrc/plan.cpp`, compiled for the host) and prints the table the kernels
receive; each entry is recomputed here from the oracle's plan (Sec. 3.2,
Eq. (11)): the moduli, y_l = (M_l mod m_l)^-1 mod m_l, the low 32-bit words
of M_l = P / m_l and of P, 2^(16 j) mod m_l, ceil(2^32 / m_l) for the
one-multiply reduction, and 1 / m_l rounded to binary32 for F.
"""
import os
import shutil
import subprocess

import numpy as np
import pytest

from oracle.plan import make_plan

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = [os.path.join(ROOT, "tests", "plan_host", "plan_host.cpp"),
       os.path.join(ROOT, "paper_2609_29554_gb300", "csrc", "plan.cpp"),
       os.path.join(ROOT, "paper_2609_29554_gb300", "csrc", "noalloc_plan.cpp")]
INC = os.path.join(ROOT, "paper_2609_29554_gb300", "csrc")
MAXH, MAXWG = 16, 16
# 0: the p-bit planner; -1: the allocation-free GEMM's planner (INT8)
BACKENDS = {-1: "int8", 0: "int8", 1: "int8", 2: "fp8", 3: "fp64", 4: "fp16"}
CONFIGS = [(106, 32, 1), (159, 512, 1), (212, 256, 1), (212, 4096, 1), (212, 256, 2),
           (212, 256, 4), (106, 512, 3), (212, 512, 3), (3136, 256, 0), (12544, 256, 0),
           (64, 1, 0), (106, 19, -1), (159, 256, -1), (212, 256, -1), (212, 100, -1),
           (150, 4096, -1)]


def _cuda_include():
    for d in (os.environ.get("CUDA_HOME"), "/usr/local/cuda"):
        if d and os.path.exists(os.path.join(d, "include", "cuda_runtime.h")):
            return os.path.join(d, "include")
    return None


@pytest.fixture(scope="module")
def tables(tmp_path_factory):
    cxx = shutil.which("g++") or shutil.which("c++")
    inc = _cuda_include()
    if cxx is None or inc is None:
        pytest.skip("no C++ compiler or CUDA headers")
    exe = str(tmp_path_factory.mktemp("plan") / "plan_host")
    subprocess.run([cxx, "-O1", "-std=c++17", "-I", INC, "-I", inc, "-o", exe, *SRC], check=True,
                   capture_output=True, text=True)
    args = [str(v) for c in CONFIGS for v in c]
    out = subprocess.run([exe, *args], check=True, capture_output=True, text=True).stdout
    res, cur = {}, None
    for line in out.splitlines():
        t = line.split()
        if t[0] == "plan":
            p, K, be, S, w, N, WG = map(int, t[1:])
            cur = {"S": S, "w": w, "N": N, "WG": WG, "mods": []}
            res[(p, K, be)] = cur
        elif t[0] == "mod":
            m, y, magic = int(t[2]), int(t[3]), int(t[4])
            invm = float.fromhex(t[5])
            pow16 = [int(v) for v in t[6:6 + MAXH]]
            mlow = [int(v) for v in t[6 + MAXH:6 + MAXH + MAXWG]]
            cur["mods"].append((m, y, magic, invm, pow16, mlow))
        elif t[0] == "Plow":
            cur["Plow"] = [int(v) for v in t[1:]]
    return res


def _words(x, n):
    return [(x >> (32 * i)) & 0xffffffff for i in range(n)]


@pytest.mark.parametrize("cfg", CONFIGS, ids=lambda c: f"p{c[0]}-K{c[1]}-be{c[2]}")
def test_table_matches_oracle(tables, cfg):
    p, K, be = cfg
    tab = tables[cfg]
    ref = make_plan(p, K, backend=BACKENDS[be])
    assert (tab["S"], tab["w"], tab["N"]) == (ref.S, ref.w, ref.N)
    assert [m for m, *_ in tab["mods"]] == list(ref.moduli)
    mask = (1 << (32 * MAXWG)) - 1
    for l, (m, y, magic, invm, pow16, mlow) in enumerate(tab["mods"]):
        M = ref.P // m
        assert M == ref.M[l] and (M * y) % m == 1 and y == ref.y[l]
        assert mlow == _words(M & mask, MAXWG)
        assert pow16 == [pow(2, 16 * j, m) for j in range(MAXH)]
        assert magic == -(-(1 << 32) // m)
        assert invm == float(np.float32(1.0) / np.float32(m))
    assert tab["Plow"] == _words(ref.P & mask, MAXWG)


@pytest.mark.parametrize("p,K", [(106, 19), (159, 256), (212, 256), (212, 100), (150, 4096)])
def test_noalloc_table_equals_handle_planner(tables, p, K):
    # the allocation-free GEMM keeps its own fixed-array planner: its table
    # must be the handle planner's INT8 table entry for entry
    na = tables[(p, K, -1)]
    assert na["N"] > 0
    ref = make_plan(p, K, backend="int8")
    assert (na["S"], na["w"], na["N"]) == (ref.S, ref.w, ref.N)
