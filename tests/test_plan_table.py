"""The constant table every kernel reads, against the oracle's integers (CPU).

`tests/plan_host/plan_host.cpp` builds plans with the library's planner
(`csrc/plan.cpp`, compiled for the host) and prints the table the kernels
receive; each entry is recomputed here from the oracle's plan (Sec. 3.2,
Eq. (11)): the moduli, y_l = (M_l mod m_l)^-1 mod m_l, the low 32-bit words
of M_l = P / m_l and of P, 2^(16 j) mod m_l, ceil(2^32 / m_l) for the
one-multiply reduction, and 1 / m_l rounded to binary32 for F.
"""
import math
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


EXT_CONFIGS = [(300, 9, 0), (600, 19, 2), (3136, 256, 0), (12544, 256, 2)]


@pytest.fixture(scope="module")
def ext_tables(tmp_path_factory):
    cxx = shutil.which("g++") or shutil.which("c++")
    inc = _cuda_include()
    if cxx is None or inc is None:
        pytest.skip("no C++ compiler or CUDA headers")
    exe = str(tmp_path_factory.mktemp("ext") / "ext_host")
    src = [os.path.join(ROOT, "tests", "plan_host", "ext_host.cpp"), SRC[1]]
    subprocess.run([cxx, "-O1", "-std=c++17", "-I", INC, "-I", inc, "-o", exe, *src], check=True,
                   capture_output=True, text=True)
    args = [str(v) for c in EXT_CONFIGS for v in c]
    out = subprocess.run([exe, *args], check=True, capture_output=True, text=True).stdout
    res, cur = {}, None
    for line in out.splitlines():
        t = line.split()
        if t[0] == "plan":
            p, K, S, N, WG, WD, w = map(int, t[1:])
            cur = {"N": N, "WG": WG, "WD": WD, "w": w, "mods": {}}
            res[(p, K, S)] = cur
        elif t[0] == "mod":
            cur["mods"][int(t[1])] = [int(v) for v in t[2:]]
        elif t[0] == "P":
            cur["P"] = [int(v) for v in t[1:]]
    return res


@pytest.mark.parametrize("cfg", EXT_CONFIGS, ids=lambda c: f"p{c[0]}-K{c[1]}-S{c[2]}")
def test_ext_tables_match_oracle(ext_tables, cfg):
    # the device tables of the extended route (Sec. 4.2.4, Eq. (11)): moduli,
    # y_l, ceil(2^32/m), the Karatsuba plane weights (1 - 128, 16384 - 128,
    # 128) mod m, 2^w and 2^32 mod m, round(2^40/m), 2^(32 j) mod m, words of
    # M_l and of P, recomputed from the oracle's plan
    p, K, S = cfg
    tab = ext_tables[cfg]
    ref = make_plan(p, K, modset="ext", S=S or None)
    WG, WD, w = tab["WG"], tab["WD"], ref.w
    assert (tab["N"], tab["w"]) == (ref.N, ref.w)
    assert WD == (w + 2 + 31) // 32
    assert WG == (2 * w - 1 + math.ceil(math.log2(ref.S * K) - 1e-12) + 1 + 31) // 32
    for l, v in tab["mods"].items():
        m = ref.moduli[l]
        M = ref.M[l]
        inv = (1 << 40) // m + (1 if 2 * ((1 << 40) % m) >= m else 0)
        want = [m, ref.y[l], -(-(1 << 32) // m), (1 - 128) % m, (16384 - 128) % m, 128 % m,
                pow(2, w, m), (1 << 32) % m, inv, 1 % m, pow(2, 32, m), pow(2, 64, m),
                pow(2, 32 * (WD - 1), m), M & 0xffffffff, (M >> 32) & 0xffffffff,
                (M >> (32 * (WG - 1))) & 0xffffffff]
        assert v == want, l
    P = ref.P
    assert tab["P"] == [P & 0xffffffff, (P >> 32) & 0xffffffff, (P >> (32 * (WG - 1))) & 0xffffffff]


def test_autotuner_seed_is_eq_lhint(tmp_path):
    # the autotuner seeds its slice count with Eq. (Lhint); the library's
    # function (compiled for the host) against the oracle's formula
    from oracle.plan import lhint_S
    cxx = shutil.which("g++") or shutil.which("c++")
    inc = _cuda_include()
    if cxx is None or inc is None:
        pytest.skip("no C++ compiler or CUDA headers")
    exe = str(tmp_path / "plan_host")
    subprocess.run([cxx, "-O1", "-std=c++17", "-I", INC, "-I", inc, "-o", exe, *SRC], check=True,
                   capture_output=True, text=True)
    cases = [(30, 132, 512, 512), (17.9, 238, 512, 512), (30, 238, 3840, 3840), (30, 6297, 256, 256),
             (17.9, 185, 512, 512), (30, 12569, 64, 1), (30, 16, 1, 1), (30, 3161, 1792, 1792)]
    args = ["L"] + [str(v) for c in cases for v in c]
    out = subprocess.run([exe, *args], check=True, capture_output=True, text=True).stdout.split("\n")
    got = [int(l.split()[-1]) for l in out if l.startswith("lhint")]
    assert got == [lhint_S(*c) for c in cases]
