"""Host build of the binary64 expansion arithmetic against exact rationals (CPU).

`tests/mpf_host/exp_host.cpp` compiles `csrc/expansion.cuh` (TwoSum/TwoProd
expansions of N = 2, 3, 4 components: the native per-element LU comparison and
the non-cooperative panel column kernels) as plain C++ without contraction and
prints seeded cases, near-cancelling sums included.  Checked here exactly:
add, mul, div and fms (c - a b) stay within 4 units of 2^(-53 N) of the exact
result, relative to the operands' magnitude (|a| + |b|, |a b|, |a / b|,
|c| + |a b|), and every result is non-overlapping, |x[k+1]| <= ulp(x[k]) / 2.
"""
import math
import os
import shutil
import subprocess
from fractions import Fraction

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "tests", "mpf_host", "exp_host.cpp")
INC = os.path.join(ROOT, "paper_2609_29554_gb300", "csrc")


@pytest.fixture(scope="module")
def cases(tmp_path_factory):
    cxx = shutil.which("g++") or shutil.which("c++")
    if cxx is None:
        pytest.skip("no C++ compiler")
    exe = str(tmp_path_factory.mktemp("exp") / "exp_host")
    subprocess.run([cxx, "-O1", "-std=c++17", "-ffp-contract=off", "-I", INC, "-o", exe, SRC],
                   check=True, capture_output=True, text=True)
    out = subprocess.run([exe, "600"], check=True, capture_output=True, text=True).stdout
    rows = []
    for line in out.splitlines():
        t = line.split()
        op, N = t[0], int(t[1])
        v = [float.fromhex(x) for x in t[2:]]
        rows.append((op, N, [v[i * N:(i + 1) * N] for i in range(len(v) // N)]))
    return rows


def _val(x):
    return sum((Fraction(c) for c in x), Fraction(0))


@pytest.mark.parametrize("op", ["add", "mul", "div", "fms"])
def test_error_bound_and_nonoverlap(cases, op):
    n = 0
    for o, N, ops in cases:
        if o != op:
            continue
        n += 1
        v = [_val(x) for x in ops]
        if op == "add":
            exact, scale = v[0] + v[1], abs(v[0]) + abs(v[1])
        elif op == "mul":
            exact = v[0] * v[1]
            scale = abs(exact)
        elif op == "div":
            exact = v[0] / v[1]
            scale = abs(exact)
        else:
            exact = v[0] - v[1] * v[2]
            scale = abs(v[0]) + abs(v[1] * v[2])
        assert abs(v[-1] - exact) <= 4 * scale * Fraction(2) ** (-53 * N), (op, N)
        r = ops[-1]
        for k in range(N - 1):
            if r[k] == 0.0:
                assert r[k + 1] == 0.0
            else:
                assert abs(r[k + 1]) <= math.ulp(r[k]) / 2
    assert n == 1800
