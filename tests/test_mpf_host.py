"""Host build of the panel's multi-limb float arithmetic against exact rationals.

`tests/mpf_host/mpf_host.cpp` compiles the device header `csrc/mpf.cuh` as
plain C++ (portable definitions of the few CUDA intrinsics it uses) and prints
seeded cases for L = 4, 6, 7, 8 words; every result is checked here with exact
rational arithmetic:
  * mpf_mul, mpf_add: the exact result rounded to L words, to nearest even;
  * mpf_fms (c - a b with one rounding): the same, including exact
    cancellations (c = a b gives zero);
  * mpf_recip: |1 - a r| < 2^-(32 L - 1) and the sign of a, for random,
    f = 1/2, all-ones and single-low-bit mantissas over a wide exponent range;
  * mpf_from_exp (N binary64 components, nonoverlapping, mixed signs, zero
    components) rounds the exact sum to L words; mpf_to_exp gives the
    successive round-to-nearest-even components x_c = RN(v - x_0 - ... - x_{c-1});
  * mod_small (x mod m by one high multiply, used for every residue and t
    value) equals x % m for every m <= 255 over edge values and a sample of
    [0, 2^32).
"""
import os
import shutil
import subprocess
from fractions import Fraction

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "tests", "mpf_host", "mpf_host.cpp")
INC = os.path.join(ROOT, "paper_2609_29554_gb300", "csrc")


@pytest.fixture(scope="module")
def cases(tmp_path_factory):
    cxx = shutil.which("g++") or shutil.which("c++")
    if cxx is None:
        pytest.skip("no C++ compiler")
    exe = str(tmp_path_factory.mktemp("mpf") / "mpf_host")
    subprocess.run([cxx, "-O1", "-std=c++17", "-I", INC, "-o", exe, SRC], check=True,
                   capture_output=True, text=True)
    out = subprocess.run([exe, "600"], check=True, capture_output=True, text=True).stdout
    rows = []
    for line in out.splitlines():
        t = line.split()
        op, L = t[0], int(t[1]) if t[0] != "mod" else 0

        def mpf(k):
            return int(t[k]), int(t[k + 1]), int("".join(t[k + 2:k + 2 + L]), 16)

        if op == "mod":            # cases mismatches
            rows.append((op, 0, (int(t[1]), int(t[2]))))
            continue
        if op == "fromexp":        # L N x[0..N) result
            N = int(t[2])
            rows.append((op, L, ([float.fromhex(v) for v in t[3:3 + N]], mpf(3 + N))))
        elif op == "toexp":        # L N a out[0..N)
            N = int(t[2])
            rows.append((op, L, (mpf(3), [float.fromhex(v) for v in t[5 + L:5 + L + N]])))
        else:
            vals, k = [], 2
            while k < len(t):
                vals.append(mpf(k))
                k += 2 + L
            rows.append((op, L, vals))
    return rows


def value(x, L):
    neg, e, m = x
    v = Fraction(m) * Fraction(2) ** (e - 32 * L)
    return -v if neg else v


def rne(x, L):
    """(neg, e, m) of x rounded to L words, to nearest even; m = 0 for zero."""
    if x == 0:
        return None
    neg = 1 if x < 0 else 0
    ax = abs(x)
    k = ax.numerator.bit_length() - ax.denominator.bit_length()
    E = k + 1 if ax >= Fraction(2) ** k else k
    s = ax * Fraction(2) ** (32 * L - E)
    q = s.numerator // s.denominator
    rem = s - q
    if rem > Fraction(1, 2) or (rem == Fraction(1, 2) and q & 1):
        q += 1
    if q == 1 << (32 * L):
        q >>= 1
        E += 1
    return neg, E, q


def same(got, want):
    if want is None:
        return got[2] == 0
    return got[2] != 0 and got == want


@pytest.mark.parametrize("op", ["mul", "add", "fms"])
def test_correctly_rounded(cases, op):
    n = bad = 0
    for o, L, v in cases:
        if o != op:
            continue
        if op == "mul":
            a, b, r = v
            exact = value(a, L) * value(b, L)
        elif op == "add":
            a, b, r = v
            exact = value(a, L) + value(b, L)
        else:
            c, a, b, r = v
            exact = value(c, L) - value(a, L) * value(b, L)
        n += 1
        bad += not same(r, rne(exact, L))
    assert n > 1000
    assert bad == 0, f"{bad} of {n} {op} results not correctly rounded"


def test_fms_exact_cancellation_is_zero(cases):
    n = 0
    for o, L, v in cases:
        if o == "fms":
            c, a, b, r = v
            if value(a, L) != 0 and value(c, L) == value(a, L) * value(b, L):
                n += 1
                assert r[2] == 0
    assert n > 100


def test_recip(cases):
    n = 0
    for o, L, v in cases:
        if o != "recip":
            continue
        a, r = v
        n += 1
        assert r[2] != 0 and r[0] == a[0]
        err = abs(1 - value(a, L) * value(r, L))
        assert err < Fraction(2) ** -(32 * L - 1), (L, float(err))
    assert n >= 1800


def test_from_expansion(cases):
    n = bad = 0
    for o, L, (x, r) in ((o, L, v) for o, L, v in cases if o == "fromexp"):
        n += 1
        exact = sum((Fraction(c) for c in x), Fraction(0))
        bad += not same(r, rne(exact, L))
    assert n >= 1800
    assert bad == 0, f"{bad} of {n} conversions not correctly rounded"


def test_to_expansion(cases):
    n = 0
    for o, L, (a, out) in ((o, L, v) for o, L, v in cases if o == "toexp"):
        n += 1
        rem = value(a, L)
        for c in out:
            want = float(rem)          # round to nearest even
            assert c == want
            rem -= Fraction(c)
    assert n >= 1800


def test_mod_small(cases):
    (n, bad), = [v for o, L, v in cases if o == "mod"]
    assert n > 40_000_000 and bad == 0
