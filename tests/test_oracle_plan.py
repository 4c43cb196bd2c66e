"""Pins of oracle/plan.py against the paper's printed counts and arithmetic."""
import math
import os

import pytest

from oracle.plan import (fp64_moduli, int8_moduli, make_plan, pairs_in_group,
                         primes_upto, single_pass_pmax)

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "paper_counts.txt")


def _rows():
    for line in open(GOLDEN):
        line = line.split("#", 1)[0].strip()
        if line:
            be, p, K, S, N, ng = line.split()
            yield (be, int(p), int(K), None if S == "-" else int(S),
                   None if N == "-" else int(N), None if ng == "-" else int(ng))


@pytest.mark.parametrize("row", list(_rows()), ids=lambda r: f"{r[0]}-p{r[1]}-K{r[2]}")
def test_printed_counts(row):
    be, p, K, S, N, ng = row
    plan = make_plan(p, K, backend=be, S=S)
    if N is not None:
        assert plan.N == N
    if ng is not None:
        assert plan.n_gemm == ng


def test_54_moduli_capacity():
    # Sec. 3.2: at most 54 pairwise-coprime moduli <= 255, about 362.8 bits
    ms = int8_moduli()
    assert len(ms) == 54 and max(ms) == 251 and ms == sorted(ms, reverse=True)
    for i in range(len(ms)):
        for j in range(i + 1, len(ms)):
            assert math.gcd(ms[i], ms[j]) == 1
    assert abs(sum(map(math.log2, ms)) - 361.83) < 0.01
    # the printed 362.8 is the same set with 2^8 in place of 2^7
    assert abs(sum(map(math.log2, int8_moduli(use_256=True))) - 362.83) < 0.01
    # every modulus is the largest power of its prime not above 255
    for m in ms:
        q = next(q for q in primes_upto(255) if m % q == 0)
        assert m <= 255 < m * q


def test_fp8_single_digit_capacity():
    # Table fpfmt / Sec. 4.2.3: one E4M3 digit allows only m <= 33, 47.0 bits
    mods = []
    for q in primes_upto(33):
        v = q
        while v * q <= 33:
            v *= q
        mods.append(v)
    assert round(sum(map(math.log2, mods)), 1) == 47.0


def test_fp64_modulus_bound():
    # Eq. (17): m < sqrt(2^55/K); at K = 512, m < 8.4e6, about 23 bits
    ms = fp64_moduli(512)
    assert ms[0] < 8.4e6 and ms[0] > 8.38e6
    assert 512 * (ms[0] / 2) ** 2 < 2 ** 53


def test_crt_constants():
    plan = make_plan(212, 256)
    for Ml, m, y in zip(plan.M, plan.moduli, plan.y):
        assert Ml * m == plan.P
        assert (Ml * y) % m == 1
    assert plan.P == math.prod(plan.moduli)
    assert math.log2(plan.P) > plan.need


def test_pair_count_eq4():
    # Eq. (4): groups S-1..2S-2 hold S(S+1)/2 pair terms
    for S in range(1, 12):
        assert sum(pairs_in_group(g, S) for g in range(S - 1, 2 * S - 1)) == S * (S + 1) // 2
        assert sum(pairs_in_group(g, S) for g in range(0, 2 * S - 1)) == S * S


def test_proposition1_example():
    # Prop. 1: K = 4096, g = 8 gives p_max "about 155" bits
    assert abs(single_pass_pmax(4096, 8) - 155) < 3


def test_single_pass_dd_only():
    # Sec. 3.2 after Prop. 1: DD barely fits one pass, TD and QD need slices
    assert make_plan(106, 512).S == 1
    assert make_plan(159, 512).S >= 2 and make_plan(212, 512).S >= 2


def test_capacity_margin_and_int32():
    for p in (106, 159, 212, 1024, 12544):
        for K in (32, 256, 1024):
            plan = make_plan(p, K)
            cap = sum(math.log2(m) for m in plan.moduli)
            assert cap > plan.need
            assert cap - math.log2(plan.moduli[-1]) <= plan.need  # fewest moduli
            # |S_g| <= S K 2^(2w-2): 2|S_g| < P with >= 5 bits to spare
            assert math.log2(plan.S * K) + 2 * plan.w - 1 + 5 < cap
            assert K * plan.S * 127 * 127 < 2 ** 31


def test_extra_groups():
    plan = make_plan(212, 256, extra_groups=1)
    assert plan.g0 == plan.S - 2 and plan.pair_terms == 4  # S = 2: groups 0,1,2
