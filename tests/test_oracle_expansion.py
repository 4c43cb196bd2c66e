"""Pins of oracle/expansion.py: rounding against CPython's correctly rounded
rational-to-float conversion, and the expansion invariants of Sec. 2.1."""
import math
import random
from fractions import Fraction

from oracle.expansion import (double_to_dyadic, expansion_value, fl_expansion,
                              is_nonoverlapping, rn_double, ulp_p)


def test_rn_double_matches_correctly_rounded_division():
    rng = random.Random(7)
    for _ in range(3000):
        N = rng.getrandbits(rng.randint(1, 300)) * rng.choice((1, -1))
        E = rng.randint(-400, 100)
        if N == 0:
            continue
        ref = float(Fraction(N) * Fraction(2) ** E)  # correctly rounded, ties even
        assert rn_double(N, E) == ref


def test_rn_double_ties_to_even():
    assert rn_double((1 << 53) + 1, 0) == float(1 << 53)
    assert rn_double((1 << 53) + 3, 0) == float((1 << 53) + 4)
    assert rn_double(-((1 << 54) + 2), -1) == -float(1 << 53)


def test_double_to_dyadic_exact():
    rng = random.Random(3)
    for _ in range(1000):
        x = rng.uniform(-1e10, 1e10) * 2.0 ** rng.randint(-300, 300)
        N, E = double_to_dyadic(x)
        assert Fraction(N) * Fraction(2) ** E == Fraction(x)
        assert abs(N) < 2 ** 53


def test_fl_expansion_properties():
    rng = random.Random(11)
    for nc in (2, 3, 4):
        for _ in range(300):
            N = rng.getrandbits(rng.randint(60, 400)) * rng.choice((1, -1))
            E = rng.randint(-300, 0)
            limbs = fl_expansion(N, E, nc)
            v = Fraction(N) * Fraction(2) ** E
            assert is_nonoverlapping(limbs)
            # first component is the correctly rounded value
            assert limbs[0] == float(v)
            # the expansion is within about 2^-(53 nc) of v
            err = abs(expansion_value(limbs) - v)
            assert err <= abs(v) * Fraction(2) ** (-53 * nc + 1) + Fraction(0)
            # exact when the integer fits
    assert fl_expansion(12345, -3, 2) == [12345 / 8, 0.0]


def test_ulp_p():
    assert ulp_p(Fraction(1), 106) == Fraction(2) ** -105
    assert ulp_p(Fraction(3, 4), 53) == Fraction(2) ** -53
    assert ulp_p(Fraction(-8), 10) == Fraction(2) ** -6
