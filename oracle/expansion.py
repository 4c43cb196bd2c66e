"""Exact values of binary64 numbers and non-overlapping expansions.

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

Sec. 2.1: a DD/TD/QD number is a non-overlapping expansion x = sum_c x[c] of
nc = 2/3/4 binary64 components stored contiguously as double[nc]; x[0] is the
rounded value and each later component the rounded residual.  Sec. 3.3 writes
each component as x[c] = +-m_c 2^(e_c - 53) with a 53-bit integer m_c.

A dyadic number is carried here as an exact pair (N, E) meaning N * 2^E with
Python integers, so nothing is ever rounded unless a function says so.
"""
from __future__ import annotations

import math
from fractions import Fraction


def frexp_exponent(x: float) -> int:
    """e with 2^(e-1) <= |x| < 2^e (math.frexp), for x != 0."""
    if x == 0.0:
        raise ValueError("zero has no exponent")
    return math.frexp(x)[1]


def double_to_dyadic(x: float) -> tuple[int, int]:
    """x = N * 2^E exactly, |N| < 2^53 (Sec. 3.3: x = +-m 2^(e-53))."""
    if x == 0.0:
        return 0, 0
    if not math.isfinite(x):
        raise ValueError("non-finite component")
    m, e = math.frexp(x)
    return int(m * (1 << 53)), e - 53


def dyadic_to_fraction(N: int, E: int) -> Fraction:
    return Fraction(N) * (Fraction(2) ** E)


def expansion_value(limbs) -> Fraction:
    """Exact value sum_c x[c] of an expansion (Sec. 2.1)."""
    total = Fraction(0)
    for x in limbs:
        N, E = double_to_dyadic(float(x))
        total += dyadic_to_fraction(N, E)
    return total


def expansion_dyadic(limbs) -> tuple[int, int]:
    """Exact value of an expansion as one (N, E) on the finest limb grid."""
    parts = [double_to_dyadic(float(x)) for x in limbs if float(x) != 0.0]
    if not parts:
        return 0, 0
    E = min(e for _, e in parts)
    return sum(n << (e - E) for n, e in parts), E


def rn_double(N: int, E: int) -> float:
    """Round N * 2^E to the nearest binary64, ties to even.

    Written from the definition: keep the top 53 bits of |N|, look at the
    discarded part against one half unit, break exact halves to even.
    The result must lie in the normal binary64 range.
    """
    if N == 0:
        return 0.0
    sign = -1.0 if N < 0 else 1.0
    a = -N if N < 0 else N
    L = a.bit_length()
    if L <= 53:
        q, shift = a, 0
    else:
        shift = L - 53
        q = a >> shift
        r = a - (q << shift)
        half = 1 << (shift - 1)
        if r > half or (r == half and (q & 1)):
            q += 1
    exp = E + shift
    # q * 2^exp must be a normal binary64 (q <= 2^53)
    top = exp + q.bit_length()
    if top > 1024 or exp + q.bit_length() - 1 < -1022:
        raise OverflowError("result outside the normal binary64 range")
    return sign * math.ldexp(float(q), exp)


def fl_expansion(N: int, E: int, nc: int) -> list[float]:
    """Round N * 2^E to nc components by successive round-to-nearest.

    x0 = RN(v), x1 = RN(v - x0), ...: the component-by-component rounding the
    expansion format defines (Sec. 2.1), used for the single rounding of (S6)
    and for the output slicing of Sec. 3.3.  Each residual is an exact
    integer multiple of 2^E, so the loop never rounds the residual itself.
    """
    out = []
    R = N
    for _ in range(nc):
        x = rn_double(R, E) if R != 0 else 0.0
        out.append(x)
        if x != 0.0:
            n, e = double_to_dyadic(x)
            # x is a multiple of 2^E whenever it rounded away any bits
            if e >= E:
                R -= n << (e - E)
            else:
                assert (n % (1 << (E - e))) == 0
                R -= n >> (E - e)
    return out


def fl_expansion_of_fraction(v: Fraction, nc: int, guard_bits: int = 64) -> list[float]:
    """Successive RN of an arbitrary rational, exact for dyadic v.

    For a non-dyadic v the value is first truncated to a dyadic grid guard_bits
    below nc*53 bits of its leading bit; the caller states the guard it needs.
    """
    if v == 0:
        return [0.0] * nc
    lead = math.floor(math.log2(abs(v))) if v != 0 else 0
    E = lead - 53 * nc - guard_bits
    scaled = v / (Fraction(2) ** E)
    # round to nearest on the fine grid (exact for dyadic v at this grid)
    N = math.floor(scaled + Fraction(1, 2))
    return fl_expansion(N, E, nc)


def ulp_p(v: Fraction, p: int) -> Fraction:
    """ulp_p(c) = 2^(floor(log2|c|) - p + 1) (the target precision unit)."""
    if v == 0:
        return Fraction(0)
    a = abs(v)
    e = a.numerator.bit_length() - a.denominator.bit_length()
    # fix e so that 2^e <= a < 2^(e+1)
    if Fraction(2) ** e > a:
        e -= 1
    elif Fraction(2) ** (e + 1) <= a:
        e += 1
    return Fraction(2) ** (e - p + 1)


def is_nonoverlapping(limbs) -> bool:
    """|x[c+1]| <= ulp(x[c]) / 2 for consecutive nonzero components."""
    prev = None
    for x in limbs:
        x = float(x)
        if x == 0.0:
            continue
        if prev is not None:
            half_ulp = math.ldexp(1.0, frexp_exponent(prev) - 54)
            if abs(x) > half_ulp:
                return False
        prev = x
    return True
