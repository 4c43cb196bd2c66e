"""Binary floating point with a p-bit significand, round to nearest even.

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

The reference LU of the oracle runs at p + 64 bits (p the target precision).
A number is an exact pair (N, E) meaning N * 2^E with |N| < 2^prec after
rounding; every operation forms the exact result with Python integers and
rounds it once, so each add, multiply, fused multiply-subtract and divide is
correctly rounded.
"""
from __future__ import annotations

from fractions import Fraction


def bf_round(N: int, E: int, prec: int) -> tuple[int, int]:
    """Round N * 2^E to prec significant bits, ties to even."""
    if N == 0:
        return 0, 0
    neg = N < 0
    a = -N if neg else N
    L = a.bit_length()
    if L > prec:
        sh = L - prec
        q = a >> sh
        r = a - (q << sh)
        half = 1 << (sh - 1)
        if r > half or (r == half and (q & 1)):
            q += 1
        a, E = q, E + sh
        if a.bit_length() > prec:  # carried into a new bit
            a >>= 1
            E += 1
    return (-a if neg else a), E


def bf_from_fraction(v: Fraction, prec: int) -> tuple[int, int]:
    """Correctly rounded p-bit value of a rational."""
    if v == 0:
        return 0, 0
    neg = v < 0
    a = -v if neg else v
    num, den = a.numerator, a.denominator
    # choose k with num * 2^k // den having prec + 2 bits at least
    k = prec + 2 - (num.bit_length() - den.bit_length())
    if k >= 0:
        q, r = divmod(num << k, den)
    else:
        q, r = divmod(num, den << (-k))
    # sticky: append one bit that is set when the remainder is nonzero
    q = (q << 1) | (1 if r else 0)
    N, E = bf_round(q, -k - 1, prec)
    return (-N if neg else N), E


def bf_to_fraction(x: tuple[int, int]) -> Fraction:
    N, E = x
    return Fraction(N) * (Fraction(2) ** E)


def bf_add(x, y, prec):
    (a, ea), (b, eb) = x, y
    if a == 0:
        return bf_round(b, eb, prec)
    if b == 0:
        return bf_round(a, ea, prec)
    e = min(ea, eb)
    return bf_round((a << (ea - e)) + (b << (eb - e)), e, prec)


def bf_neg(x):
    return (-x[0], x[1])


def bf_sub(x, y, prec):
    return bf_add(x, bf_neg(y), prec)


def bf_mul(x, y, prec):
    return bf_round(x[0] * y[0], x[1] + y[1], prec)


def bf_fms(c, a, b, prec):
    """c - a*b rounded once."""
    pa, pe = a[0] * b[0], a[1] + b[1]
    if c[0] == 0:
        return bf_round(-pa, pe, prec)
    if pa == 0:
        return bf_round(c[0], c[1], prec)
    e = min(pe, c[1])
    return bf_round((c[0] << (c[1] - e)) - (pa << (pe - e)), e, prec)


def bf_div(x, y, prec):
    if y[0] == 0:
        raise ZeroDivisionError("p-bit division by zero")
    if x[0] == 0:
        return 0, 0
    return bf_from_fraction(Fraction(x[0], y[0]) * (Fraction(2) ** (x[1] - y[1])), prec)


def bf_abs_cmp(x, y) -> int:
    """Compare |x| with |y| exactly: -1, 0, 1."""
    a, ea = abs(x[0]), x[1]
    b, eb = abs(y[0]), y[1]
    if a == 0 or b == 0:
        return (a > 0) - (b > 0)
    e = min(ea, eb)
    a <<= ea - e
    b <<= eb - e
    return (a > b) - (a < b)
