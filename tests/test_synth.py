"""The seeded generators produce what their docstrings state (CPU)."""
from fractions import Fraction

import numpy as np
import pytest

from oracle.expansion import expansion_value, fl_expansion, is_nonoverlapping
from synth import (lotkin_expansions, prescribed_cond_expansions, random_expansions,
                   rational_to_expansion)
from synth.prescribed import GRID_BITS, factors

torch = pytest.importorskip("torch")


def test_random_expansions_nonoverlapping_and_seeded():
    A = random_expansions(7, 9, 4, 5, -30, 30)
    B = random_expansions(7, 9, 4, 5, -30, 30)
    assert np.array_equal(A, B)
    assert all(is_nonoverlapping(A[i, j]) for i in range(7) for j in range(9))
    e = np.frexp(A[..., 0])[1]
    assert e.max() <= 30 and np.median(e) > -31


def test_lotkin_entries_are_successive_rn():
    L = lotkin_expansions(6, 3)
    for i in range(1, 6):
        for j in range(6):
            v = Fraction(1, i + j + 1)
            assert list(L[i, j]) == rational_to_expansion(v, 3)
            assert abs(expansion_value(L[i, j]) - v) <= v * Fraction(2) ** -158


@pytest.mark.parametrize("n,c,seed,nc", [(20, 12.0, 3, 4), (33, 40.0, 4, 3), (9, 5.0, 1, 2)])
def test_prescribed_cond_exact(n, c, seed, nc):
    A = prescribed_cond_expansions(n, c, seed, nc).numpy()
    Ui, Vi, m, e = factors(n, c, seed)
    for i in range(n):
        for j in range(n):
            N = sum(int(Ui[i, k]) * int(m[k]) * int(Vi[j, k]) << (int(e[k]) - int(e.min()))
                    for k in range(n))
            E = int(e.min()) - 3 - 2 * GRID_BITS
            assert list(A[i, j]) == fl_expansion(N, E, nc)


def test_prescribed_cond_spectrum():
    n, c = 24, 10.0
    A = prescribed_cond_expansions(n, c, 7, 2).numpy()
    s = np.linalg.svd(A[..., 0], compute_uv=False)
    assert abs(np.log10(s[0] / s[-1]) - c) < 0.1


@pytest.mark.parametrize("nc_in,nc,seed", [(3, 3, 1), (4, 2, 2), (2, 4, 3)])
def test_exact_row_sums(nc_in, nc, seed):
    from synth import exact_row_sums
    A = random_expansions(6, 11, nc_in, seed, -60, 60)
    A[2] = 0.0                                # an all-zero row
    A[3, :, :] = -A[4, :, :]                  # two rows that cancel each other ...
    A[3, 0, :] = A[4, 0, :]                   # ... but for one element
    A[5, 3, nc_in - 1] = 5e-324               # a subnormal component
    got = exact_row_sums(torch.from_numpy(A), nc).numpy()
    for i in range(6):
        s = sum((Fraction(float(x)) for x in A[i].ravel()), Fraction(0))
        k = s.denominator.bit_length() - 1
        assert s.denominator == 1 << k
        assert list(got[i]) == fl_expansion(s.numerator, -k, nc)


def test_exact_row_sums_long_rows():
    """More components per row than one accumulation chunk holds."""
    from synth import exact_row_sums
    A = random_expansions(2, 3000, 4, 9, -3, 3)          # 12000 components per row
    got = exact_row_sums(torch.from_numpy(A), 2).numpy()
    for i in range(2):
        s = sum((Fraction(float(x)) for x in A[i].ravel()), Fraction(0))
        k = s.denominator.bit_length() - 1
        assert list(got[i]) == fl_expansion(s.numerator, -k, 2)
