"""Seeded synthetic inputs shared by the tests, the benchmark and the oracle.

This package generates matrices only: it holds none of the Ozaki-II
arithmetic and none of the LU.  Every generator is deterministic given its
arguments (numpy default_rng seeds).

  random_expansions   the standalone-GEMM workload (Sec. 4.2 style data):
                      leading components uniform [-1, 1) times 2^e,
                      e uniform in [emin, emax], each lower component random
                      below a quarter ulp of the one before it
  lotkin_expansions   the Lotkin matrix of Sec. 4.4 rounded component by
                      component from exact rationals
  lotkin_rhs          b = A * ones formed exactly from the rational matrix,
                      then rounded
  prescribed_cond_expansions
                      A = U diag(sigma) V^T with U, V from the QR of seeded
                      N(0, 1) matrices and sigma geometric from 1 to 10^-c,
                      formed exactly (synth/prescribed.py)
  exact_row_sums      b = A * ones of a stored expansion matrix, exactly,
                      then rounded
"""
from .matrices import (lotkin_expansions, lotkin_rhs, random_expansions,
                       rational_to_expansion)
from .prescribed import exact_row_sums, prescribed_cond_expansions

__all__ = ["random_expansions", "lotkin_expansions", "lotkin_rhs",
           "rational_to_expansion", "prescribed_cond_expansions", "exact_row_sums"]
