"""CPU oracle for the Ozaki-scheme-II multiple-precision GEMM and LU.

TEST INFRASTRUCTURE ONLY.  Nothing in the product path (the CUDA library and
its Python binding) may import, call or link anything in this package; only
the tests, ``__graft_entry__.smoke()`` and the ``cpu_baseline`` / reference
legs of ``bench.py`` use it.

Everything here is plain, slow and exact: Python integers and fractions,
numpy integer matrix products used only as an exact library matmul.  Each
function cites the passage of the paper (Kouya, "Accelerating
Multiple-Precision LU Decomposition with Ozaki Scheme II") that it follows.

Modules
  plan       modulus set, CRT constants, the (S, w, N_mod) rule    Sec. 3.2
  expansion  exact values of DD/TD/QD expansions, RN to binary64   Sec. 2.1, 3.3
  oz2        Ozaki-II GEMM replay in exact integers (S1)-(S6)       Sec. 3.1-3.3
  mp         the same replay for p-bit multi-limb numbers           Sec. 3.1, 3.4
  bigfloat   p-bit floating point with round-to-nearest-even        (LU at p+64)
  lu         exact rational LU, p-bit LU, solve, error measures     Sec. 3.4, 4.4

Parity pins: every function is checked in tests/ against values the paper
prints, closed forms, brute force on tiny inputs or independent procedures;
the one function without such a pin is marked "parity unpinned" in its
docstring (the exact truncation errors of the cancellation experiment of
Sec. 3.2, whose matrix construction the paper does not give).
"""
