"""CPU oracle for the time-periodic fixed-point solver (TEST INFRASTRUCTURE).

This package is a plain, slow, fp64 CPU implementation of what the CUDA path
computes.  It exists only to check that path: the only code allowed to
import it is the test suite, the smoke check and the CPU-baseline leg of the
benchmark.  The product path never calls it, and it shares no code with the
CUDA library (the two meet only in the seeded input generators of
`workloads.py`, which hold no arithmetic of the method).

Contents (each function cites the passage of the paper it follows):
  fem       P1 geometry, stiffness and mass assembly, the reluctivity law and
            the nonlinear operator K(u) of Section 4 (test problem).
  periodic  the discrete operator A(U) of Problem 1 / eq. (disc), the source
            F, exact solvers for the periodic time-invariant linear system of
            eq. (iter1)-(iter2) (space-time sparse LU and time-DFT), the
            fixed-point iteration of eq. (iter1)-(iter2) and a dense Newton
            solver used as an independent brute force on tiny meshes.
  adjoint   the discrete adjoint of the period-averaged eddy-current loss.

Parity status: every function is pinned by tests in tests/test_oracle_*.py
against closed forms, textbook stencils and brute force (see each test).
"""
from . import fem, periodic  # noqa: F401
