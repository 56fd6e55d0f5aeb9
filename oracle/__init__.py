"""CPU FP64 oracle for dynamic safe screening in box-constrained least squares.

TEST INFRASTRUCTURE.  This package is the plain, slow, obviously-correct statement of
what the GPU path computes, written from Dantas, Soubies and Fevotte, "Accelerating
Non-Negative and Bounded-Variable Linear Regression Algorithms with Safe Screening"
(Sections 2-5, Algorithms 1-2, Appendices B-C).  It shares no code with the CUDA path and
neither imports the other.  Only the test suite, the smoke check of the package entry
point and the CPU-baseline leg of the benchmark may import or run it; the product path
never routes through it.

Parity status: every function in ``oracle.bvls`` is pinned by tests against closed forms,
brute-force enumeration, library routines for the textbook special cases, duality
invariants or hand-derived fixtures (tests/test_oracle_*.py, tests/golden/).
"""
from .bvls import *  # noqa: F401,F403
