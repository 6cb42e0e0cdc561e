"""CPU oracle for the sketched inexact interior-point method (arXiv 2209.08722).

TEST INFRASTRUCTURE ONLY.  This package is a plain, slow FP64 NumPy
restatement of the paper's method, written to check the CUDA path.  Only the
test suite, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline leg
may import it.  The product path (the CUDA library and its Python binding)
never imports, links or calls anything here, and this package shares no code
with it: the only common input is the seeded problem generator ``lpgen``,
which contains none of the method's arithmetic.

Contents (each function cites the passage it follows):
  sketch      SplitMix64 counter-based generator; CountSketch and Gaussian
              sketching matrices W (Section 2, eq. pdprec; Section 6).
  pcg         Algorithm 1: SVD of ADW, Q^{-1/2}, CG and Chebyshev iteration
              on eq. (precond_alt); residual bounds eqs. (rec), (cs).
  correction  the correction vector v of eq. (compv) and the exact
              minimum-norm alternative.
  ipm         Algorithms 2 and 3: residuals, right-hand side p, directions,
              step lengths, the outer loop; "exact" mode solves the normal
              equations by Cholesky (v = 0), "sketch" mode is the paper's
              method.
  vertex      brute-force vertex enumeration for tiny LPs.

Parity status: every function here is pinned by the ``-m "not gpu"`` tests in
``tests/test_oracle_*.py`` (closed forms, invariants, brute force, library
special cases).  Functions with no such pin are marked "parity unpinned".
"""
