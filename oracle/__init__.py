"""CPU oracle for the block-CGrQ improved-staggered solver.

TEST INFRASTRUCTURE: only the tests, the smoke check and the benchmark's CPU
baseline leg may import or run anything in this package.  The product path
(the CUDA library and its Python binding) never imports it, and this package
never imports the product path.

Contents:
  hisq_oracle.c   plain FP64 C: staggered stencil D (Eq. 2), the even-odd
                  normal operator A = m^2 - D_eo D_oe (Sec. 3.2) and textbook
                  CG per column (the baseline of Sec. 7.1)
  hisq.py         ctypes wrappers of the C functions on NumPy arrays
  block.py        block cDot / block caxpy (Sec. 6.3, 5.4), thin QR
                  (Algorithm 2), blockCGrQ (Algorithm 1) and block reliable
                  updates (Algorithm 3), in NumPy FP64, step by step
  dense.py        dense matrix of A on tiny lattices, for brute-force checks
  build.py        compiles hisq_oracle.c with gcc

Pins (in tests/test_oracle_*.py) tie every function to something other than
itself: free-field plane-wave eigenvalues, pure-gauge spectra, gauge
covariance, hermiticity and positivity, dense solves, N=1 equivalence with
textbook CG, and the algebraic invariants of Algorithms 1-3.
"""
