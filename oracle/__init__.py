"""CPU FP64 oracle for the low-rank PCG control solve (TEST INFRASTRUCTURE ONLY).

This package is the slow, plain reference that the CUDA library is checked
against.  Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline /
reference legs of ``bench.py`` may import it; the library package never does,
and the oracle never imports the library.  The two share no code; the only
common import is the seeded input generator ``fc_inputs``, which holds none of
the method's arithmetic.

Paper: Heidel, Khoromskaia, Khoromskij, Schulz, "Tensor product method for fast
solution of optimal control problems with fractional multidimensional Laplacian
in constraints" (arXiv:1809.01971).  Every function cites the section /
equation / algorithm it follows.

Modules
  spectrum    1D Dirichlet Laplacian, closed-form eigenvalues (eqn:eig_lap),
              orthonormal DST-I (Section 3.2).
  quadrature  sinc quadrature of the Laplace transform (eqn:Laplace_transf,
              eqn:Sinc_quadr_trunc, eqn:Func_of_rho), the CP symbol of the
              control operator with Lemma 4.1 for the positive power, and the
              low-rank preconditioner fit.
  cp          canonical tensors (eqn:CP_form): full expansion, inner product,
              linear combination, the mode-wise mat-vec (eqn:Lap2DtimesX,
              eqn:Lap3DtimesX).
  truncate    RHOSVD canonical -> Tucker -> canonical rank truncation
              (Section 5, eqn:two_level) and the 2D reduced SVD.
  pcg         Algorithm 1 (low-rank PCG).
  full        full-format eigenbasis solve (eqn:DiagFLaplace3D), the state
              y = beta A^-alpha u (eqn:State), the directionally fractional
              Laplacian solve (Remark after Lemma 4.1), and dense
              eigendecomposition brute forces of both for small n.
  eigerr      the error of a CP solution against the exact full-format solution
              (eqn:DiagFLaplace3D), summed point by point over the whole eigen-index
              grid in plain C (csrc/eigerr.c), no n^d array formed.

Parity status: every function is pinned by tests/test_oracle_*.py against
closed forms, brute force or library routines; none is "parity unpinned".
"""
