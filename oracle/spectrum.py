"""1D spectrum and sine transform (paper Section 3.2).

Readings of the paper (its printed formulas carry sign/scale slips):
  * A_(l) = h^-2 tridiag(-1, 2, -1) (the paper prints a -1/h prefactor), so
    A_(l) is symmetric positive definite.
  * n interior points, h = 1/(n+1) (Section 4.1 states h = 1/(n+1)).
  * lambda_k = +(4/h^2) sin^2(pi k / (2(n+1))), k = 1..n (eqn:eig_lap with the
    spurious minus sign dropped).
  * F is the orthonormal DST-I, F[j,k] = sqrt(2/(n+1)) sin(pi j k/(n+1)), so
    F = F^T = F^-1 and A_(l) = F Lambda F.
"""
from __future__ import annotations

import numpy as np
import scipy.fft


def laplacian_1d(n: int) -> np.ndarray:
    """Dense 1D FD Dirichlet Laplacian h^-2 tridiag(-1,2,-1) (Section 3.2)."""
    h = 1.0 / (n + 1)
    A = 2.0 * np.eye(n) - np.eye(n, k=1) - np.eye(n, k=-1)
    return A / h**2


def eigenvalues(n: int) -> np.ndarray:
    """lambda_k = (4/h^2) sin^2(pi k/(2(n+1))), k = 1..n (eqn:eig_lap)."""
    N = n + 1
    h = 1.0 / N
    k = np.arange(1, n + 1, dtype=np.float64)
    return (4.0 / h**2) * np.sin(np.pi * k / (2.0 * N)) ** 2


def sine_matrix(n: int) -> np.ndarray:
    """Explicit orthonormal DST-I matrix F_l (Section 3.2, A_(l) = F* Lambda F)."""
    N = n + 1
    j = np.arange(1, n + 1, dtype=np.float64)
    return np.sqrt(2.0 / N) * np.sin(np.pi * np.outer(j, j) / N)


def dst1(X: np.ndarray, axis: int = 0) -> np.ndarray:
    """Orthonormal DST-I along ``axis`` (library FFT; same map as sine_matrix)."""
    return scipy.fft.dst(X, type=1, axis=axis, norm="ortho")
