"""Pins of the oracle's 1D spectrum and sine transform (Section 3.2)."""
import os

import numpy as np
import pytest

from oracle import spectrum

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "eigs_small.txt")


def test_hand_derived_eigenvalues():
    rows = np.loadtxt(GOLDEN)
    for n, k, lam in rows:
        got = spectrum.eigenvalues(int(n))[int(k) - 1]
        assert abs(got - lam) <= 1e-13 * lam


@pytest.mark.parametrize("n", [1, 2, 5, 16, 63, 255])
def test_eigenvalues_match_dense_eigh(n):
    A = spectrum.laplacian_1d(n)
    w = np.linalg.eigvalsh(A)
    lam = spectrum.eigenvalues(n)
    assert np.all(np.diff(lam) > 0)
    assert np.max(np.abs(w - lam)) <= 1e-12 * lam[-1]


@pytest.mark.parametrize("n", [3, 16, 63, 64])
def test_sine_matrix_is_symmetric_orthogonal_eigenbasis(n):
    F = spectrum.sine_matrix(n)
    A = spectrum.laplacian_1d(n)
    assert np.allclose(F, F.T, atol=0)
    assert np.max(np.abs(F @ F - np.eye(n))) < 1e-13
    L = F @ A @ F
    lam = spectrum.eigenvalues(n)
    assert np.max(np.abs(L - np.diag(lam))) < 1e-12 * lam[-1]


@pytest.mark.parametrize("n", [1, 7, 63, 100])
def test_fft_dst_equals_sine_matrix(n):
    rng = np.random.default_rng(n)
    X = rng.standard_normal((n, 5))
    assert np.allclose(spectrum.dst1(X, axis=0), spectrum.sine_matrix(n) @ X, rtol=0, atol=1e-13)
