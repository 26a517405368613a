"""Pins of the oracle's RHOSVD truncation (Section 5, eqn:two_level; 2D reduced SVD)."""
import numpy as np
import pytest

import fc_inputs as fi
from oracle import cp
from oracle.truncate import truncate


@pytest.mark.parametrize("d", [2, 3])
def test_exact_when_rank_is_low(d):
    """X + 0*P and duplicated terms: the truncation reproduces the tensor."""
    X = fi.random_cp(12, d, 3, seed=7)
    Y = cp.axpy(X, 0.0, fi.random_cp(12, d, 4, seed=8))
    Y = cp.axpy(Y, 1.0, X)                      # 2X, rank 6 representation of rank 3
    T = truncate(Y, 1e-12, 64)
    assert len(T[0]) <= 3 ** (d - 1) if d == 3 else len(T[0]) <= 3
    ref = 2 * cp.to_full(X)
    assert np.linalg.norm(cp.to_full(T) - ref) <= 1e-12 * np.linalg.norm(ref)


def test_2d_is_optimal_svd_truncation():
    """d = 2: the reduced SVD truncation equals the Eckart-Young best rank-q approximation."""
    X = fi.random_cp(30, 2, 10, seed=9, scale_spread=2.0)
    M = cp.to_full(X)
    for q in (1, 4, 7):
        T = truncate(X, 0.0, q)
        s = np.linalg.svd(M, compute_uv=False)
        err = np.linalg.norm(cp.to_full(T) - M)
        assert abs(err - np.sqrt(np.sum(s[q:] ** 2))) <= 1e-10 * np.linalg.norm(M)


def test_3d_error_within_tolerance_and_against_hosvd():
    """Smooth 3D tensor: error <= eps * ||T||, and not worse than HOSVD of the full tensor
    with the same Tucker ranks by more than the stage-2 budget."""
    X = fi.gaussians_cp(40, 3, 8, np.random.default_rng(11))
    Xf = cp.to_full(X)
    for eps in (1e-4, 1e-7):
        info = {}
        T = truncate(X, eps, 1024, info)
        err = np.linalg.norm(cp.to_full(T) - Xf) / np.linalg.norm(Xf)
        assert err <= eps
        assert info["est_err"] >= 0.0
    # columns of the result are unit vectors, weights positive and sorted
    T = truncate(X, 1e-6, 1024)
    for u in T[1]:
        assert np.allclose(np.linalg.norm(u, axis=0), 1.0)
    assert np.all(np.diff(T[0]) <= 0) and np.all(T[0] > 0)


def test_eps_to_zero_reproduces_input():
    X = fi.random_cp(10, 3, 4, seed=12)
    T = truncate(X, 0.0, 4096)
    assert np.linalg.norm(cp.to_full(T) - cp.to_full(X)) <= 1e-12 * np.linalg.norm(cp.to_full(X))


def test_rank_cap_and_empty():
    X = fi.random_cp(10, 3, 6, seed=13)
    T = truncate(X, 0.0, 5)
    assert len(T[0]) == 5
    E = truncate(cp.empty([10, 10, 10]), 1e-8, 5)
    assert len(E[0]) == 0
