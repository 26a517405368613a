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


def test_3d_error_within_tolerance():
    """Smooth 3D tensor: error <= eps * ||T||; unit columns, positive sorted weights."""
    X = fi.gaussians_cp(40, 3, 8, np.random.default_rng(11))
    Xf = cp.to_full(X)
    for eps in (1e-4, 1e-7):
        info = {}
        T = truncate(X, eps, 1024, info)
        err = np.linalg.norm(cp.to_full(T) - Xf) / np.linalg.norm(Xf)
        assert err <= eps
        assert info["est_err"] >= 0.0
    T = truncate(X, 1e-6, 1024)
    for u in T[1]:
        assert np.allclose(np.linalg.norm(u, axis=0), 1.0)
    assert np.all(np.diff(T[0]) <= 0) and np.all(T[0] > 0)


def _hosvd_bases(F, ranks):
    """HOSVD of a full tensor: leading left singular vectors of each mode unfolding."""
    out = []
    for l, r in enumerate(ranks):
        M = np.moveaxis(F, l, 0).reshape(F.shape[l], -1)
        Ul, _, _ = np.linalg.svd(M, full_matrices=False)
        out.append(Ul[:, :r])
    return out


def _project(F, bases):
    """F x_1 P_1 x_2 P_2 x_3 P_3 with the orthogonal projectors P_l = Z_l Z_l^T."""
    G = F
    for l, Z in enumerate(bases):
        G = np.moveaxis(np.tensordot(Z @ Z.T, np.moveaxis(G, l, 0), axes=(1, 0)), 0, l)
    return G


def test_3d_orthogonal_factors_reduce_to_hosvd():
    """With orthonormal factor columns in every mode the side matrix U_l diag(xi) carries the
    singular vectors of the mode-l unfolding, so RHOSVD (Section 5) is the HOSVD: the same
    Tucker subspaces, and the truncation keeps exactly the largest terms."""
    rng = np.random.default_rng(21)
    n, R = 14, 6
    xi = np.array([9.0, -5.0, 3.0, 2.0, -1.0, 0.5])
    U = [np.linalg.qr(rng.standard_normal((n, R)))[0] for _ in range(3)]
    F = cp.to_full((xi, U))
    info = {}
    eps = 1.6 / np.linalg.norm(xi)       # stage-1 budget 1.6/sqrt(6) drops the smallest term
    T = truncate((xi, U), eps, 64, info)
    r = info["ranks"]
    for Z, H in zip(info["bases"], _hosvd_bases(F, r)):
        assert np.linalg.norm(Z @ Z.T - H @ H.T) <= 1e-12
    keep = np.argsort(-np.abs(xi))[:len(T[0])]
    ref = cp.to_full((xi[keep], [u[:, keep] for u in U]))
    assert np.linalg.norm(cp.to_full(T) - ref) <= 1e-12 * np.linalg.norm(F)
    assert min(r) < R


@pytest.mark.parametrize("seed,count", [(11, 40), (12, 60)])
def test_3d_tucker_stage_against_hosvd(seed, count):
    """Stage 1 against the HOSVD of the full tensor at the same Tucker ranks (Section 5).
    No Tucker approximation of those ranks beats the optimum, which is at least the HOSVD
    error / sqrt(d); and the RHOSVD error obeys its a-priori bound: projecting mode l costs
    at most ||(I - Z_l Z_l^T) W_l||_F ||M_l||_2, M_l the Khatri-Rao product of the other
    modes' unit factors (so sum over modes of tail_l ||M_l||_2)."""
    X = fi.gaussians_cp(40, 3, count, np.random.default_rng(seed))
    F = cp.to_full(X)
    xi, U = X[0], [u / np.linalg.norm(u, axis=0) for u in X[1]]
    for eps in (1e-2, 1e-4, 1e-6):
        info = {}
        truncate(X, eps, 4096, info)
        e1 = np.linalg.norm(_project(F, info["bases"]) - F)
        eh = np.linalg.norm(_project(F, _hosvd_bases(F, info["ranks"])) - F)
        bound = 0.0
        for l in range(3):
            a, b = [U[m] for m in range(3) if m != l]
            G = (a.T @ a) * (b.T @ b)
            bound += info["stage1_tails"][l] * np.sqrt(np.linalg.eigvalsh(G).max())
        assert eh / np.sqrt(3) <= e1 * (1 + 1e-12)
        assert e1 <= bound * (1 + 1e-12)
        assert e1 <= 10 * eh           # measured 2.4x to 8x on these tensors


def test_3d_core_to_canonical_error_is_the_dropped_energy():
    """Stage 2 (eqn:two_level): the canonical terms from the mode-3 rotation and the slice
    SVDs are mutually orthogonal, so keeping q of them leaves exactly the energy of the
    rest.  With stage 1 exact (eps = 0, Tucker ranks = CP rank) the whole error is that."""
    X = fi.random_cp(10, 3, 6, seed=14)
    F = cp.to_full(X)
    for q in (3, 10, 20):
        info = {}
        T = truncate(X, 0.0, q, info)
        err = np.linalg.norm(cp.to_full(T) - F)
        dropped = np.sqrt(np.sum(np.asarray(info["sigma"])[q:] ** 2))
        assert abs(err - dropped) <= 1e-12 * np.linalg.norm(F)
        assert info["stage1_tails"] == [0.0, 0.0, 0.0] or max(info["stage1_tails"]) < 1e-12


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
