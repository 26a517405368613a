"""Pins of the oracle's full-format solve (Section 3.2, eqn:DiagFLaplace3D) against brute
force by dense eigendecomposition (spectral definition of A^alpha, Section 2) and against
manufactured sine-mode solutions."""
import math

import numpy as np
import pytest

from oracle import full


@pytest.mark.parametrize("ns", [(5, 7), (4, 3, 5), (8, 8)])
@pytest.mark.parametrize("alpha,beta,gamma_", [(0.5, 1.0, 1e-2), (0.25, 2.0, 1e-1), (1.0, 1.0, 1e-3)])
def test_full_solve_matches_brute_force(ns, alpha, beta, gamma_):
    rng = np.random.default_rng(sum(ns))
    b = rng.standard_normal(ns)
    u = full.solve_full(b, alpha, beta, gamma_)
    ub = full.brute_force_solve(b, alpha, beta, gamma_)
    assert np.linalg.norm(u - ub) <= 1e-12 * np.linalg.norm(ub)


def test_dense_laplacian_is_kronecker_sum_of_5_point_stencil():
    """A acts as the 5-point stencil / h^2 on the interior grid (Section 3.2)."""
    n = 6
    h = 1.0 / (n + 1)
    rng = np.random.default_rng(0)
    x = rng.standard_normal((n, n))
    A = full.dense_laplacian([n, n])
    y = (A @ x.reshape(-1)).reshape(n, n)
    xp = np.pad(x, 1)
    st = (4 * xp[1:-1, 1:-1] - xp[:-2, 1:-1] - xp[2:, 1:-1] - xp[1:-1, :-2] - xp[1:-1, 2:]) / h**2
    assert np.allclose(y, st, rtol=0, atol=1e-9 * np.abs(st).max())


@pytest.mark.parametrize("modes", [(1, 2, 3), (5, 1, 7), (2, 2)])
def test_manufactured_sine_mode(modes):
    """A sampled product of sines is an eigenvector of A with eigenvalue sum_l lambda_{m_l}."""
    n = 31
    d = len(modes)
    x = np.arange(1, n + 1) / (n + 1)
    b = np.ones([n] * d)
    for l, m in enumerate(modes):
        shape = [1] * d
        shape[l] = n
        b = b * np.sin(math.pi * m * x).reshape(shape)
    A = None  # eigenvalue from the stencil, not from the closed form
    v = np.sin(math.pi * np.arange(1, n + 1)[:, None] * x[None, :])
    rho = 0.0
    for m in modes:
        vm = np.sin(math.pi * m * x)
        lap = (2 * vm - np.concatenate([[0], vm[:-1]]) - np.concatenate([vm[1:], [0]])) * (n + 1) ** 2
        rho += lap[0] / vm[0]
    alpha, beta, gamma_ = 0.5, 1.5, 1e-2
    g = beta**2 * rho ** (-alpha) + gamma_ * rho**alpha
    u = full.solve_full(b, alpha, beta, gamma_)
    assert np.linalg.norm(u - b / g) <= 1e-12 * np.linalg.norm(b / g)
    del A, v


def test_apply_then_solve_is_identity():
    rng = np.random.default_rng(3)
    b = rng.standard_normal((9, 10, 11))
    u = full.solve_full(b, 0.3, 1.0, 1e-2)
    assert np.linalg.norm(full.apply_full(u, 0.3, 1.0, 1e-2) - b) <= 1e-12 * np.linalg.norm(b)


@pytest.mark.parametrize("ns,alpha", [((6, 5), 0.5), ((4, 3, 5), 0.3), ((5, 5, 4), 1.0)])
def test_directional_solve_matches_dense(ns, alpha):
    """Directionally fractional Laplacian (Remark after Lemma 4.1): the eigenbasis solve equals
    a dense solve with sum_l I x A_(l)^alpha x I built from 1D eigendecompositions; at alpha = 1
    it coincides with the plain Laplacian operator beta^2 A^-1 + gamma A."""
    rng = np.random.default_rng(3)
    b = rng.standard_normal(ns)
    beta, gamma_ = 1.3, 2e-2
    Ad = full.dense_directional(ns, alpha)
    M = beta**2 * np.linalg.inv(Ad) + gamma_ * Ad
    ref = np.linalg.solve(M, b.reshape(-1)).reshape(ns)
    got = full.solve_full_directional(b, alpha, beta, gamma_)
    assert np.linalg.norm(got - ref) <= 1e-11 * np.linalg.norm(ref)
    if alpha == 1.0:
        plain = full.solve_full(b, 1.0, beta, gamma_)
        assert np.linalg.norm(got - plain) <= 1e-12 * np.linalg.norm(plain)


def test_state_is_beta_A_minus_alpha_u():
    """eqn:State: y = beta A^-alpha u against the dense spectral definition A^-alpha."""
    ns = (5, 4, 3)
    rng = np.random.default_rng(4)
    u = rng.standard_normal(ns)
    alpha, beta = 0.4, 1.7
    Am = full.brute_force_power(ns, -alpha)
    ref = beta * (Am @ u.reshape(-1)).reshape(ns)
    assert np.linalg.norm(full.state_full(u, alpha, beta) - ref) <= 1e-11 * np.linalg.norm(ref)


@pytest.mark.parametrize("kind,alpha", [(1, 0.5), (1, 0.1), (2, 0.5), (2, 0.1), (0, 0.5)])
@pytest.mark.parametrize("ns", [(9, 11), (5, 6, 7)])
def test_test_operators_match_brute_force(kind, alpha, ns):
    """Section 6 test operators A^alpha, I + A^(2 alpha) (and A^alpha + A^-alpha = the control
    operator at beta = gamma = 1): eigenbasis solve vs a dense eigendecomposition solve."""
    rng = np.random.default_rng(300 + kind + len(ns))
    b = rng.standard_normal(ns)
    u = full.solve_full_op(b, kind, alpha)
    ref = full.brute_force_op(b, kind, alpha)
    assert np.linalg.norm(u - ref) <= 1e-12 * np.linalg.norm(ref)


def test_test_operator_symbols_special_cases():
    """Closed forms: A^alpha at alpha = 1 is A itself (the 5-point Laplacian: rho = sum of the
    eigenvalues); I + A^(2 alpha) at alpha = 1/2 is I + A; kind 0 at beta = gamma = 1 is
    rho^alpha + rho^-alpha."""
    rho = np.array([3.0, 10.0, 1e4])
    assert np.allclose(full.g_operator(rho, 1, 1.0), rho, rtol=1e-15)
    assert np.allclose(full.g_operator(rho, 2, 0.5), 1.0 + rho, rtol=1e-15)
    assert np.allclose(full.g_operator(rho, 0, 0.3), rho**0.3 + rho**-0.3, rtol=1e-15)
    # dense check: kind 1 at alpha = 1 solves with A itself
    rng = np.random.default_rng(301)
    b = rng.standard_normal((6, 7))
    A = full.dense_laplacian(b.shape)
    assert np.allclose(full.solve_full_op(b, 1, 1.0).reshape(-1), np.linalg.solve(A, b.reshape(-1)),
                       rtol=1e-11, atol=1e-14)


def _coef(n, kind):
    x = (np.arange(n + 1) + 0.5) / (n + 1)
    return {0: 1.0 + 0.5 * np.sin(2 * np.pi * x), 1: np.exp(x), 2: 0.3 + x**2}[kind]


def test_stiffness_with_unit_coefficient_is_the_laplacian():
    for n in (1, 4, 9):
        assert np.allclose(full.stiffness_1d(n, np.ones(n + 1)), full.laplacian_1d(n), rtol=1e-15)


@pytest.mark.parametrize("ns,kinds", [((9, 11), (0, 1)), ((5, 6, 7), (0, None, 2)),
                                      ((6, 5, 4), (1, 2, 0))])
@pytest.mark.parametrize("op", [(0, 0.5, 1.0, 1e-2), (1, 0.3, 1.0, 1.0), (2, 0.5, 1.0, 1.0)])
def test_varcoef_solve_matches_brute_force(ns, kinds, op):
    """Separable variable coefficients: per-mode eigenbasis solve vs the dense operator from
    the eigendecomposition of the assembled Kronecker sum."""
    kind, alpha, beta, gamma_ = op
    coeffs = [None if k is None else _coef(n, k) for n, k in zip(ns, kinds)]
    rng = np.random.default_rng(400 + len(ns) + kind)
    b = rng.standard_normal(ns)
    u = full.solve_full_varcoef(b, coeffs, kind, alpha, beta, gamma_)
    ref = full.brute_force_varcoef(b, coeffs, kind, alpha, beta, gamma_)
    assert np.linalg.norm(u - ref) <= 1e-11 * np.linalg.norm(ref)


def test_varcoef_with_constant_coefficients_reduces_to_the_laplacian():
    rng = np.random.default_rng(402)
    b = rng.standard_normal((8, 9, 7))
    u = full.solve_full_varcoef(b, [np.ones(9), None, np.ones(8)], 0, 0.5, 1.0, 1e-2)
    assert np.linalg.norm(u - full.solve_full(b, 0.5, 1.0, 1e-2)) <= 1e-12 * np.linalg.norm(u)
