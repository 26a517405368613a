"""Pins of the oracle's whole-grid error evaluator (oracle/eigerr.py, csrc/eigerr.c):
the exact solution of eqn:DiagFLaplace3D / 2D taken point by point on the eigen-index grid."""
import math

import numpy as np
import pytest

import fc_inputs as fi
from oracle import cp, eigerr, full


@pytest.mark.parametrize("d,n", [(2, 20), (3, 12), (3, 17)])
def test_matches_dense_full_format_solve(d, n):
    """Same relative error as the dense n^d solve (d DST passes, division, d passes)."""
    rng = np.random.default_rng(31 + n)
    b = fi.gaussians_cp(n, d, 3, rng)
    ustar = full.solve_full(cp.to_full(b), 0.5, 1.0, 1e-2)
    u = fi.random_cp(n, d, 5, seed=4 + n)
    ref = np.linalg.norm(cp.to_full(u) - ustar) / np.linalg.norm(ustar)
    got, nrm = eigerr.control_error(u, b, 0.5, 1.0, 1e-2)
    assert abs(got - ref) <= 1e-13 * ref
    assert abs(nrm - np.linalg.norm(ustar)) <= 1e-13 * nrm


@pytest.mark.parametrize("eta", [1e-3, 1e-9])
def test_sine_mode_relative_error_is_exact(eta):
    """b = sin(pi x) sin(2 pi y) sin(3 pi z) has u* = b / g(rho_m) in closed form; a solution
    scaled by (1 + eta) is exactly eta away, whatever the grid size."""
    n, alpha, beta, gamma_ = 63, 0.75, 1.3, 1e-3
    b = fi.sine_cp(n, (1, 2, 3))
    lam = [(2 * (n + 1)) ** 2 * math.sin(math.pi * m / (2 * (n + 1))) ** 2 for m in (1, 2, 3)]
    rho = sum(lam)
    g = beta**2 * rho ** (-alpha) + gamma_ * rho**alpha
    u = (np.array([(1 + eta) / g]), b[1])
    got, nrm = eigerr.control_error(u, b, alpha, beta, gamma_)
    assert abs(got / eta - 1) < 1e-6
    assert abs(nrm / (np.linalg.norm(cp.to_full(b)) / g) - 1) < 1e-12


def test_general_symbol_and_zero_solution():
    """g = rho^alpha (the test operator A^alpha of Section 6); u = 0 has relative error 1."""
    n, d, alpha = 14, 3, 0.4
    b = fi.random_cp(n, d, 2, seed=99)
    s = eigerr.error_sums((np.zeros(0), [np.zeros((n, 0))] * d), b, 0.0, alpha, 1.0, alpha)
    ustar = full.apply_g_full(cp.to_full(b), lambda r: r ** (-alpha))
    assert abs(s[0] / s[1] - 1) < 1e-14 and s[2] == 0.0
    assert abs(math.sqrt(s[1]) / np.linalg.norm(ustar) - 1) < 1e-13


def _oracle_solution(n, d, alpha, gamma_, seed, eps):
    from oracle import pcg, quadrature as q
    b = fi.gaussians_cp(n, d, 3, np.random.default_rng(seed))
    fs = q.control_symbol(n, d, alpha, 1.0, gamma_, 1e-10)
    ps = q.precond_symbol(n, d, alpha, 1.0, gamma_, 12)
    return b, pcg.pcg(fs, ps, b, eps, eps, 64).X


@pytest.mark.parametrize("eps", [1e-5, 1e-8])
def test_box_sum_matches_whole_grid(eps):
    """The low-index box with the CP-form remainder gives the whole-grid error of a real
    solution (oracle CP-PCG) to the resolution of the remainder (~1e-8 relative)."""
    b, X = _oracle_solution(47, 3, 0.5, 1e-3, 77, eps)
    e_full, n_full = eigerr.control_error(X, b, 0.5, 1.0, 1e-3)
    e_box, n_box = eigerr.control_error(X, b, 0.5, 1.0, 1e-3, force_box=True)
    assert e_full < 1e-3
    assert abs(e_box - e_full) <= 2e-8 + 1e-6 * e_full
    assert e_box >= e_full * (1 - 1e-9)          # the box result is the upper end
    assert abs(n_box / n_full - 1) < 1e-12


@pytest.mark.parametrize("alpha", [0.25, 0.75])
def test_box_sum_on_the_8191_grid_sine_mixture(alpha):
    """n = 8191 (5.5e11 points): a mixture of grid sine modes has its solution in closed form
    (each mode divided by g at its eigenvalue); a solution with mode-wise relative errors
    eta_m is eta-weighted away, and the box holds exactly the modes' indices."""
    n, gamma_ = 8191, 1e-4
    modes = [(1, 2, 3), (5, 1, 2), (40, 33, 7)]
    amps = np.array([1.0, -0.5, 0.25])
    etas = np.array([1e-7, -3e-7, 2e-6])
    x = fi.grid(n)
    U = [np.stack([np.sin(math.pi * m[l] * x) for m in modes], axis=1) for l in range(3)]
    lam1 = lambda k: (2 * (n + 1)) ** 2 * math.sin(math.pi * k / (2 * (n + 1))) ** 2
    g = np.array([sum(lam1(k) for k in m) ** -alpha + gamma_ * sum(lam1(k) for k in m) ** alpha
                  for m in modes])
    u = (amps * (1 + etas) / g, U)
    got, _ = eigerr.control_error(u, (amps, U), alpha, 1.0, gamma_)
    ref = np.sqrt(np.sum((amps * etas / g) ** 2) / np.sum((amps / g) ** 2))
    assert abs(got / ref - 1) < 1e-6
