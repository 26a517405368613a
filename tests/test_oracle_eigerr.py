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
