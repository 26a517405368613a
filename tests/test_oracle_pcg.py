"""Pins of the oracle's Algorithm 1 (low-rank PCG, Section 3.3) against the full-format
solve and manufactured sine-mode solutions."""
import math

import numpy as np
import pytest

import fc_inputs as fi
from oracle import cp, full, pcg, quadrature as q


def _solve(prob, eps, tol, max_rank, rpc=12):
    fs = q.control_symbol(prob.n, prob.d, prob.alpha, prob.beta, prob.gamma, 1e-10)
    ps = q.precond_symbol(prob.n, prob.d, prob.alpha, prob.beta, prob.gamma, rpc)
    return fs, pcg.pcg(fs, ps, prob.rhs(), eps, tol, max_rank)


@pytest.mark.parametrize("modes,alpha,gamma_", [((1, 2, 3), 0.5, 1e-3), ((3, 1), 0.25, 1e-1)])
def test_sine_mode_is_solved_exactly(modes, alpha, gamma_):
    n = 31
    y = fi.sine_cp(n, modes)
    prob = fi.Problem(n, len(modes), alpha, 1.0, gamma_, y)
    fs, res = _solve(prob, 1e-10, 1e-10, 16)
    assert res.status == "ok"
    x = fi.grid(n)
    lam = [(2 * (n + 1)) ** 2 * math.sin(math.pi * m / (2 * (n + 1))) ** 2 for m in modes]
    rho = sum(lam)
    g = rho ** (-alpha) + gamma_ * rho**alpha
    ref = cp.to_full(y) / g
    err = np.linalg.norm(cp.to_full(res.X) - ref) / np.linalg.norm(ref)
    assert err < 1e-8
    del x


def test_config1_2d_matches_full_solution():
    prob = fi.config1()
    fs, res = _solve(prob, prob.eps, prob.tol, 64)
    assert res.status == "ok" and res.iters <= 10
    u = full.solve_full(cp.to_full(prob.rhs()), prob.alpha, prob.beta, prob.gamma)
    err = np.linalg.norm(cp.to_full(res.X) - u) / np.linalg.norm(u)
    assert err < 1e-7
    assert pcg.true_relres(fs, prob.rhs(), res.X) < 1e-7


def test_small_3d_gaussians_match_full_solution():
    rng = np.random.default_rng(fi.seed_for(9))
    y = fi.gaussians_cp(23, 3, 3, rng)
    prob = fi.Problem(23, 3, 0.5, 1.0, 1e-2, y)
    fs, res = _solve(prob, 1e-9, 1e-9, 512)
    u = full.solve_full(cp.to_full(prob.rhs()), prob.alpha, prob.beta, prob.gamma)
    err = np.linalg.norm(cp.to_full(res.X) - u) / np.linalg.norm(u)
    assert res.status == "ok"
    assert err < 1e-6


def test_residual_history_and_zero_rhs():
    prob = fi.config1()
    _, res = _solve(prob, 1e-8, 1e-8, 64)
    assert res.history[-1] <= 1e-8 < res.history[0]
    zero = fi.Problem(15, 2, 0.5, 1.0, 1e-2, (np.zeros(1), [np.ones((15, 1))] * 2))
    _, r0 = _solve(zero, 1e-8, 1e-8, 8)
    assert r0.iters == 0 and len(r0.X[0]) == 0
