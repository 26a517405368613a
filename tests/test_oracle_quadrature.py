"""Pins of the oracle's sinc-quadrature symbols (Sections 2, 4.1-4.2, Lemma 4.1)."""
import math

import numpy as np
import pytest
from scipy.special import gamma as Gamma

from oracle import quadrature as q
from oracle import spectrum


@pytest.mark.parametrize("s", [0.1, 0.25, 0.5, 0.75, 0.9])
def test_exp_sum_relative_error(s):
    """The plain trapezoidal rule reaches delta on [1, B], checked on a grid other than the
    one its step search uses (4001 points, and both ends)."""
    B = 3.0 * (2 * 256 / math.pi) ** 2
    t, c = q.exp_sum(s, B, 1e-10)
    rho = np.concatenate([[1.0, B], np.exp(np.linspace(0.0, math.log(B), 4001))])
    approx = np.exp(-np.outer(rho, t)) @ c
    rel = np.abs(approx * rho**s - 1.0)
    assert rel.max() <= 1e-10
    assert np.all(c > 0) and np.all(t > 0)


def test_exp_sum_error_decays_with_delta():
    """Bound (ff6) of Section 4.2: the error falls exponentially as the step shrinks and the
    range grows, and the node count grows with log(1/delta)."""
    B = 1e5
    rho = np.exp(np.linspace(0.0, math.log(B), 2001))
    errs, ranks = [], []
    for delta in (1e-4, 1e-6, 1e-8, 1e-10):
        t, c = q.exp_sum(0.5, B, delta)
        errs.append(np.max(np.abs((np.exp(-np.outer(rho, t)) @ c) * rho**0.5 - 1)))
        ranks.append(len(t))
    assert all(e2 < e1 for e1, e2 in zip(errs, errs[1:]))
    assert errs[-1] < 1e-10
    assert all(r2 > r1 for r1, r2 in zip(ranks, ranks[1:]))


@pytest.mark.parametrize("s", [0.1, 0.5, 0.9])
def test_tail_cuts_by_direct_integration(s):
    """The truncation points cut off delta/4 of the Laplace integral at the ends of [1, B]:
    checked by adaptive quadrature of t^(s-1) e^(-rho t) / Gamma(s) itself."""
    from scipy.integrate import quad
    B, delta = 1e6, 1e-10
    t_lo, t_hi = q.tail_cuts(s, B, delta)
    hi, _ = quad(lambda t: t ** (s - 1) * math.exp(-t), t_hi, np.inf, epsabs=0, epsrel=1e-12)
    # int_0^t_lo t^(s-1) e^(-B t) dt = t_lo^s / s (1 - O(B t_lo)), relative to B^-s Gamma(s)
    lo, _ = quad(lambda x: x ** (s - 1) * math.exp(-B * x), 0.0, t_lo, epsabs=0, epsrel=1e-10)
    assert abs(hi / Gamma(s) / (delta / 4) - 1) < 1e-6
    assert abs(lo * B**s / Gamma(s) / (delta / 4) - 1) < 1e-6


def test_rule_is_the_trapezoid_of_the_substituted_integrand():
    """Every node is kept: the rule's sum at rho equals h sum_k f(k h) with the integrand
    f(u) = log(1+e^u)^(s-1) e^(-rho log(1+e^u)) / (1 + e^-u) / Gamma(s) of Section 4.2,
    summed term by term over the same range of k."""
    s, B, delta, h = 0.4, 1e4, 1e-8, 0.37
    t, c = q.trapezoid_rule(s, B, delta, h)
    t_lo, t_hi = q.tail_cuts(s, B, delta)
    k0 = math.floor(math.log(math.expm1(t_lo)) / h)
    k1 = math.ceil(math.log(math.expm1(t_hi)) / h)
    assert len(t) == k1 - k0 + 1
    for rho in (1.0, 37.0, B):
        acc = 0.0
        for k in range(k0, k1 + 1):
            u = k * h
            ph = math.log1p(math.exp(u)) if u < 30 else u + math.log1p(math.exp(-u))
            acc += h * ph ** (s - 1) * math.exp(-rho * ph) / (1.0 + math.exp(-u)) / Gamma(s)
        assert abs(np.sum(c * np.exp(-t * rho)) - acc) <= 1e-13 * acc


def test_laplace_transform_identity_direct():
    """rho^-s = Gamma(s)^-1 int t^(s-1) e^(-rho t) dt (Section 2) by scipy quadrature."""
    from scipy.integrate import quad
    for s in (0.3, 0.7):
        for rho in (1.0, 10.0):
            val, _ = quad(lambda u: math.exp(s * u - rho * math.exp(u)), -200, 10, limit=400,
                          epsabs=0, epsrel=1e-13)
            assert abs(val / Gamma(s) - rho ** (-s)) < 1e-10 * rho ** (-s)


def _all_rho(n, d):
    lam = spectrum.eigenvalues(n)
    out = lam
    for _ in range(d - 1):
        out = np.add.outer(out, lam)
    return out


@pytest.mark.parametrize("alpha,gamma_", [(0.5, 1e-2), (0.25, 1e-1), (0.75, 1e-3), (1.0, 1e-2)])
def test_control_symbol_on_all_grid_points_2d(alpha, gamma_):
    n, d, beta = 63, 2, 1.0
    sym = q.control_symbol(n, d, alpha, beta, gamma_, 1e-10)
    full = q.symbol_full(sym)
    rho = _all_rho(n, d)
    exact = beta**2 * rho ** (-alpha) + gamma_ * rho**alpha
    assert np.max(np.abs(full / exact - 1)) < 1e-9


def test_control_symbol_3d_and_rank_structure():
    n, d = 31, 3
    sym = q.control_symbol(n, d, 0.5, 2.0, 1e-3, 1e-10)
    full = q.symbol_full(sym)
    rho = _all_rho(n, d)
    exact = 4.0 * rho ** (-0.5) + 1e-3 * rho**0.5
    assert np.max(np.abs(full / exact - 1)) < 1e-9
    # Lemma 4.1: R_A = R_- + d R_+
    B = rho.max() / rho.min()
    Rm = len(q.exp_sum(0.5, B, 1e-10)[0])
    Rp = len(q.exp_sum(0.5, B, 1e-10)[0])
    assert len(sym.xi) == Rm + d * Rp
    for u in sym.U:
        assert np.allclose(np.linalg.norm(u, axis=0), 1.0)


def test_power_symbol_matches_brute_force_power():
    from oracle import full as fullmod
    n, d, s = 6, 2, 0.5
    sym = q.power_symbol(n, d, s, 1e-10)
    G = q.symbol_full(sym)
    F = spectrum.sine_matrix(n)
    # dense operator F (x) F diag(G) F (x) F against A^-s by dense eigh
    FF = np.kron(F, F)
    Op = FF @ np.diag(G.reshape(-1)) @ FF
    Ref = fullmod.brute_force_power([n, n], -s)
    assert np.max(np.abs(Op - Ref)) < 1e-9 * np.max(np.abs(Ref))


@pytest.mark.parametrize("alpha,gamma_", [(0.5, 1e-2), (0.25, 1e-1), (0.75, 1e-3)])
def test_precond_fit_positive_and_close(alpha, gamma_):
    n, d = 63, 3
    sym = q.precond_symbol(n, d, alpha, 1.0, gamma_, 12)
    full = q.symbol_full(sym)
    rr = _all_rho(n, d)
    g = 1.0 * rr ** (-alpha) + gamma_ * rr**alpha
    assert np.all(full > 0)
    assert np.max(np.abs(full * g - 1)) <= 0.5
