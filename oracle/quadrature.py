"""Separable (CP) symbols by sinc quadrature of the Laplace transform.

Paper Section 2 (eqn:Laplace_transf, eqn:sinc_Laplace_tr), Section 4.2
(eqn:Sinc_quadr_trunc, eqn:Func_of_rho, eqn:Laplace_transf_rhom1) and
Lemma 4.1 (lem:Rank_positive_power).

For s > 0 and rho > 0 the Laplace transform gives

    rho^-s = Gamma(s)^-1 int_0^inf t^(s-1) exp(-rho t) dt .

With rho = sum_l lambda_{i_l} every exponential factorises over the modes,
exp(-t rho) = prod_l exp(-t lambda_{i_l}), so a quadrature sum
sum_k c_k exp(-t_k rho) is a CP tensor of rank = number of nodes
(eqn:Func_of_rho).

The rule is the paper's, kept plain (every node of the truncated trapezoidal
sum is a term of the symbol; nothing is merged or compressed):
  * Substitution t = phi(u) = log(1 + e^u) (Section 4.2), so that
    rho^-s = Gamma(s)^-1 int_R phi(u)^(s-1) phi'(u) exp(-rho phi(u)) du,
    phi'(u) = 1/(1 + e^-u).
  * Scaling: rho is scaled to [1, B] by rho_min (eqn:Laplace_transf_rhom1).
  * Trapezoidal sinc sum (eqn:Sinc_quadr_trunc) with nodes u_k = k h,
    k = -M_- .. M_+, t_k = phi(u_k), c_k = h phi(u_k)^(s-1) phi'(u_k) / Gamma(s).

Readings where the paper leaves the parameters open (it writes
h = kappa pi / sqrt(M) with unspecified kappa, M and a symmetric range):
  * Truncation.  The integral cut at u = U, transformed back to t, is an
    incomplete gamma function: the part of rho^-s beyond t_hi = phi(U) is
    rho^-s Q(s, rho t_hi) and the part below t_lo is rho^-s P(s, rho t_lo)
    (P, Q the regularised lower / upper incomplete gamma).  Over rho in [1, B]
    the first is largest at rho = 1 and the second at rho = B, so
    Q(s, t_hi) = delta/4 and P(s, B t_lo) = delta/4 fix both ends exactly:
    M_- and M_+ need not be equal.
  * Step.  h starts at 1 and shrinks by a factor 0.9 until the rule's largest
    relative error on 3001 geometric points of [1, B] is <= delta; the
    trapezoidal error decays like exp(-pi^2 / h) (the integrand is analytic
    in the strip |Im u| < pi/2), bound (ff6).
  * Positive power.  gamma rho^alpha = gamma rho * rho^(alpha-1) (Lemma 4.1):
    each node of the rho^(alpha-1) sum yields d rank-one terms whose mode-m
    factor is lambda * exp(-t lambda).  At alpha = 1 the term is exactly
    gamma * sum_m lambda_{i_m} (rank d).
  * Preconditioner.  The paper precomputes a rank-r CP of 1/g by multigrid
    Tucker on the full n^d tensor (Section 5), infeasible at large n.  We fit
    p(rho) = sum_k w_k exp(-tau_k rho) with R_pc fixed geometric nodes
    tau_k in [0.2/rho_max, 20/rho_min] by linear least squares of p*g - 1 on a
    geometric grid of 3000 points in [rho_min, rho_max] (columns scaled to unit
    norm).  The fit is unique (full column rank) and is checked for p > 0.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np
from scipy.special import gammaincinv, gammainccinv, gammaln

from .spectrum import eigenvalues


def phi(u):
    """t = phi(u) = log(1 + e^u) (the substitution of Section 4.2)."""
    return np.logaddexp(0.0, u)


def phi_inverse(t: float) -> float:
    """u with phi(u) = t: log(e^t - 1)."""
    return math.log(math.expm1(t))


def tail_cuts(s: float, B: float, delta: float):
    """(t_lo, t_hi): the parts of the Laplace integral below t_lo and above t_hi are at
    most delta/4 of rho^-s for every rho in [1, B] (incomplete gamma functions)."""
    t_hi = float(gammainccinv(s, delta / 4.0))
    t_lo = float(gammaincinv(s, delta / 4.0)) / B
    return t_lo, t_hi


def trapezoid_rule(s: float, B: float, delta: float, h: float):
    """Nodes t_k and weights c_k of the truncated trapezoidal sum with step h
    (eqn:Sinc_quadr_trunc with the substitution t = phi(u))."""
    t_lo, t_hi = tail_cuts(s, B, delta)
    k = np.arange(math.floor(phi_inverse(t_lo) / h), math.ceil(phi_inverse(t_hi) / h) + 1)
    u = k * h
    t = phi(u)
    # c_k = h t_k^(s-1) phi'(u_k) / Gamma(s), formed in logarithms (t_k spans many decades)
    logc = math.log(h) + (s - 1.0) * np.log(t) - np.logaddexp(0.0, -u) - gammaln(s)
    return t, np.exp(logc)


def rule_error(s: float, B: float, t: np.ndarray, c: np.ndarray, points: int = 3001) -> float:
    """Largest relative error of sum_k c_k exp(-t_k rho) against rho^-s on a geometric grid
    of [1, B]."""
    rho = np.exp(np.linspace(0.0, math.log(B), points))
    return float(np.max(np.abs((np.exp(-np.outer(rho, t)) @ c) * rho**s - 1.0)))


def exp_sum(s: float, B: float, delta: float = 1e-10):
    """Nodes t_k and weights c_k with rho^-s ~ sum_k c_k exp(-t_k rho) on [1, B] to relative
    accuracy delta (the rule and its readings in the module docstring)."""
    if s <= 0.0:
        raise ValueError("s must be positive")
    h = 1.0
    while True:
        t, c = trapezoid_rule(s, B, delta, h)
        if rule_error(s, B, t, c) <= delta:
            return t, c
        h *= 0.9
        if h < 1e-3:
            raise RuntimeError("sinc rule did not reach the requested accuracy")


def normalise_columns(xi, U):
    """Same CP tensor with unit columns; the weights absorb the norms."""
    xi = np.array(xi, dtype=np.float64)
    out = []
    for u in U:
        c = np.linalg.norm(u, axis=0)
        xi = xi * c
        out.append(u / c)
    return xi, out


@dataclass
class Symbol:
    """CP representation diag(G) = sum_k xi_k (x)_l U_l[:, k] of a function of
    Lambda, with unit columns U_l[:, k] (the weights carry the norms)."""
    xi: np.ndarray
    U: list
    lam: list
    kind: str


def rho_range(lams):
    return sum(l[0] for l in lams), sum(l[-1] for l in lams)


def control_symbol(n, d, alpha, beta, gamma_, delta=1e-10) -> Symbol:
    """CP symbol of beta^2 A^-alpha + gamma A^alpha (eqn:forControl times beta).

    beta^2 rho^-alpha : sinc sum (eqn:Func_of_rho), rank R_-.
    gamma rho^alpha   : gamma rho * rho^(alpha-1), rank d R_+ (Lemma 4.1).
    """
    ns = [n] * d if np.isscalar(n) else list(n)
    lams = [eigenvalues(m) for m in ns]
    rmin, rmax = rho_range(lams)
    B = rmax / rmin
    cols = [[] for _ in range(d)]
    w = []
    tm, cm = exp_sum(alpha, B, delta)
    for t, c in zip(tm, cm):
        for l in range(d):
            cols[l].append(np.exp(-(t / rmin) * lams[l]))
        w.append(beta**2 * c * rmin ** (-alpha))
    if alpha < 1.0:
        tp, cp = exp_sum(1.0 - alpha, B, delta)
        for t, c in zip(tp, cp):
            for m in range(d):
                for l in range(d):
                    v = np.exp(-(t / rmin) * lams[l])
                    if l == m:
                        v = lams[l] * v
                    cols[l].append(v)
                w.append(gamma_ * c * rmin ** (alpha - 1.0))
    else:
        for m in range(d):
            for l in range(d):
                cols[l].append(lams[l].copy() if l == m else np.ones(ns[l]))
            w.append(gamma_)
    xi, U = normalise_columns(np.array(w), [np.array(c).T.copy() for c in cols])
    return Symbol(xi, U, lams, "control")


def power_symbol(n, d, s, delta=1e-10) -> Symbol:
    """CP symbol of A^-s (s > 0), e.g. g_1 = rho^-alpha (eq:3a / eq:2a)."""
    ns = [n] * d if np.isscalar(n) else list(n)
    lams = [eigenvalues(m) for m in ns]
    rmin, rmax = rho_range(lams)
    t, c = exp_sum(s, rmax / rmin, delta)
    xi, U = normalise_columns(c * rmin ** (-s), [np.exp(-np.outer(lams[l], t / rmin)) for l in range(d)])
    return Symbol(xi, U, lams, "power")


def g_control(rho, alpha, beta, gamma_):
    """Exact symbol g(rho) = beta^2 rho^-alpha + gamma rho^alpha."""
    return beta**2 * rho ** (-alpha) + gamma_ * rho**alpha


PC_GRID = 3000
PC_TLO = 0.2
PC_THI = 20.0


def precond_symbol(n, d, alpha, beta, gamma_, rank=12) -> Symbol:
    """Rank-R_pc exponential-sum CP of 1/g (least-squares fit, reading above)."""
    ns = [n] * d if np.isscalar(n) else list(n)
    lams = [eigenvalues(m) for m in ns]
    rmin, rmax = rho_range(lams)
    tau = np.exp(np.linspace(math.log(PC_TLO / rmax), math.log(PC_THI / rmin), rank))
    rho = np.exp(np.linspace(math.log(rmin), math.log(rmax), PC_GRID))
    g = g_control(rho, alpha, beta, gamma_)
    A = g[:, None] * np.exp(-np.outer(rho, tau))
    cn = np.linalg.norm(A, axis=0)
    w, *_ = np.linalg.lstsq(A / cn, np.ones(PC_GRID), rcond=None)
    w = w / cn
    p = np.exp(-np.outer(rho, tau)) @ w
    if not np.all(p > 0):
        raise ValueError("preconditioner fit is not positive on [rho_min, rho_max]")
    xi, U = normalise_columns(w, [np.exp(-np.outer(lams[l], tau)) for l in range(d)])
    return Symbol(xi, U, lams, "precond")


def symbol_full(sym: Symbol) -> np.ndarray:
    """Expand the CP symbol to the full n_1 x ... x n_d tensor."""
    d = len(sym.U)
    out = np.zeros([u.shape[0] for u in sym.U])
    for k in range(len(sym.xi)):
        t = sym.xi[k]
        for l in range(d):
            t = np.multiply.outer(t, sym.U[l][:, k])
        out += t
    return out


def rho_full(lams) -> np.ndarray:
    """rho(i) = sum_l lambda_{i_l} as a full tensor (eqn:DiagLaplace)."""
    out = lams[0]
    for l in range(1, len(lams)):
        out = np.add.outer(out, lams[l])
    return out
