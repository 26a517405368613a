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

Readings where the paper is silent or garbled:
  * Substitution.  The paper substitutes t = log(1+e^u); its right tail then
    decays only like exp(-rho u) and needs about twice the nodes.  We use
    t = e^u (same trapezoidal sinc rule, eqn:Sinc_quadr_trunc, applied to
    rho^-s = Gamma(s)^-1 int_R exp(s u - rho e^u) du), whose right tail decays
    double-exponentially.
  * Scaling.  rho is scaled to [1, B] by rho_s = rho_min (eqn:Laplace_transf_rhom1).
  * Step and truncation.  h = pi^2 / (ln(1/delta) + 3) (the paper's
    h = kappa pi / sqrt(M) leaves kappa, M open); the sum is truncated
    asymmetrically: on the right at the first node whose largest relative
    contribution over rho in [1, B] is below delta/20.
  * Left tail.  Nodes with t_k B < s0 (their exponentials are almost linear on
    [1, B]) form a positive discrete measure; it is replaced by its m-point
    Gauss rule (moments up to degree 2m-1 preserved, error <= s0^(2m)/(2m)!
    relative).  This replaces hundreds of nodes for small s by m.
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
from scipy.special import gamma as Gamma

from .spectrum import eigenvalues


def sinc_step(delta: float) -> float:
    """Trapezoid step h for a target relative accuracy delta."""
    return math.pi**2 / (math.log(1.0 / delta) + 3.0)


def tail_points(delta: float, s0: float) -> int:
    """Smallest m with s0^(2m)/(2m)! <= delta/100 (Gauss-rule remainder)."""
    m = 1
    while s0 ** (2 * m) / math.factorial(2 * m) > delta / 100.0:
        m += 1
    return m


def gauss_rule_discrete(t: np.ndarray, c: np.ndarray, m: int):
    """m-point Gauss rule of the positive discrete measure sum_k c_k delta(t - t_k).

    Discretised Stieltjes procedure: three-term recurrence of the monic
    orthogonal polynomials evaluated at the support points, then the Jacobi
    matrix eigen-decomposition (Golub-Welsch).  Returns (nodes, weights).
    """
    scale = t.max()
    x = t / scale
    mu0 = c.sum()
    p_prev = np.zeros_like(x)
    p = np.ones_like(x)
    a = np.zeros(m)
    b = np.zeros(m)
    norm_prev = None
    for j in range(m):
        norm = np.sum(c * p * p)
        a[j] = np.sum(c * x * p * p) / norm
        if j > 0:
            b[j] = norm / norm_prev
        p_next = (x - a[j]) * p - (b[j] * p_prev if j > 0 else 0.0)
        p_prev, p = p, p_next
        norm_prev = norm
    J = np.diag(a) + np.diag(np.sqrt(b[1:]), 1) + np.diag(np.sqrt(b[1:]), -1)
    ev, V = np.linalg.eigh(J)
    return ev * scale, mu0 * V[0, :] ** 2


def exp_sum(s: float, B: float, delta: float = 1e-10, s0: float = 0.5):
    """Nodes t_k and weights c_k with rho^-s ~ sum_k c_k exp(-t_k rho) on [1, B].

    Trapezoidal sinc quadrature (eqn:Sinc_quadr_trunc) of
    Gamma(s)^-1 int_R exp(s u - rho e^u) du with nodes u_k = k h, t_k = e^(u_k),
    c_k = h e^(s u_k) / Gamma(s); left tail merged by its Gauss rule.
    """
    if s <= 0.0:
        raise ValueError("s must be positive")
    h = sinc_step(delta)
    m = tail_points(delta, s0)
    gs = Gamma(s)
    k0 = int(math.floor(math.log(s0 / B) / h))
    # left tail: k0 - L .. k0 - 1, L such that c_k / c_k0 < e^-46
    L = int(math.ceil(46.0 / (s * h)))
    kt = np.arange(k0 - L, k0, dtype=np.float64)
    ut = kt * h
    tt = np.exp(ut)
    ct = h * np.exp(s * ut) / gs
    tg, cg = gauss_rule_discrete(tt, ct, m)
    # body: k0, k0+1, ... until the node is insignificant on [1, B]
    tb, cb = [], []
    k = k0
    while True:
        u = k * h
        t = math.exp(u)
        c = h * math.exp(s * u) / gs
        r = min(max(1.0, s / t), B)
        contrib = c * math.exp(-t * r) * r**s
        if u > 0.0 and contrib < delta / 20.0:
            break
        tb.append(t)
        cb.append(c)
        k += 1
    return np.concatenate([tg, tb]), np.concatenate([cg, cb])


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
