"""Algorithm 1: preconditioned CG in low-rank format (paper Section 3.3).

fun     = X -> F(A) X with the control symbol (eqn:forControl times beta),
precond = X -> P(A) X with the fitted inverse symbol,
trunc   = RHOSVD truncation (oracle.truncate).

Readings: B is column-normalised on entry (same tensor);
every truncation, of mat-vec outputs too, works on the column-normalised
representation (the RHOSVD of Section 5 with unit columns, the weights
carrying the norms); X^(0) = 0 so R^(0) = B; "R sufficiently
small" is the recursive ||R^(k+1)|| / ||B|| <= tol; k_max = 100 (the paper's
failure threshold for its tables).  The true residual ||B - fun(X)|| / ||B|| is
reported at exit.
"""
from __future__ import annotations

from dataclasses import dataclass, field

from . import cp
from .quadrature import normalise_columns
from .truncate import truncate


@dataclass
class PCGResult:
    X: tuple
    iters: int
    relres: float
    status: str
    history: list = field(default_factory=list)
    ranks: list = field(default_factory=list)


def pcg(fun_sym, pre_sym, B, eps, tol, max_rank, kmax=100) -> PCGResult:
    """Algorithm 1 with X^(0) = 0."""
    def fun(X):
        return cp.apply_symbol(fun_sym, X)

    def precond(X):
        return cp.apply_symbol(pre_sym, X)

    def trunc(X, normalize=True):
        return truncate(X, eps, max_rank, normalize=normalize)

    ns = [u.shape[0] for u in B[1]]
    bnorm = cp.norm(B)
    X = cp.empty(ns)
    if bnorm == 0.0:
        return PCGResult(X, 0, 0.0, "ok")
    B = normalise_columns(*B)               # same tensor, unit columns
    R = B                                   # R0 = B - fun(X0), X0 = 0
    Z = trunc(precond(R))                   # Z0 = trunc(precond(R0))
    P = Z                                   # P0 = Z0
    rz = cp.inner(R, Z)
    hist = []
    ranks = []
    for k in range(kmax):
        S = trunc(fun(P))                   # S = trunc(fun(P))
        ps = cp.inner(P, S)
        if not ps > 0.0:
            return PCGResult(X, k, hist[-1] if hist else 1.0, "breakdown", hist, ranks)
        a = rz / ps                         # alpha_k
        X = trunc(cp.axpy(X, a, P))         # X = trunc(X + alpha P)
        R = trunc(cp.axpy(R, -a, S))        # R = trunc(R - alpha S)
        rel = cp.norm(R) / bnorm
        hist.append(rel)
        ranks.append(dict(X=cp.rank(X), R=cp.rank(R), S=cp.rank(S), P=cp.rank(P)))
        if rel <= tol:
            return PCGResult(X, k + 1, rel, "ok", hist, ranks)
        Zn = trunc(precond(R))              # Z = trunc(precond(R))
        rzn = cp.inner(R, Zn)
        b = rzn / rz                        # beta_k = <R+,Z+>/<Z,R>
        P = trunc(cp.axpy(Zn, b, P))        # P = trunc(Z + beta P)
        Z, rz = Zn, rzn
    return PCGResult(X, kmax, hist[-1], "noconv", hist, ranks)


def true_relres(fun_sym, B, X) -> float:
    """||B - fun(X)|| / ||B|| in full format (small n only)."""
    import numpy as np
    r = cp.to_full(B) - cp.to_full(cp.apply_symbol(fun_sym, X))
    return float(np.linalg.norm(r) / np.linalg.norm(cp.to_full(B)))
