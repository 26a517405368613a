"""Canonical (CP) tensors and the mode-wise mat-vec (paper Sections 3.2, 5).

A CP tensor is a pair (xi, U) with xi of shape (R,) and U = [U_1, ..., U_d],
U_l of shape (n_l, R):  T = sum_r xi_r U_1[:, r] x ... x U_d[:, r]
(eqn:CP_form; columns need not be normalised here).
"""
from __future__ import annotations

import numpy as np

from .spectrum import dst1


def rank(T) -> int:
    return len(T[0])


def to_full(T) -> np.ndarray:
    """Expand to the full n_1 x ... x n_d array (i_1 is axis 0)."""
    xi, U = T
    d = len(U)
    letters = "abcdefgh"[:d]
    spec = ",".join(f"{c}r" for c in letters)
    return np.einsum(f"r,{spec}->{letters}", xi, *U, optimize=True)


def inner(X, Y) -> float:
    """<X, Y> = sum_{k,j} xi_k eta_j prod_l <x_k^l, y_j^l> (inner products of
    Algorithm 1, alpha_k and beta_k)."""
    xi, U = X
    eta, V = Y
    if len(xi) == 0 or len(eta) == 0:
        return 0.0
    M = np.outer(xi, eta)
    for Ul, Vl in zip(U, V):
        M = M * (Ul.T @ Vl)
    return float(M.sum())


def norm(X) -> float:
    return float(np.sqrt(max(inner(X, X), 0.0)))


def axpy(X, a, Y):
    """X + a*Y by concatenating the terms (Algorithm 1, lines X+aP, R-aS, Z+bP)."""
    xi, U = X
    eta, V = Y
    return (np.concatenate([xi, a * eta]),
            [np.concatenate([Ul, Vl], axis=1) for Ul, Vl in zip(U, V)])


def scale(X, a):
    return (a * X[0], [u.copy() for u in X[1]])


def empty(ns):
    return (np.zeros(0), [np.zeros((n, 0)) for n in ns])


def apply_symbol(sym, X):
    """F(A) x in low-rank form (eqn:Lap2DtimesX, eqn:Lap3DtimesX).

    F(A) x = sum_k sum_j xi_k eta_j (x)_l F_l (u_l^k . F_l x_l^j)
    with F_l the orthonormal DST-I (F* = F).  The result has rank R * S; the
    column index of term (k, j) is k*S + j.
    """
    xi_s, E = sym.xi, sym.U
    eta, V = X
    R, S = len(xi_s), len(eta)
    d = len(V)
    out_U = []
    for l in range(d):
        Vh = dst1(V[l], axis=0)                       # F x_l^j
        W = np.empty((V[l].shape[0], R * S))
        for k in range(R):
            W[:, k * S:(k + 1) * S] = E[l][:, k:k + 1] * Vh   # u_l^k . F x_l^j
        out_U.append(dst1(W, axis=0))                  # F* (...)
    out_xi = np.outer(xi_s, eta).reshape(-1)
    return out_xi, out_U
