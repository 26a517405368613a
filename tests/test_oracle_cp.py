"""Pins of the oracle's CP tensor operations (eqn:CP_form) and the mode-wise mat-vec
(eqn:Lap2DtimesX, eqn:Lap3DtimesX) against full-format expansions."""
import itertools

import numpy as np
import pytest

import fc_inputs as fi
from oracle import cp, quadrature as q, spectrum


def _loop_full(T):
    xi, U = T
    ns = [u.shape[0] for u in U]
    out = np.zeros(ns)
    for idx in itertools.product(*[range(n) for n in ns]):
        s = 0.0
        for r in range(len(xi)):
            p = xi[r]
            for l, i in enumerate(idx):
                p *= U[l][i, r]
            s += p
        out[idx] = s
    return out


def test_to_full_matches_loops():
    T = fi.random_cp(4, 3, 3, seed=1)
    assert np.allclose(cp.to_full(T), _loop_full(T), rtol=0, atol=1e-13)


@pytest.mark.parametrize("d", [2, 3])
def test_inner_norm_axpy(d):
    X = fi.random_cp(7, d, 4, seed=2)
    Y = fi.random_cp(7, d, 5, seed=3)
    Xf, Yf = cp.to_full(X), cp.to_full(Y)
    assert abs(cp.inner(X, Y) - np.sum(Xf * Yf)) < 1e-12 * np.linalg.norm(Xf) * np.linalg.norm(Yf)
    assert abs(cp.norm(X) - np.linalg.norm(Xf)) < 1e-12 * np.linalg.norm(Xf)
    Z = cp.axpy(X, -0.7, Y)
    assert np.allclose(cp.to_full(Z), Xf - 0.7 * Yf, atol=1e-12)
    assert cp.inner(cp.empty([7] * d), X) == 0.0


@pytest.mark.parametrize("d,n", [(2, 15), (3, 9)])
def test_apply_symbol_equals_full_format_matvec(d, n):
    """The mode-wise product equals F diag(G) F x with G the full symbol tensor."""
    sym = q.control_symbol(n, d, 0.5, 1.0, 1e-2, 1e-10)
    X = fi.random_cp(n, d, 3, seed=5)
    Y = cp.apply_symbol(sym, X)
    assert len(Y[0]) == len(sym.xi) * 3
    G = q.symbol_full(sym)
    Xf = cp.to_full(X)
    F = spectrum.sine_matrix(n)
    Z = Xf
    for ax in range(d):
        Z = np.moveaxis(np.tensordot(F, Z, axes=([1], [ax])), 0, ax)
    Z = Z * G
    for ax in range(d):
        Z = np.moveaxis(np.tensordot(F, Z, axes=([1], [ax])), 0, ax)
    assert np.linalg.norm(cp.to_full(Y) - Z) <= 1e-12 * np.linalg.norm(Z)
