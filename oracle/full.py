"""Full-format references (paper Section 3.2, eqn:DiagFLaplace3D / 2D).

solve_full:  u = (F_1 x ... x F_d) diag(1/g(rho)) (F_1 x ... x F_d) b, the exact
             eigenbasis solve of (beta^2 A^-alpha + gamma A^alpha) u = b; d passes
             of the 1D DST-I, a pointwise division, d passes again.
brute_force: dense A = sum_l I x A_(l) x I (eqn_low_rank_lap), symmetric
             eigendecomposition, A^{+-alpha} by the spectral definition
             (eqn:frac_Oper), dense solve.  Independent of the DST; n <= 16.
g_operator / solve_full_op / brute_force_op: the same for the test operators of Section 6
             (Tables 6.1-6.4): A^alpha and I + A^(2 alpha), besides the control operator.
stiffness_1d / solve_full_varcoef / brute_force_varcoef: separable variable coefficients
             (Remark on generalised directionally fractional operators): mode l carries the
             stiffness matrix of -(a_l u')', its orthonormal eigenvectors replace the DST-I.
"""
from __future__ import annotations

import numpy as np

from .spectrum import dst1, eigenvalues, laplacian_1d
from .quadrature import g_control, rho_full


def dst_all(Y: np.ndarray) -> np.ndarray:
    for ax in range(Y.ndim):
        Y = dst1(Y, axis=ax)
    return Y


def apply_g_full(Y: np.ndarray, gfun) -> np.ndarray:
    """F g(Lambda) F y for a full tensor y (eqn:DiagFLaplace3D)."""
    lams = [eigenvalues(m) for m in Y.shape]
    return dst_all(dst_all(Y) * gfun(rho_full(lams)))


def solve_full(b: np.ndarray, alpha, beta, gamma_) -> np.ndarray:
    """Exact solution u* of (beta^2 A^-alpha + gamma A^alpha) u = b."""
    return apply_g_full(b, lambda r: 1.0 / g_control(r, alpha, beta, gamma_))


def apply_full(x: np.ndarray, alpha, beta, gamma_) -> np.ndarray:
    """(beta^2 A^-alpha + gamma A^alpha) x in full format."""
    return apply_g_full(x, lambda r: g_control(r, alpha, beta, gamma_))


def state_full(u: np.ndarray, alpha, beta) -> np.ndarray:
    """State y = beta A^-alpha u (eqn:State, eqn:L_alp_state) in full format."""
    return apply_g_full(u, lambda r: beta * r ** (-alpha))


def solve_full_directional(b: np.ndarray, alpha, beta, gamma_) -> np.ndarray:
    """Exact solution of (beta^2 A_(alpha)^-1 + gamma A_(alpha)) u = b for the directionally
    fractional Laplacian A_(alpha) = sum_l (-Delta_l)^alpha (Remark after Lemma 4.1,
    eq:Laplace_1Dfract, eq:3b1d): in the DST-I eigenbasis A_(alpha) is diagonal with
    mu(i) = sum_l lambda_{i_l}^alpha."""
    mu = rho_full([eigenvalues(m) ** alpha for m in b.shape])
    return dst_all(dst_all(b) / (beta**2 / mu + gamma_ * mu))


def dense_directional(ns, alpha) -> np.ndarray:
    """Dense A_(alpha) = sum_l I x (A_(l))^alpha x I, (A_(l))^alpha by the 1D eigendecomposition
    (no DST involved)."""
    d = len(ns)
    N = int(np.prod(ns))
    A = np.zeros((N, N))
    for l in range(d):
        w, V = np.linalg.eigh(laplacian_1d(ns[l]))
        mats = [np.eye(m) for m in ns]
        mats[l] = V @ np.diag(w**alpha) @ V.T
        K = mats[0]
        for M in mats[1:]:
            K = np.kron(K, M)
        A += K
    return A


def dense_laplacian(ns) -> np.ndarray:
    """A = sum_l I x ... x A_(l) x ... x I with axis 0 = mode 1 fastest-varying
    last in numpy C order (A acts on x.reshape(-1) of an array of shape ns)."""
    d = len(ns)
    N = int(np.prod(ns))
    A = np.zeros((N, N))
    for l in range(d):
        mats = [np.eye(m) for m in ns]
        mats[l] = laplacian_1d(ns[l])
        K = mats[0]
        for M in mats[1:]:
            K = np.kron(K, M)
        A += K
    return A


def brute_force_solve(b: np.ndarray, alpha, beta, gamma_) -> np.ndarray:
    """Dense eigendecomposition solve (eqn:frac_Oper), no DST involved."""
    A = dense_laplacian(b.shape)
    w, V = np.linalg.eigh(A)
    Mop = V @ np.diag(beta**2 * w ** (-alpha) + gamma_ * w**alpha) @ V.T
    return np.linalg.solve(Mop, b.reshape(-1)).reshape(b.shape)


def brute_force_power(ns, s) -> np.ndarray:
    """Dense A^s by the spectral definition (eqn:frac_Oper)."""
    A = dense_laplacian(ns)
    w, V = np.linalg.eigh(A)
    return V @ np.diag(w**s) @ V.T


def g_operator(rho, kind, alpha, beta=1.0, gamma_=1.0):
    """Symbol of the operator: kind 0 beta^2 rho^-alpha + gamma rho^alpha (the control
    operator; A^alpha + A^-alpha at beta = gamma = 1), kind 1 rho^alpha (A^alpha), kind 2
    1 + rho^(2 alpha) (I + A^(2 alpha))."""
    if kind == 0:
        return g_control(rho, alpha, beta, gamma_)
    if kind == 1:
        return rho ** alpha
    if kind == 2:
        return 1.0 + rho ** (2.0 * alpha)
    raise ValueError(kind)


def solve_full_op(b: np.ndarray, kind, alpha, beta=1.0, gamma_=1.0) -> np.ndarray:
    """Exact solution of L u = b, L the operator of `kind`, in the DST-I eigenbasis."""
    return apply_g_full(b, lambda r: 1.0 / g_operator(r, kind, alpha, beta, gamma_))


def brute_force_op(b: np.ndarray, kind, alpha, beta=1.0, gamma_=1.0) -> np.ndarray:
    """Dense solve with the operator assembled from the dense A by its eigendecomposition:
    A^alpha, I + A^(2 alpha) or beta^2 A^-alpha + gamma A^alpha (no DST involved)."""
    A = dense_laplacian(b.shape)
    w, V = np.linalg.eigh(A)
    if kind == 0:
        f = beta**2 * w ** (-alpha) + gamma_ * w**alpha
    elif kind == 1:
        f = w**alpha
    elif kind == 2:
        f = 1.0 + w ** (2.0 * alpha)
    else:
        raise ValueError(kind)
    return np.linalg.solve(V @ np.diag(f) @ V.T, b.reshape(-1)).reshape(b.shape)


def stiffness_1d(n: int, a_half) -> np.ndarray:
    """Dense 1D stiffness matrix of -(a u')' with Dirichlet ends: a_half[i] = a((i+1/2) h),
    i = 0..n; row i: (a_half[i] + a_half[i+1]) / h^2 on the diagonal, -a_half[i+1] / h^2 next
    to it.  a = 1 gives A_(l)."""
    a = np.asarray(a_half, dtype=np.float64)
    h2 = (n + 1.0) ** 2
    T = np.diag((a[:-1] + a[1:]) * h2)
    off = -a[1:-1] * h2
    return T + np.diag(off, 1) + np.diag(off, -1)


def _mode_bases(shape, coeffs):
    """Per mode: eigenvalues (ascending) and orthonormal eigenvectors of the 1D operator."""
    out = []
    for l, m in enumerate(shape):
        a = coeffs[l] if coeffs is not None and l < len(coeffs) else None
        if a is None:
            out.append((eigenvalues(m), None))
        else:
            w, V = np.linalg.eigh(stiffness_1d(m, a))
            out.append((w, V))
    return out


def solve_full_varcoef(b: np.ndarray, coeffs, kind, alpha, beta=1.0, gamma_=1.0) -> np.ndarray:
    """Exact solution of L u = b for the operator of `kind` built on A = sum_l I x A_l x I,
    A_l the stiffness matrix of mode l (DST-I for a constant coefficient): transform every
    mode to its eigenbasis, divide by g(sum_l lambda_l), transform back."""
    bases = _mode_bases(b.shape, coeffs)
    Y = b.copy()
    for l, (w, V) in enumerate(bases):
        Y = dst1(Y, axis=l) if V is None else np.moveaxis(np.tensordot(V.T, Y, axes=(1, l)), 0, l)
    Y = Y / g_operator(rho_full([w for w, _ in bases]), kind, alpha, beta, gamma_)
    for l, (w, V) in enumerate(bases):
        Y = dst1(Y, axis=l) if V is None else np.moveaxis(np.tensordot(V, Y, axes=(1, l)), 0, l)
    return Y


def brute_force_varcoef(b: np.ndarray, coeffs, kind, alpha, beta=1.0, gamma_=1.0) -> np.ndarray:
    """Dense solve: A = sum_l I x A_l x I assembled from the dense 1D matrices, the operator
    from A's eigendecomposition (no per-mode transform involved)."""
    ns = b.shape
    N = int(np.prod(ns))
    A = np.zeros((N, N))
    for l in range(len(ns)):
        a = coeffs[l] if coeffs is not None and l < len(coeffs) else None
        mats = [np.eye(m) for m in ns]
        mats[l] = laplacian_1d(ns[l]) if a is None else stiffness_1d(ns[l], a)
        K = mats[0]
        for Mx in mats[1:]:
            K = np.kron(K, Mx)
        A += K
    w, V = np.linalg.eigh(A)
    f = g_operator(w, kind, alpha, beta, gamma_)
    return np.linalg.solve(V @ np.diag(f) @ V.T, b.reshape(-1)).reshape(b.shape)
