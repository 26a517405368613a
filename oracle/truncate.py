"""RHOSVD rank truncation, canonical -> Tucker -> canonical (paper Section 5).

Algorithm 1 applies ``trunc`` after every update; in 2D the paper uses the
reduced SVD, in 3D the RHOSVD canonical-to-Tucker-to-canonical transform
(Section 3.3 after Algorithm 1; Section 5, eqn:two_level).

Steps (the paper's order):
  1. RHOSVD (Section 5): per mode l, the leading left singular vectors Z_l of
     the side matrix of the normalised canonical tensor (eqn:CP_form,
     normalised u, weights xi).  No full tensor is formed.
  2. Tucker core beta = T x_1 Z_1^T ... x_d Z_d^T (eqn:coret), computed from
     the projected side matrices C_l = Z_l^T U_l: beta = sum_r xi_r (x)_l C_l[:, r].
  3. Tucker-to-canonical of the small core (mixed format eqn:two_level):
     d = 2: SVD of the r_1 x r_2 core (the 2D reduced SVD);
     d = 3: rotate mode 3 to the core's mode-3 singular vectors, then SVD of
     each r_1 x r_2 slice; rank <= r_3 min(r_1, r_2) <= r^2.
  4. Side matrices of the result U'_l = Z_l C'_l (eqn:two_level).

Readings (the paper does not state the thresholds):
  * Side-matrix weighting: W_l = U_l diag(|xi|) with U_l column-normalised and
    xi carrying the term norms, so the singular values are in the units of T.
    Mat-vec outputs (columns e_k . y_j, not unit) are normalised the same way:
    the weight of a term is |xi_k eta_j| prod_l ||e_lk . y_lj||.
  * Stage-1 rank: smallest r_l with (sum_{k>r_l} sigma_{l,k}^2)^(1/2)
    <= eps ||xi||_2 / sqrt(2d), capped at max_tucker = 48.  ||xi||_2 of the
    normalised representation is the scale of the RHOSVD error bound
    (Section 5): projecting mode l costs at most the discarded side-matrix
    energy times ||M_l||_2, M_l the Khatri-Rao product of the other modes'
    unit columns.  The CP cap max_rank applies to the canonical terms of
    stage 2 only, so that in 2D the result is the reduced-SVD (Eckart-Young)
    truncation the paper names.
  * Stage-2 rank: the canonical terms of step 3 are mutually orthogonal, so
    dropping a set of them costs exactly (sum dropped sigma^2)^(1/2); we drop the
    smallest while that is <= eps ||beta|| / sqrt(2), then keep at most max_rank.
  * The oracle computes the side-matrix singular vectors by LAPACK SVD
    (Householder bidiagonalisation), not by Gram matrices.
"""
from __future__ import annotations

import math

import numpy as np


def _normalise(T):
    xi, V = T
    d = len(V)
    if len(xi) == 0:
        return xi, V
    nrm = np.ones(len(xi))
    U = []
    for l in range(d):
        c = np.linalg.norm(V[l], axis=0)
        nrm = nrm * c
        U.append(V[l] / np.where(c > 0, c, 1.0))
    w = xi * nrm
    keep = w != 0.0
    return w[keep], [u[:, keep] for u in U]


MAX_TUCKER = 48


def truncate(T, eps: float, max_rank: int, info: dict | None = None,
             normalize: bool = True, max_tucker: int = MAX_TUCKER):
    """trunc(T, eps) of Algorithm 1 (reading above).  Returns a CP tensor with
    orthonormal-slice structure and normalised columns.

    normalize=True (what Algorithm 1 uses) rescales every column to unit norm first
    (weights absorb the norms).  normalize=False keeps the representation as given.
    """
    if normalize:
        xi, U = _normalise(T)
    else:
        keep = T[0] != 0.0
        xi, U = T[0][keep], [u[:, keep] for u in T[1]]
    d = len(U)
    ns = [u.shape[0] for u in U]
    if len(xi) == 0:
        if info is not None:
            info.update(ranks=[0] * d, rank=0, est_err=0.0, core_norm=0.0)
        return np.zeros(0), [np.zeros((n, 0)) for n in ns]
    wnorm = float(np.linalg.norm(xi))
    thr1 = eps * wnorm / math.sqrt(2.0 * d)
    Z, C, e1, tails1 = [], [], 0.0, []
    for l in range(d):
        W = U[l] * np.abs(xi)[None, :]
        Zl, s, _ = np.linalg.svd(W, full_matrices=False)
        tail = np.sqrt(np.cumsum((s**2)[::-1])[::-1])   # tail[r] = ||s[r:]||
        tail = np.append(tail, 0.0)
        r = next(i for i in range(len(tail)) if tail[i] <= thr1)
        r = max(1, min(r, max_tucker, len(s)))
        e1 += tail[r] ** 2
        tails1.append(float(tail[r]))
        Z.append(Zl[:, :r])
        C.append(Zl[:, :r].T @ U[l])
    # Tucker core (eqn:coret)
    if d == 2:
        core = (C[0] * xi[None, :]) @ C[1].T
    elif d == 3:
        core = np.einsum("r,ar,br,cr->abc", xi, C[0], C[1], C[2], optimize=True)
    else:
        raise ValueError("d must be 2 or 3")
    bnorm = float(np.linalg.norm(core))
    # canonical terms from the core
    if d == 2:
        X, s, Yt = np.linalg.svd(core, full_matrices=False)
        terms = [(s[i], (X[:, i], Yt[i, :])) for i in range(len(s))]
    else:
        r1, r2, r3 = core.shape
        unf3 = core.reshape(r1 * r2, r3).T               # mode-3 unfolding
        W3, s3, _ = np.linalg.svd(unf3, full_matrices=False)
        terms = []
        for c in range(W3.shape[1]):
            S = np.tensordot(core, W3[:, c], axes=([2], [0]))
            X, s, Yt = np.linalg.svd(S, full_matrices=False)
            for i in range(len(s)):
                terms.append((s[i], (X[:, i], Yt[i, :], W3[:, c])))
    terms.sort(key=lambda t: -t[0])
    sig = np.array([t[0] for t in terms])
    tail = np.sqrt(np.cumsum((sig**2)[::-1])[::-1])
    tail = np.append(tail, 0.0)
    thr2 = eps * bnorm / math.sqrt(2.0)
    q = next(i for i in range(len(tail)) if tail[i] <= thr2)
    q = max(1 if bnorm > 0 else 0, min(q, max_rank))
    e2 = tail[q]
    out_xi = sig[:q].copy()
    out_U = []
    for l in range(d):
        cols = np.stack([t[1][l] for t in terms[:q]], axis=1) if q else np.zeros((Z[l].shape[1], 0))
        out_U.append(Z[l] @ cols)
    if info is not None:
        info.update(ranks=[z.shape[1] for z in Z], rank=q,
                    est_err=float(math.sqrt(e1 + e2**2)), core_norm=bnorm, bases=Z,
                    stage1_tails=tails1, stage2_err=float(e2), sigma=sig)
    return out_xi, out_U
