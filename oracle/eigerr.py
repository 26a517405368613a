"""Error of a CP-format solution against the exact full-format solution, over the whole grid.

Paper Section 3.2 (eqn:DiagFLaplace3D / eqn:DiagFLaplace2D): the exact solution of
g(A) u = b is u* = (F x .. x F) diag(1/g(rho)) (F x .. x F) b.  Because F x .. x F is
orthogonal, ||u - u*|| is the distance between the DST-transformed CP tensor uh and
bh / g(rho) on the eigen-index grid.  The sum over all n^d points runs in plain C
(``csrc/eigerr.c``, OpenMP over the outer index), so grids of 10^9 points (n = 1023) take
seconds and no n^d array is formed.  The transforms of the factor columns are the library
DST-I of ``spectrum.dst1``.

On grids too large to sum whole (n = 8191) the sum runs over the box of low eigen-indices
that carries the right-hand side's transform, with the remainder bounded from the CP forms
(``control_error``).

This is test infrastructure: the C source is compiled here with gcc on first use (or by the
repository's build step) into ``oracle/_build``.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess

import numpy as np

from .spectrum import dst1, eigenvalues

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "csrc", "eigerr.c")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(BUILD, "libeigerr.so")
_lib = None


def build() -> str:
    """Compile csrc/eigerr.c (gcc, OpenMP) into oracle/_build/libeigerr.so."""
    os.makedirs(BUILD, exist_ok=True)
    tmp = LIB + f".{os.getpid()}.tmp"
    subprocess.run(["gcc", "-O3", "-fopenmp", "-fPIC", "-shared", "-o", tmp, SRC, "-lm"],
                   check=True, capture_output=True)
    os.replace(tmp, LIB)
    return LIB


def _load():
    global _lib
    if _lib is None:
        if not os.path.exists(LIB) or os.path.getmtime(LIB) < os.path.getmtime(SRC):
            build()
        L = C.CDLL(LIB)
        P = C.POINTER(C.c_double)
        L.eig_error.restype = C.c_int
        L.eig_error.argtypes = [C.c_int, C.c_int, C.POINTER(C.c_int), P, C.c_double, C.c_double,
                                C.c_double, C.c_double, C.c_double, C.c_int, P, C.POINTER(P),
                                C.c_int, P, C.POINTER(P), C.c_int, P]
        _lib = L
    return _lib


def _ptr(a):
    return a.ctypes.data_as(C.POINTER(C.c_double))


def transform(T):
    """Weights and DST-transformed factors (F U_l), row-major (n, R) per mode."""
    xi, U = T
    xi = np.ascontiguousarray(np.asarray(xi, dtype=np.float64))
    Uh = [np.ascontiguousarray(dst1(np.asarray(u, dtype=np.float64), axis=0)) for u in U]
    return xi, Uh


def box_sums(uh, bh, ga, sn, gb, sp, gc=0.0, box=None, lam=None, threads=0):
    """(sum (uh - bh/g)^2, sum (bh/g)^2, sum uh^2) over the eigen-index box i_l < box[l]
    (default: the whole grid) for g(rho) = ga rho^-sn + gb rho^sp + gc.  uh, bh: transformed
    CP tensors (weights, row-major factors).  lam: per-mode spectra (default eqn:eig_lap)."""
    xu, Uu = uh
    xb, Ub = bh
    d = len(Ub)
    n = int(Ub[0].shape[0])
    if lam is None:
        lam = [eigenvalues(n)] * d
    m = (C.c_int * 3)(*([int(k) for k in (box if box is not None else [n] * d)] + [0] * (3 - d)))
    lam_all = np.ascontiguousarray(np.concatenate(list(lam) + [np.zeros(n)] * (3 - d)))
    P = C.POINTER(C.c_double)
    Up = (P * 3)(*[_ptr(Uu[min(l, d - 1)]) for l in range(3)])
    Bp = (P * 3)(*[_ptr(Ub[min(l, d - 1)]) for l in range(3)])
    out = np.zeros(3)
    if threads <= 0:
        threads = len(os.sched_getaffinity(0))
    rc = _load().eig_error(d, n, m, _ptr(lam_all), float(ga), float(sn), float(gb), float(sp),
                           float(gc), len(xu), _ptr(xu), Up, len(xb), _ptr(xb), Bp, int(threads),
                           _ptr(out))
    if rc != 0:
        raise ValueError("eig_error: bad arguments")
    return out


def error_sums(u_cp, b_cp, ga, sn, gb, sp, gc=0.0, lam=None, threads=0):
    """box_sums over the whole grid, from untransformed CP tensors."""
    return box_sums(transform(u_cp), transform(b_cp), ga, sn, gb, sp, gc, None, lam, threads)


def _restricted_norm2(T, K, modes):
    """||T restricted to rows >= K[l] in the modes of `modes`||^2 of a CP tensor (Gram sum)."""
    xi, U = T
    M = np.outer(xi, xi)
    for l, u in enumerate(U):
        v = u[K[l]:] if l in modes else u
        M = M * (v.T @ v)
    return float(M.sum())


def _g_min(alpha, beta, gamma_, rmin, rmax):
    """Smallest value of g(rho) = beta^2 rho^-alpha + gamma rho^alpha on [rmin, rmax]."""
    cand = [rmin, rmax]
    rstar = (beta**2 / gamma_) ** (1.0 / (2.0 * alpha))
    if rmin < rstar < rmax:
        cand.append(rstar)
    return min(beta**2 * r ** (-alpha) + gamma_ * r**alpha for r in cand)


def control_error(u_cp, b_cp, alpha, beta, gamma_, threads=0, full_limit=1.2e9,
                  rel_tail=1e-13, force_box=False):
    """Relative L2 error ||u - u*|| / ||u*|| of a CP solution u of
    (beta^2 A^-alpha + gamma A^alpha) u = b (eqn:DiagFLaplace3D), and ||u*||.

    Grids of at most full_limit points are summed whole.  Larger grids (n = 8191: 5.5e11
    points) are summed over the box of low eigen-indices that holds b's transform: per mode
    the smallest K_l whose slab {i_l >= K_l} carries at most rel_tail ||bh|| of it by the
    triangle bound over the CP terms (sum_r |xi_r| ||f_rl[K_l:]|| prod_{m != l} ||f_rm||).
    Outside the box the solution's own energy is taken exactly from its CP form
    (inclusion-exclusion over the slabs), and u*'s is bounded by that tail / min g; the
    returned error is the upper end of the resulting interval."""
    d = len(b_cp[1])
    n = int(b_cp[1][0].shape[0])
    uh, bh = transform(u_cp), transform(b_cp)
    if force_box or float(n) ** d > full_limit:
        xb, Fb = bh
        bnorm = np.sqrt(max(_restricted_norm2((xb, Fb), [0] * d, ()), 0.0))
        colnorm = [np.linalg.norm(f, axis=0) for f in Fb]
        K, tails = [], []
        for l in range(d):
            other = np.ones(len(xb))
            for m_ in range(d):
                if m_ != l:
                    other = other * colnorm[m_]
            suffix = np.sqrt(np.cumsum((Fb[l] ** 2)[::-1], axis=0)[::-1])      # ||f[k:]||
            tail = np.append(suffix @ (np.abs(xb) * other), 0.0)           # tail[k], k = 0..n
            k = int(np.argmax(tail <= rel_tail * bnorm))
            K.append(max(k, 1))
            tails.append(tail[K[-1]])
        s = box_sums(uh, bh, beta**2, alpha, gamma_, alpha, 0.0, K, None, threads)
        out_u = 0.0
        for mask in range(1, 1 << d):                    # inclusion-exclusion over the slabs
            modes = tuple(l for l in range(d) if mask >> l & 1)
            out_u += (-1) ** (len(modes) + 1) * _restricted_norm2(uh, K, modes)
        out_u = max(out_u, 0.0)
        lam = eigenvalues(n)
        gmin = _g_min(alpha, beta, gamma_, d * lam[0], d * lam[-1])
        out_w = (np.sqrt(np.sum(np.square(tails))) / gmin) ** 2
        err2 = s[0] + (np.sqrt(out_u) + np.sqrt(out_w)) ** 2
        return float(np.sqrt(err2 / s[1])), float(np.sqrt(s[1]))
    s = box_sums(uh, bh, beta**2, alpha, gamma_, alpha, 0.0, None, None, threads)
    return float(np.sqrt(s[0] / s[1])), float(np.sqrt(s[1]))
