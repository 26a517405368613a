"""Error of a CP-format solution against the exact full-format solution, over the whole grid.

Paper Section 3.2 (eqn:DiagFLaplace3D / eqn:DiagFLaplace2D): the exact solution of
g(A) u = b is u* = (F x .. x F) diag(1/g(rho)) (F x .. x F) b.  Because F x .. x F is
orthogonal, ||u - u*|| is the distance between the DST-transformed CP tensor uh and
bh / g(rho) on the eigen-index grid.  The sum over all n^d points runs in plain C
(``csrc/eigerr.c``, OpenMP over the outer index), so grids of 10^9 points (n = 1023) take
seconds and no n^d array is formed.  The transforms of the factor columns are the library
DST-I of ``spectrum.dst1``.

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
        L.eig_error.argtypes = [C.c_int, C.c_int, P, C.c_double, C.c_double, C.c_double,
                                C.c_double, C.c_double, C.c_int, P, C.POINTER(P), C.c_int, P,
                                C.POINTER(P), C.c_int, P]
        _lib = L
    return _lib


def _ptr(a):
    return a.ctypes.data_as(C.POINTER(C.c_double))


def _prep(T):
    """Weights and DST-transformed factors, row-major (n, R) per mode."""
    xi, U = T
    xi = np.ascontiguousarray(np.asarray(xi, dtype=np.float64))
    Uh = [np.ascontiguousarray(dst1(np.asarray(u, dtype=np.float64), axis=0)) for u in U]
    return xi, Uh


def error_sums(u_cp, b_cp, ga, sn, gb, sp, gc=0.0, lam=None, threads=0):
    """(sum (uh - bh/g)^2, sum (bh/g)^2, sum uh^2) over the n^d eigen-index grid for
    g(rho) = ga rho^-sn + gb rho^sp + gc.  lam: per-mode spectra (default eqn:eig_lap)."""
    d = len(b_cp[1])
    n = int(b_cp[1][0].shape[0])
    if lam is None:
        lam = [eigenvalues(n)] * d
    lam_all = np.ascontiguousarray(np.concatenate(list(lam) + [np.zeros(n)] * (3 - d)))
    xu, Uu = _prep(u_cp)
    xb, Ub = _prep(b_cp)
    P = C.POINTER(C.c_double)
    Up = (P * 3)(*[_ptr(Uu[min(l, d - 1)]) for l in range(3)])
    Bp = (P * 3)(*[_ptr(Ub[min(l, d - 1)]) for l in range(3)])
    out = np.zeros(3)
    if threads <= 0:
        threads = len(os.sched_getaffinity(0))
    rc = _load().eig_error(d, n, _ptr(lam_all), float(ga), float(sn), float(gb), float(sp),
                           float(gc), len(xu), _ptr(xu), Up, len(xb), _ptr(xb), Bp, int(threads),
                           _ptr(out))
    if rc != 0:
        raise ValueError("eig_error: bad arguments")
    return out


def control_error(u_cp, b_cp, alpha, beta, gamma_, threads=0):
    """Relative L2 error ||u - u*|| / ||u*|| of a CP solution u of
    (beta^2 A^-alpha + gamma A^alpha) u = b, and ||u*||."""
    s = error_sums(u_cp, b_cp, beta**2, alpha, gamma_, alpha, 0.0, threads=threads)
    return float(np.sqrt(s[0] / s[1])), float(np.sqrt(s[1]))
