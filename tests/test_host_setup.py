"""The library's host set-up routines (csrc/setup_host.cpp) on the CPU, through a test shim
(tests/host/setup_shim.cpp) compiled here with g++: no GPU and no oracle code.  Each is
checked against what the mathematics fixes:

* the spectrum (Section 3.2) against LAPACK eigenvalues of the 1D Laplacian;
* the symbol's exponential sums (sinc quadrature of the Laplace transform, Section 4.2,
  with Lemma 4.1 for the positive power) against the exact symbol g(rho) on the grids;
* the preconditioner fit against 1/g;
* the implicit-QR tridiagonal eigen-solver of the variable-coefficient modes against LAPACK;
* the 1D stiffness matrix against its quadratic form;
* the symbol-factor compression against its defining identities.
"""
import ctypes as C
import os
import shutil
import subprocess

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_1809_01971_gb300", "csrc")

P = C.POINTER(C.c_double)
PI = C.POINTER(C.c_int)


@pytest.fixture(scope="module")
def shim(tmp_path_factory):
    gxx = shutil.which("g++")
    if gxx is None:
        pytest.skip("g++ not available")
    out = str(tmp_path_factory.mktemp("shim") / "libsetup_shim.so")
    subprocess.run([gxx, "-O2", "-std=c++17", "-fPIC", "-shared", "-I", CSRC,
                    os.path.join(CSRC, "setup_host.cpp"),
                    os.path.join(ROOT, "tests", "host", "setup_shim.cpp"), "-o", out],
                   check=True, capture_output=True, timeout=300)
    L = C.CDLL(out)
    L.shim_spectrum.argtypes = [C.c_int, P]
    L.shim_symbol_nodes.argtypes = [C.c_double, C.c_double, C.c_int] + [C.c_double] * 6 + \
        [C.c_int, P, P, PI, PI, P]
    L.shim_precond_nodes.argtypes = [C.c_double, C.c_double] + [C.c_double] * 5 + \
        [C.c_int, C.c_int, P, P, PI]
    L.shim_inverse_power_nodes.argtypes = [C.c_double, C.c_double, C.c_int, C.c_double,
                                           C.c_double, C.c_int, P, P, PI]
    L.shim_stiffness_1d.argtypes = [C.c_int, P, P, P]
    L.shim_tridiag_eig.argtypes = [C.c_int, P, P, P, P]
    L.shim_compress.argtypes = [P, C.c_int, C.c_int, P, C.c_double, P, P]
    return L


def ptr(a, t=P):
    return a.ctypes.data_as(t)


def spectrum(L, n):
    out = np.empty(n)
    L.shim_spectrum(n, ptr(out))
    return out


def lap1d(n):
    h2 = (n + 1.0) ** 2
    return h2 * (2.0 * np.eye(n) - np.eye(n, k=1) - np.eye(n, k=-1))


CAP = 4096


def nodes(L, kind, *args):
    tau, w = np.zeros(CAP), np.zeros(CAP)
    mode = np.zeros(CAP, dtype=np.int32)
    if kind == "symbol":
        counts, err = np.zeros(2, dtype=np.int32), np.zeros(1)
        r = L.shim_symbol_nodes(*args, CAP, ptr(tau), ptr(w), ptr(mode, PI), ptr(counts, PI),
                                ptr(err))
    elif kind == "precond":
        r = L.shim_precond_nodes(*args, CAP, ptr(tau), ptr(w), ptr(mode, PI))
    else:
        r = L.shim_inverse_power_nodes(*args, CAP, ptr(tau), ptr(w), ptr(mode, PI))
    assert r > 0, f"{kind} nodes failed: {r}"
    return tau[:r], w[:r], mode[:r]


def eval_nodes(tau, w, mode, lams):
    """sum_k w_k exp(-tau_k rho) * (lambda_{mode_k} if mode_k >= 0 else 1) at every grid
    point, lams the list of per-mode eigenvalue arrays (rho = sum_l lambda_l)."""
    grids = np.meshgrid(*lams, indexing="ij")
    rho = sum(grids)
    val = np.zeros_like(rho)
    for t, wk, m in zip(tau, w, mode):
        term = wk * np.exp(-t * rho)
        if m >= 0:
            term = term * grids[m]
        val += term
    return rho, val


@pytest.mark.parametrize("n", [1, 2, 7, 64, 255])
def test_spectrum_matches_lapack(shim, n):
    lam = spectrum(shim, n)
    ref = np.linalg.eigvalsh(lap1d(n))
    assert np.all(np.diff(lam) > 0)
    assert np.max(np.abs(lam - ref)) <= 1e-13 * ref[-1] * max(1, n)


def g_exact(spec, rho):
    a, sn, b, sp, c = spec
    g = np.full_like(rho, c)
    if a:
        g = g + a * rho ** (-sn)
    if b:
        g = g + b * rho ** sp
    return g


SPECS = ([("control", (1.0, al, ga, al, 0.0)) for al in (0.25, 0.5, 0.75, 1.0)
          for ga in (1e-1, 1e-3)]
         + [("A^alpha", (0.0, 1.0, 1.0, al, 0.0)) for al in (0.1, 0.5, 0.9)]
         + [("I+A^2alpha", (0.0, 1.0, 1.0, 2 * al, 1.0)) for al in (0.25, 0.5)])


@pytest.mark.parametrize("name,spec", SPECS)
@pytest.mark.parametrize("d,n", [(2, 31), (3, 15)])
def test_symbol_nodes_match_exact_symbol(shim, name, spec, d, n):
    """The CP symbol's node list reproduces g(rho) = a rho^-sn + b rho^sp + c at every grid
    point (rho = lambda_i + lambda_j (+ lambda_k)) to the quadrature accuracy (delta = 1e-10),
    the positive power through Lemma 4.1 (its terms carry lambda in one mode)."""
    lam = spectrum(shim, n)
    rmin, rmax = d * lam[0], d * lam[-1]
    tau, w, mode = nodes(shim, "symbol", rmin, rmax, d, *spec, 1e-10)
    rho, val = eval_nodes(tau, w, mode, [lam] * d)
    err = np.max(np.abs(val / g_exact(spec, rho) - 1.0))
    print(f"{name} {spec} d={d} n={n}: {len(tau)} terms, max rel err {err:.2e}")
    assert err <= 1e-9
    assert len(tau) <= 400
    assert np.all(mode < d) and np.all(mode >= -1)


@pytest.mark.parametrize("s", [0.1, 0.5, 0.75, 1.0])
def test_inverse_power_nodes(shim, s):
    """rho^-s as an exponential sum over the range of a 3D n = 255 grid (B ~ 2.6e4)."""
    lam = spectrum(shim, 255)
    rmin, rmax = 3 * lam[0], 3 * lam[-1]
    tau, w, mode = nodes(shim, "inverse", rmin, rmax, 3, s, 1e-10)
    rho = np.geomspace(rmin, rmax, 4001)
    val = (w[None, :] * np.exp(-np.outer(rho, tau))).sum(axis=1)
    assert np.all(mode == -1)
    assert np.all(w > 0)
    assert np.max(np.abs(val * rho ** s - 1.0)) <= 1e-9


def test_precond_fit_improves_with_rank(shim):
    """The least-squares exponential sum p ~ 1/g: positive, p g within (0.5, 1.5) from a few
    terms on, and closer to 1 as the rank grows."""
    lam = spectrum(shim, 255)
    rmin, rmax = 3 * lam[0], 3 * lam[-1]
    spec = (1.0, 0.75, 1e-3, 0.75, 0.0)
    rho = np.geomspace(rmin, rmax, 4001)
    devs = []
    for rank in (3, 6, 12, 24):
        tau, w, mode = nodes(shim, "precond", rmin, rmax, *spec, rank)
        p = (w[None, :] * np.exp(-np.outer(rho, tau))).sum(axis=1)
        assert np.all(p > 0)
        devs.append(np.max(np.abs(p * g_exact(spec, rho) - 1.0)))
    print("max |p g - 1| for rank 3/6/12/24:", ["%.2e" % x for x in devs])
    assert devs[-1] <= 0.5 and devs[-1] < devs[0]
    assert all(b <= a * 1.0001 for a, b in zip(devs, devs[1:]))


def test_precond_single_eigenvalue_is_exact(shim):
    lam = spectrum(shim, 1)
    spec = (1.0, 0.5, 1e-2, 0.5, 0.0)
    tau, w, mode = nodes(shim, "precond", 2 * lam[0], 2 * lam[0], *spec, 8)
    p = (w * np.exp(-tau * 2 * lam[0])).sum()
    assert abs(p * g_exact(spec, np.array([2 * lam[0]]))[0] - 1.0) <= 1e-14


def stiffness(shim, a_half):
    n = len(a_half) - 1
    dg, off = np.empty(n), np.empty(max(n - 1, 0))
    shim.shim_stiffness_1d(n, ptr(np.ascontiguousarray(a_half)), ptr(dg), ptr(off))
    return dg, off


def test_stiffness_quadratic_form_and_constant_coefficient(shim):
    """x^T T x = (n+1)^2 sum_j a((j+1/2)h) (x_{j+1} - x_j)^2 with x_0 = x_{n+1} = 0; a = 1
    gives the Laplacian."""
    rng = np.random.default_rng(11)
    n = 40
    a_half = np.exp(rng.standard_normal(n + 1))
    dg, off = stiffness(shim, a_half)
    T = np.diag(dg) + np.diag(off, 1) + np.diag(off, -1)
    for _ in range(5):
        x = rng.standard_normal(n)
        xe = np.concatenate([[0.0], x, [0.0]])
        q = (n + 1.0) ** 2 * np.sum(a_half * np.diff(xe) ** 2)
        assert abs(x @ T @ x - q) <= 1e-12 * q
    dg1, off1 = stiffness(shim, np.ones(n + 1))
    T1 = np.diag(dg1) + np.diag(off1, 1) + np.diag(off1, -1)
    assert np.max(np.abs(T1 - lap1d(n))) <= 1e-12 * (n + 1) ** 2


def tridiag_eig(shim, d, e):
    n = len(d)
    lam, V = np.empty(n), np.empty(n * n)
    rc = shim.shim_tridiag_eig(n, ptr(np.ascontiguousarray(d, dtype=float)),
                               ptr(np.ascontiguousarray(e if n > 1 else np.zeros(1), dtype=float)),
                               ptr(lam), ptr(V))
    assert rc == 0
    return lam, V.reshape(n, n, order="F")


def _cases():
    rng = np.random.default_rng(12)
    out = []
    for n in (1, 2, 3, 17, 100):
        out.append((f"random n={n}", rng.standard_normal(n), rng.standard_normal(max(n - 1, 0))))
    n = 64
    a_half = np.exp(2.0 * rng.standard_normal(n + 1))
    dg = (a_half[:-1] + a_half[1:]) * (n + 1.0) ** 2
    out.append(("stiffness n=64", dg, -a_half[1:-1] * (n + 1.0) ** 2))
    out.append(("identity n=10", np.ones(10), np.zeros(9)))
    out.append(("graded diagonal n=12", 10.0 ** -np.arange(12.0), np.zeros(11)))
    m = 10                                   # Wilkinson W21+: nearly equal eigenvalue pairs
    out.append(("Wilkinson W21+", np.abs(np.arange(-m, m + 1.0)), np.ones(2 * m)))
    out.append(("Laplacian n=255", np.full(255, 2.0), -np.ones(254)))
    return out


@pytest.mark.parametrize("name,d,e", _cases(), ids=[c[0] for c in _cases()])
def test_tridiag_eig_against_lapack(shim, name, d, e):
    n = len(d)
    lam, V = tridiag_eig(shim, d, e)
    T = np.diag(d) + (np.diag(e, 1) + np.diag(e, -1) if n > 1 else 0.0)
    nrm = max(np.max(np.abs(np.linalg.eigvalsh(T))), 1e-300)
    assert np.all(np.diff(lam) >= 0)
    assert np.max(np.abs(lam - np.linalg.eigvalsh(T))) <= 1e-13 * nrm * max(1, n) ** 0.5
    assert np.max(np.abs(V.T @ V - np.eye(n))) <= 1e-12
    assert np.max(np.abs(T @ V - V * lam[None, :])) <= 1e-12 * nrm


def test_tridiag_eig_recovers_the_laplacian_spectrum(shim):
    """The eigen-solver on the constant-coefficient stiffness matrix reproduces the closed-form
    spectrum and the DST-I eigenvectors up to sign."""
    n = 63
    dg, off = stiffness(shim, np.ones(n + 1))
    lam, V = tridiag_eig(shim, dg, off)
    assert np.max(np.abs(lam - spectrum(shim, n))) <= 1e-12 * lam[-1]
    j = np.arange(1, n + 1)
    F = np.sqrt(2.0 / (n + 1)) * np.sin(np.pi * np.outer(j, j) / (n + 1))
    assert np.max(np.abs(np.abs(F.T @ V) - np.eye(n))) <= 1e-10


def test_compress_factor_identities(shim):
    """E ~ Et Mt row by row to the tolerance, and Mt diag(xa^2) Mt^T = I, on a symbol-like
    factor E[:, k] = exp(-tau_k lambda) / ||.|| of low numerical rank."""
    lam = spectrum(shim, 127)
    tau = np.geomspace(0.2 / lam[-1], 20.0 / lam[0], 60)
    E = np.exp(-np.outer(lam, tau))
    E /= np.linalg.norm(E, axis=0)
    xa = np.exp(np.random.default_rng(13).standard_normal(60))
    n, R = E.shape
    Et, Mt = np.zeros(n * R), np.zeros(R * R)
    tol = 1e-12
    r = shim.shim_compress(ptr(np.asfortranarray(E)), n, R, ptr(xa), tol, ptr(Et), ptr(Mt))
    assert 0 < r < R
    Et = Et[:n * r].reshape(n, r, order="F")
    Mt = Mt[:r * R].reshape(r, R, order="F")
    X = E * np.abs(xa)[None, :]
    rowerr = np.linalg.norm(Et @ Mt * np.abs(xa)[None, :] - X, axis=1) / np.linalg.norm(X, axis=1)
    print(f"compressed rank {r} of {R}, max row rel err {rowerr.max():.2e}")
    assert rowerr.max() <= 100 * tol
    assert np.max(np.abs(Mt @ np.diag(xa ** 2) @ Mt.T - np.eye(r))) <= 1e-10
