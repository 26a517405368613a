"""Parity of the CUDA path (through the C ABI) with the CPU FP64 oracle.

Every case runs on seeded synthetic inputs (fc_inputs) at sizes the oracle finishes in
seconds, with ragged n (not a multiple of the 64-wide GEMM tile) and several tiles.
Tolerances (relative L2 of the represented full tensors unless stated):
  * exact-arithmetic steps (DST-I mat-vec, inner product, full expansion, full-format
    solve): 1e-12, the FP64 rounding level of O(n) sums of O(1) terms;
  * symbol against the exact g(rho): 1e-9 (setup targets 1e-10 on a rho grid);
  * truncation: c * eps * ||T|| with c from the split of eps over the RHOSVD stages;
  * CP-PCG solve against the oracle's full solution: max(eps, 1e-8) scaled by the
    operator's conditioning as stated per test.
"""
import math

import numpy as np
import pytest
import torch

import fc_inputs as fi
from oracle import cp, full, quadrature as q

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def fc():
    import paper_1809_01971_gb300 as m
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    m.lib()
    return m


def rel(a, b):
    a = np.asarray(a)
    b = np.asarray(b)
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def sym_obj(fc, h, which):
    s = fc.CP(h.d, h.n, h.info.rank_symbol if which == 0 else h.info.rank_precond)
    fc.fc_get_symbol(h, which, s)
    xi, U = s.factors()
    return q.Symbol(xi, U, None, "gpu")


def gpu_full(fc, h, X):
    return fc.fc_to_full(h, X).cpu().numpy()


@pytest.mark.parametrize("n,d,alpha,gamma_", [(15, 2, 0.5, 1e-2), (63, 2, 0.5, 1e-2),
                                             (15, 3, 0.25, 1e-1), (37, 3, 0.75, 1e-3),
                                             (20, 3, 1.0, 1e-2)])
def test_symbol_matches_exact_g(fc, n, d, alpha, gamma_):
    h = fc.fc_setup(n, d, alpha, 1.0, gamma_, 1e-8)
    assert h.info.sym_err < 1e-9
    s = sym_obj(fc, h, 0)
    G = cp.to_full((s.xi, s.U))
    lams = [q.eigenvalues(n)] * d if hasattr(q, "eigenvalues") else None
    from oracle.spectrum import eigenvalues
    rho = q.rho_full([eigenvalues(n)] * d)
    g = q.g_control(rho, alpha, 1.0, gamma_)
    err = float(np.max(np.abs(G / g - 1.0)))
    print(f"n={n} d={d} a={alpha} RA={h.info.rank_symbol} symbol max rel err {err:.3e}")
    assert err < 1e-9
    del lams


@pytest.mark.parametrize("n,d,alpha,gamma_", [(31, 2, 0.5, 1e-2), (25, 3, 0.25, 1e-3)])
def test_precond_symbol_is_positive_and_close_to_inverse(fc, n, d, alpha, gamma_):
    h = fc.fc_setup(n, d, alpha, 1.0, gamma_, 1e-8)
    s = sym_obj(fc, h, 1)
    P = cp.to_full((s.xi, s.U))
    from oracle.spectrum import eigenvalues
    rho = q.rho_full([eigenvalues(n)] * d)
    g = q.g_control(rho, alpha, 1.0, gamma_)
    assert np.all(P > 0)
    dev = float(np.max(np.abs(P * g - 1.0)))
    print(f"precond rank {h.info.rank_precond} max|p g - 1| = {dev:.3e} (setup grid {h.info.pc_err:.3e})")
    assert dev <= 0.5


@pytest.mark.parametrize("n,d,S", [(37, 2, 3), (70, 2, 5), (29, 3, 4), (66, 3, 2)])
@pytest.mark.parametrize("which", [0, 1])
def test_apply_and_precond_match_oracle_matvec(fc, n, d, S, which):
    """fc_apply / fc_precond equal the oracle's mode-wise mat-vec with the same symbol
    (eqn:Lap2DtimesX / eqn:Lap3DtimesX) to rounding, and the exact operator to 1e-9."""
    h = fc.fc_setup(n, d, 0.5, 1.0, 1e-2, 1e-8)
    X = fi.random_cp(n, d, S, seed=fi.seed_for(7, n + S))
    Xg = fc.CP.from_factors(*X)
    R = h.info.rank_symbol if which == 0 else h.info.rank_precond
    Y = fc.CP(d, n, R * S)
    (fc.fc_apply if which == 0 else fc.fc_precond)(h, Xg, Y)
    assert Y.rank == R * S
    s = sym_obj(fc, h, which)
    ref = cp.to_full(cp.apply_symbol(s, X))
    got = gpu_full(fc, h, Y)
    e = rel(got, ref)
    print(f"which={which} n={n} d={d} S={S}: rel err vs oracle mat-vec {e:.3e}")
    assert e < 1e-12
    if which == 0:
        exact = full.apply_full(cp.to_full(X), 0.5, 1.0, 1e-2)
        assert rel(got, exact) < 1e-9


@pytest.mark.parametrize("precision", [0, 2])
@pytest.mark.parametrize("n,d", [(45, 2), (33, 3), (130, 3), (1023, 3)])
def test_inner_and_to_full_match_oracle(fc, n, d, precision):
    """<X, Y> and the full expansion against the oracle; in form 3 the cross-Grams of the
    inner product run on the tensor cores (threshold 2^10 multiply-adds here, so every one
    does), within the same 1e-13 of ||X|| ||Y||."""
    h = fc.fc_setup(n, d, 0.5, 1.0, 1e-2, 1e-8, precision=precision,
                    max_rank=256 if n >= 1000 else 0)
    prev = fc.fc_set_schedule(tc_min_log2=10)
    X = fi.random_cp(n, d, 5 if n < 1000 else 180, seed=11)
    Y = fi.random_cp(n, d, 7 if n < 1000 else 200, seed=12)
    Xg, Yg = fc.CP.from_factors(*X), fc.CP.from_factors(*Y)
    v = fc.fc_inner(h, Xg, Yg)
    ref = cp.inner(X, Y)
    scale = cp.norm(X) * cp.norm(Y)
    fc.fc_set_schedule(prev)
    assert abs(v - ref) <= 1e-13 * scale
    if n < 1000:
        assert rel(gpu_full(fc, h, Xg), cp.to_full(X)) < 1e-14
    empty = fc.CP(d, n, 4)
    assert fc.fc_inner(h, empty, Xg) == 0.0


def _decaying_cp(n, d, R, seed, rate=0.5):
    xi, U = fi.random_cp(n, d, R, seed)
    xi = np.abs(xi) * rate ** np.arange(R)
    return xi, U


# Singular values below ~1e-8 sigma_max are not resolved by the FP64 Rayleigh-Ritz step on
# the Gram of the sketched side matrix (its eigenvalues are sigma^2, absolute error ~u
# sigma_max^2), so below eps = 1e-7 the achieved accuracy has a floor of a few 1e-8.
GRAM_FLOOR = 5e-8


def _trunc_case(n, d, R):
    if R <= 6:   # exact low rank, duplicated terms: truncation must be lossless
        base = fi.random_cp(n, d, 3, seed=21)
        return cp.axpy(base, 0.5, base)
    return _decaying_cp(n, d, R, seed=22)


@pytest.mark.parametrize("n,d,R,eps", [(40, 2, 6, 1e-10), (53, 3, 6, 1e-10), (70, 3, 30, 1e-6),
                                      (61, 2, 40, 1e-8), (100, 3, 14, 1e-7)])
def test_truncate_matches_oracle(fc, n, d, R, eps):
    """trunc (Section 5 RHOSVD / 2D reduced SVD) reproduces the tensor within its eps
    budget and agrees with the oracle's QR+SVD truncation in full form."""
    X = _trunc_case(n, d, R)
    h = fc.fc_setup(n, d, 0.5, 1.0, 1e-2, eps, max_rank=1024, max_input_rank=max(32, R))
    Xg = fc.CP.from_factors(*X)
    Y = fc.CP(d, n, 1024)
    fc.fc_truncate(h, Xg, eps, 1024, Y, normalize=True)
    Xf = cp.to_full(X)
    Yf = gpu_full(fc, h, Y)
    from oracle.truncate import truncate
    ref = truncate(X, eps, 1024)
    Rf = cp.to_full(ref)
    e_in, e_or, e_oracle_in = rel(Yf, Xf), rel(Yf, Rf), rel(Rf, Xf)
    print(f"n={n} d={d} R={R} eps={eps:g}: gpu rank {Y.rank} (oracle {len(ref[0])}); "
          f"|gpu-X|={e_in:.3e} |oracle-X|={e_oracle_in:.3e} |gpu-oracle|={e_or:.3e}")
    assert Y.rank >= 1
    floor = GRAM_FLOOR if eps < 1e-7 else 0.0
    assert e_in <= 2.0 * eps + floor + 1e-13
    assert e_or <= 3.0 * eps + floor + 1e-13


@pytest.mark.parametrize("n,d,R", [(70, 3, 30), (50, 3, 20)])
def test_truncate_rank_cap_matches_oracle(fc, n, d, R):
    """With the CP cap binding, both keep the 32 largest canonical terms of the core:
    the same (capped) error."""
    X = _decaying_cp(n, d, R, seed=22)
    h = fc.fc_setup(n, d, 0.5, 1.0, 1e-2, 1e-10, max_rank=32, max_input_rank=max(32, R))
    Y = fc.CP(d, n, 32)
    fc.fc_truncate(h, fc.CP.from_factors(*X), 1e-10, 32, Y, normalize=True)
    from oracle.truncate import truncate
    ref = truncate(X, 1e-10, 32)
    Xf = cp.to_full(X)
    e_g, e_o = rel(gpu_full(fc, h, Y), Xf), rel(cp.to_full(ref), Xf)
    print(f"capped n={n} d={d} R={R}: gpu rank {Y.rank} |gpu-X|={e_g:.4e} |oracle-X|={e_o:.4e}")
    assert Y.rank == len(ref[0]) == 32
    assert abs(e_g - e_o) <= 0.01 * e_o + 1e-9


@pytest.mark.parametrize("n,d,R,eps,rate", [(80, 3, 100, 1e-7, 0.3), (57, 2, 90, 1e-7, 0.7)])
def test_truncate_sketch_path_matches_oracle(fc, n, d, R, eps, rate):
    """More terms than the 64-column sketch: the randomised range of the side matrices
    must still capture every direction above the eps budget."""
    X = _decaying_cp(n, d, R, seed=23, rate=rate)
    h = fc.fc_setup(n, d, 0.5, 1.0, 1e-2, eps, max_rank=1024, max_input_rank=R)
    Xg = fc.CP.from_factors(*X)
    Y = fc.CP(d, n, 1024)
    fc.fc_truncate(h, Xg, eps, 1024, Y, normalize=True)
    from oracle.truncate import truncate
    ref = truncate(X, eps, 1024)
    Xf, Yf, Rf = cp.to_full(X), gpu_full(fc, h, Y), cp.to_full(ref)
    print(f"sketch n={n} d={d} R={R}: gpu rank {Y.rank} oracle {len(ref[0])} "
          f"|gpu-X|={rel(Yf, Xf):.3e} |oracle-X|={rel(Rf, Xf):.3e}")
    floor = GRAM_FLOOR if eps < 1e-7 else 0.0
    assert rel(Yf, Xf) <= 2.0 * eps + floor + 1e-13
    assert rel(Yf, Rf) <= 3.0 * eps + floor + 1e-13


@pytest.mark.parametrize("precision", [0, 1, 2])
@pytest.mark.parametrize("n,d,S,which,eps", [(31, 2, 3, 0, 1e-8), (40, 3, 4, 0, 1e-7),
                                             (40, 3, 4, 1, 1e-7), (64, 3, 8, 0, 1e-6),
                                             (127, 3, 8, 0, 1e-8)])
def test_apply_trunc_matches_oracle(fc, n, d, S, which, eps, precision):
    """trunc(fun(x)) / trunc(precond(x)) of Algorithm 1 with the Khatri-Rao columns kept
    implicit, against the oracle's truncation of the explicit mat-vec.  Both budgets are
    relative to the weight norm of the column-normalised representation.  Inputs are smooth
    separable Gaussians (the solver's right-hand sides)."""
    h = fc.fc_setup(n, d, 0.5, 1.0, 1e-2, eps, max_rank=1024, max_input_rank=32,
                    precision=precision)
    X = fi.gaussians_cp(n, d, S, np.random.default_rng(fi.seed_for(6, n + S)))
    Xg = fc.CP.from_factors(*X)
    Y = fc.CP(d, n, 1024)
    fc.fc_apply_trunc(h, which, Xg, eps, 1024, Y)
    s = sym_obj(fc, h, which)
    M = cp.apply_symbol(s, X)
    from oracle.truncate import truncate
    ref = truncate(M, eps, 1024)
    Mf, Yf, Rf = cp.to_full(M), gpu_full(fc, h, Y), cp.to_full(ref)
    # the RHOSVD budget is set by the weight norm ||xi||_2 of the column-normalised
    # (non-orthogonal) Khatri-Rao representation; with overlapping terms the error bound
    # grows with the tensor norm instead (projecting a mode costs the discarded energy times
    # the norm of the other modes' Khatri-Rao product): bound the error by the larger scale
    wn = max(float(np.linalg.norm(q.normalise_columns(*M)[0])), float(np.linalg.norm(cp.to_full(M))))
    ag, ao, agr = (np.linalg.norm(Yf - Mf) / wn, np.linalg.norm(Rf - Mf) / wn,
                   np.linalg.norm(Yf - Rf) / wn)
    print(f"apply_trunc prec={precision} which={which} n={n} d={d} S={S} K={len(M[0])}: gpu rank {Y.rank} "
          f"oracle {len(ref[0])} |gpu-M|/|xi|={ag:.3e} |oracle-M|/|xi|={ao:.3e} "
          f"|gpu-oracle|/|xi|={agr:.3e} (scale/|M| = {wn / np.linalg.norm(Mf):.1f})")
    floor = GRAM_FLOOR if eps < 1e-7 else 0.0
    assert ao <= 2.0 * eps
    assert ag <= 2.0 * eps + floor
    assert agr <= 3.0 * eps + floor


@pytest.mark.parametrize("n,d", [(63, 2), (50, 2), (31, 3), (50, 3), (127, 3), (255, 3)])
def test_full_solve_matches_oracle(fc, n, d):
    """Full-format eigenbasis solve (eqn:DiagFLaplace3D): by fast sine transforms where n + 1
    is a power of two (63, 31, 127, 255), by sine-matrix products otherwise (50)."""
    rng = np.random.default_rng(fi.seed_for(8, n))
    y = fi.gaussians_cp(n, d, 3, rng)
    b = cp.to_full(y)
    h = fc.fc_setup(n, d, 0.5, 1.0, 1e-2, 1e-8)
    # column-major (i_1 fastest) = numpy array with reversed axes, C order
    flat = torch.tensor(np.ascontiguousarray(b.transpose(*reversed(range(d)))).reshape(-1),
                        device="cuda")
    u = torch.empty_like(flat)
    tmp = torch.empty_like(flat)
    fc.fc_full_solve(h, flat, u, tmp)
    got = u.cpu().numpy().reshape([n] * d).transpose(*reversed(range(d)))
    ref = full.solve_full(b, 0.5, 1.0, 1e-2)
    e = rel(got, ref)
    print(f"full solve n={n} d={d}: rel err {e:.3e}")
    assert e < 1e-12


def test_full_solve_n1023_sine_modes_at_sampled_points(fc):
    """n = 1023 (1.07e9 points, 8.6 GB per array): grid sine modes have the closed-form
    solution sum_m c_m b_m / g(rho_m); 4000 sampled points of the GPU array against it."""
    n, d, alpha, gamma_ = 1023, 3, 0.5, 1e-3
    modes = [((1, 2, 3), 1.0), ((5, 17, 2), -0.5), ((300, 1, 40), 0.25)]
    y = fi.concat_cp(*[fi.sine_cp(n, m) for m, _ in modes])
    y = (np.array([c for _, c in modes]), y[1])
    h = fc.fc_setup(n, d, alpha, 1.0, gamma_, 1e-8)
    B = fc.CP.from_factors(*y)
    b = torch.empty(n ** 3, dtype=torch.float64, device="cuda")
    fc.fc_to_full(h, B, out=b)
    u = torch.empty_like(b)
    fc.fc_full_solve(h, b, u, b)
    rng = np.random.default_rng(8)
    idx = rng.integers(0, n, size=(4000, d))
    flat = torch.tensor(idx[:, 0] + n * idx[:, 1] + n * n * idx[:, 2], device="cuda")
    got = u[flat].cpu().numpy()
    x = fi.grid(n)
    N = n + 1
    ref = np.zeros(len(idx))
    for m, c in modes:
        rho = sum((2 * N) ** 2 * math.sin(math.pi * k / (2 * N)) ** 2 for k in m)
        g = rho ** (-alpha) + gamma_ * rho ** alpha
        ref += c / g * np.prod([np.sin(math.pi * m[l] * x[idx[:, l]]) for l in range(d)], axis=0)
    e = rel(got, ref)
    print(f"full solve n=1023 sine modes: sampled rel err {e:.2e}")
    assert e < 1e-12
    del b, u


@pytest.mark.parametrize("n,modes,alpha,gamma_", [(63, (1, 2, 3), 0.5, 1e-3),
                                                  (45, (3, 1), 0.25, 1e-1)])
def test_solve_sine_mode_exact(fc, n, modes, alpha, gamma_):
    """A grid sine mode is an eigenvector of A (Section 3.2): u = b / g(rho_m) exactly."""
    d = len(modes)
    y = fi.sine_cp(n, modes)
    h = fc.fc_setup(n, d, alpha, 1.0, gamma_, 1e-10)
    B = fc.CP.from_factors(*y)
    U = fc.CP(d, n, 32)
    info = fc.fc_solve(h, B, U, tol=1e-10)
    lam = [(2 * (n + 1)) ** 2 * math.sin(math.pi * m / (2 * (n + 1))) ** 2 for m in modes]
    rho = sum(lam)
    ref = cp.to_full(y) / (rho ** (-alpha) + gamma_ * rho ** alpha)
    e = rel(gpu_full(fc, h, U), ref)
    print(f"sine mode {modes}: iters {info.iters} rank {U.rank} rel err {e:.3e}")
    assert e < 1e-8


def _solve_vs_full(fc, prob, tol, eps, max_rank=32, precision=0):
    h = fc.fc_setup(prob.n, prob.d, prob.alpha, prob.beta, prob.gamma, eps, max_rank=max_rank,
                    precision=precision)
    B = fc.CP.from_factors(*prob.rhs())
    U = fc.CP(prob.d, prob.n, max_rank)
    info = fc.fc_solve(h, B, U, tol=tol, eps=eps)
    ref = full.solve_full(cp.to_full(prob.rhs()), prob.alpha, prob.beta, prob.gamma)
    e = rel(gpu_full(fc, h, U), ref)
    hist = [info.history[i] for i in range(min(info.iters, 8))]
    print(f"{prob.label} prec={precision}: iters {info.iters} relres {info.relres:.2e} rank {U.rank} "
          f"max rank {info.max_rank_seen} err vs full {e:.3e} hist {['%.1e' % x for x in hist]}")
    return info, e


def test_solve_config1_2d(fc):
    """2D, n=63, alpha=1/2, gamma=1e-2, two Gaussians: CP-PCG vs the full oracle."""
    prob = fi.config1()
    info, e = _solve_vs_full(fc, prob, 1e-8, 1e-8)
    assert info.status == 0
    assert e < 1e-7


@pytest.mark.parametrize("problem,precision", [(0, 0), (3, 0), (4, 0), (5, 0), (1, 1), (5, 1),
                                                (2, 2), (5, 2)])
def test_solve_config2_3d_n255(fc, problem, precision):
    """3D, n=255, 4 Gaussians + sine mode: CP-PCG vs the full oracle (16.6M points), at the
    workload's settings (eps = 1e-9, tol = 1e-8, cap 192): error <= 1e-6, with FP64,
    double-float and tensor-core digit-product contractions."""
    prob = fi.config2(problem)
    info, e = _solve_vs_full(fc, prob, prob.tol, prob.eps, max_rank=prob.max_rank,
                             precision=precision)
    assert info.status == 0
    assert e < 1e-6


def test_solve_batched_matches_independent_solves(fc):
    """fc_solve_batched runs independent problems concurrently (worker streams); every
    result equals the stand-alone fc_solve of the same problem within the solve accuracy,
    and each solves its own equation (full oracle)."""
    rng = np.random.default_rng(fi.seed_for(10))
    probs = [fi.Problem(47, 3, a, 1.0, g, fi.gaussians_cp(47, 3, 3, rng), eps=1e-9, tol=1e-8,
                        max_rank=96) for a, g in [(0.25, 1e-1), (0.5, 1e-3), (0.75, 1e-2)]]
    hs = [fc.fc_setup(p.n, 3, p.alpha, 1.0, p.gamma, p.eps, max_rank=p.max_rank) for p in probs]
    Bs = [fc.CP.from_factors(*p.rhs()) for p in probs]
    Ub = [fc.CP(3, p.n, p.max_rank) for p in probs]
    infos = fc.fc_solve_batched(hs, Bs, Ub, tol=[p.tol for p in probs],
                                eps=[p.eps for p in probs])
    torch.cuda.synchronize()
    for p, h, B, U, info in zip(probs, hs, Bs, Ub, infos):
        Us = fc.CP(3, p.n, p.max_rank)
        fc.fc_solve(h, B, Us, tol=p.tol, eps=p.eps)
        ub, us = gpu_full(fc, h, U), gpu_full(fc, h, Us)
        ref = full.solve_full(cp.to_full(p.rhs()), p.alpha, 1.0, p.gamma)
        print(f"batched a={p.alpha} g={p.gamma}: iters {info.iters} |b-s|={rel(ub, us):.2e} "
              f"|b-full|={rel(ub, ref):.2e}")
        assert info.status == 0
        assert rel(ub, ref) <= 1e-6 and rel(us, ref) <= 1e-6
        assert rel(ub, us) <= 2.0 * max(rel(ub, ref), rel(us, ref)) + 1e-12
    with pytest.raises(fc.FCError):
        fc.fc_solve_batched([hs[0], hs[0]], Bs[:2], Ub[:2])


def test_batched_mixed_problems(fc):
    """Batching form with uneven problems: 3D n in {127, 255, 511}, alpha ~ U[0.1, 0.9], gamma
    log-uniform in [1e-4, 1], rank 1-8 Gaussians (the mixed-batch recipe at its 1e-6
    settings), more problems than the worker pool has threads, tensor-core form.  Every
    solution against the exact solution over the whole grid (oracle.eigerr): error <= 1e-6."""
    from oracle import eigerr
    probs = [p for p in (fi.config4(i) for i in range(80)) if p.n <= 511][:18]
    hs = [fc.fc_setup(p.n, p.d, p.alpha, p.beta, p.gamma, p.eps, max_rank=p.max_rank,
                      max_tucker=p.max_tucker, precision=2) for p in probs]
    Bs = [fc.CP.from_factors(*p.rhs()) for p in probs]
    Us = [fc.CP(p.d, p.n, p.max_rank) for p in probs]
    infos = fc.fc_solve_batched(hs, Bs, Us, tol=[p.tol for p in probs],
                                eps=[p.eps for p in probs], raise_on_fail=False)
    worst = 0.0
    for p, U, info in zip(probs, Us, infos):
        e = eigerr.control_error(U.factors(), p.rhs(), p.alpha, p.beta, p.gamma)[0]
        worst = max(worst, e)
        print(f"{p.label} status {info.status} rank {U.rank} iters {info.iters} err {e:.1e}")
        assert info.status == 0 and e <= 1e-6
    print(f"{len(probs)} mixed problems, worst error {worst:.1e}")


@pytest.mark.parametrize("problem,precision", [(5, 2), (0, 0)])
def test_spectral_resident_solve_matches(fc, problem, precision):
    """The spectral-resident iteration (iterates in the DST-I eigenbasis, one transform at
    entry and exit) reaches the same solution as the per-step path: both against the
    full-format oracle, and against each other."""
    prob = fi.config2(problem)
    h = fc.fc_setup(prob.n, prob.d, prob.alpha, prob.beta, prob.gamma, prob.eps,
                    max_rank=prob.max_rank, precision=precision)
    B = fc.CP.from_factors(*prob.rhs())
    ref = full.solve_full(cp.to_full(prob.rhs()), prob.alpha, prob.beta, prob.gamma)
    out = {}
    for spectral in (False, True):
        U = fc.CP(prob.d, prob.n, prob.max_rank)
        fc.fc_solve(h, B, U, tol=prob.tol, eps=prob.eps, spectral=spectral)   # warm
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        info = fc.fc_solve(h, B, U, tol=prob.tol, eps=prob.eps, spectral=spectral)
        e1.record()
        e1.synchronize()
        got = gpu_full(fc, h, U)
        out[spectral] = got
        e = rel(got, ref)
        print(f"{prob.label} prec={precision} spectral={spectral}: iters {info.iters} "
              f"rank {U.rank} err {e:.2e} {e0.elapsed_time(e1):.1f} ms")
        assert info.status == 0 and e < 1e-6
    assert rel(out[True], out[False]) < 1e-6
