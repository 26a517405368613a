"""The CUDA CP-PCG solve (Algorithm 1) against the oracle: the oracle's own CP-PCG at the same
settings, and the exact full-format solution (eqn:DiagFLaplace3D) at the sizes of every
workload, n = 63 ... 8191.

Accuracy that truncated PCG can reach.  Stopping at a relative residual tol and truncating
every update to relative accuracy eps leaves a residual error of order max(eps, tol) ||b||;
the operator maps it back to the solution with at most its condition number
kappa = max g / min g over [rho_min, rho_max] (g the operator's symbol), so
||u - u*|| / ||u*|| <= c kappa max(eps, tol) with c of order one.  Tests state either that
bound (kappa computed from the grid) or, where the settings are chosen for it, the target
itself: max(eps, 1e-8) for the plain solve, 1e-6 for the workloads that report solves/s at
1e-6.  Errors against the exact solution come from oracle.eigerr (the whole eigen-index grid
for n^3 <= 1.2e9, the low-index box with an exact remainder beyond that).
"""
import math

import numpy as np
import pytest
import torch

import fc_inputs as fi
from oracle import cp, eigerr, full, pcg, quadrature as q
from oracle.spectrum import eigenvalues

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def fc():
    import paper_1809_01971_gb300 as m
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    m.lib()
    return m


def kappa(n, d, alpha, beta, gamma_):
    """max g / min g of g(rho) = beta^2 rho^-alpha + gamma rho^alpha on the grid's rho range."""
    lam = eigenvalues(n)
    rmin, rmax = d * lam[0], d * lam[-1]
    rs = np.exp(np.linspace(math.log(rmin), math.log(rmax), 20001))
    g = beta**2 * rs ** (-alpha) + gamma_ * rs**alpha
    return float(g.max() / g.min())


def gpu_solve(fc, prob, eps, tol, cap, precision=None, spectral=False, h=None):
    if h is None:
        h = fc.fc_setup(prob.n, prob.d, prob.alpha, prob.beta, prob.gamma, eps, max_rank=cap)
    B = fc.CP.from_factors(*prob.rhs())
    U = fc.CP(prob.d, prob.n, cap)
    info = fc.fc_solve(h, B, U, tol=tol, eps=eps, precision=precision, spectral=spectral,
                       raise_on_fail=False)
    return h, U, info


def exact_error(prob, U):
    return eigerr.control_error(U.factors(), prob.rhs(), prob.alpha, prob.beta, prob.gamma)[0]


def test_config1_at_its_settings_within_the_attainable_bound(fc):
    """2D, n = 63 (C1) at eps = tol = 1e-8: error <= kappa max(eps, tol) (kappa ~ 9)."""
    prob = fi.config1()
    k = kappa(prob.n, prob.d, prob.alpha, prob.beta, prob.gamma)
    _, U, info = gpu_solve(fc, prob, 1e-8, 1e-8, 32)
    e = exact_error(prob, U)
    print(f"C1 eps=tol=1e-8: iters {info.iters} rank {U.rank} err {e:.2e} kappa {k:.1f}")
    assert info.status == 0
    assert e <= k * 1e-8


def test_config1_meets_max_eps_1e8(fc):
    """2D, n = 63 (C1) at eps = tol = 1e-9: the plain solve's target max(eps, 1e-8) = 1e-8."""
    prob = fi.config1()
    _, U, info = gpu_solve(fc, prob, 1e-9, 1e-9, 32)
    e = exact_error(prob, U)
    print(f"C1 eps=tol=1e-9: iters {info.iters} rank {U.rank} err {e:.2e}")
    assert info.status == 0
    assert e <= 1e-8


def _oracle_case(name):
    if name == "c1":
        return fi.config1(), 1e-9, 1e-9, 32
    rng = np.random.default_rng(fi.seed_for(11))
    y = fi.gaussians_cp(31, 3, 3, rng)
    # rank cap 256: at cap 64 both solvers stop at the cap's own error (2.2e-7), far above eps
    return fi.Problem(31, 3, 0.5, 1.0, 1e-2, y, label="3d_n31"), 1e-9, 1e-9, 256


@pytest.mark.parametrize("name", ["c1", "3d_n31"])
def test_cp_pcg_matches_oracle_cp_pcg(fc, name):
    """Algorithm 1 on the GPU and in the oracle at identical eps, tol, rank cap and
    preconditioner rank (24): both solutions within the attainable bound of the exact one,
    hence within twice of each other; the iteration counts agree to one step."""
    prob, eps, tol, cap = _oracle_case(name)
    fs = q.control_symbol(prob.n, prob.d, prob.alpha, prob.beta, prob.gamma, 1e-10)
    ps = q.precond_symbol(prob.n, prob.d, prob.alpha, prob.beta, prob.gamma, 24)
    res = pcg.pcg(fs, ps, prob.rhs(), eps, tol, cap)
    _, U, info = gpu_solve(fc, prob, eps, tol, cap)
    assert U.rank < cap          # the cap did not decide the result
    k = kappa(prob.n, prob.d, prob.alpha, prob.beta, prob.gamma)
    ref = full.solve_full(cp.to_full(prob.rhs()), prob.alpha, prob.beta, prob.gamma)
    ug, uo = fc.fc_to_full(fc.fc_setup(prob.n, prob.d, prob.alpha, prob.beta, prob.gamma, eps),
                           U).cpu().numpy(), cp.to_full(res.X)
    nref = np.linalg.norm(ref)
    eg, eo = np.linalg.norm(ug - ref) / nref, np.linalg.norm(uo - ref) / nref
    diff = np.linalg.norm(ug - uo) / nref
    print(f"{name}: gpu iters {info.iters} err {eg:.2e} | oracle iters {res.iters} err {eo:.2e}"
          f" | |gpu-oracle| {diff:.2e} kappa {k:.1f}")
    assert info.status == 0 and res.status == "ok"
    bound = k * max(eps, tol)
    assert eg <= bound and eo <= bound
    assert diff <= 2 * bound
    assert abs(info.iters - res.iters) <= 1


# ---- the metric's workloads: n = 1023 (precision forms), the mixed batch, n = 8191 -------------
# Settings reaching 1e-6 against the exact solution: fc_inputs.TARGET_SETTINGS (tol 1e-7,
# eps 1e-8: a residual tolerance one decade below the target covers the operator's
# amplification of the residual error on these right-hand sides; Tucker ranks up to 56 and CP
# ranks up to 256).

FORMS = [(0, False), (1, False), (2, False), (2, True)]   # (precision, spectral-resident)


def test_config3_n1023_every_form_meets_1e6(fc):
    """3D, n = 1023 (1.07e9 points), 8 Gaussians, alpha = 1/2, gamma = 1e-3: FP64, double-float
    and tensor-core contractions (and the spectral-resident iteration) against the exact
    solution over the whole grid: error <= 1e-6."""
    prob = fi.config3()
    h = fc.fc_setup(prob.n, prob.d, prob.alpha, prob.beta, prob.gamma, prob.eps,
                    max_rank=prob.max_rank, max_tucker=prob.max_tucker)
    for precision, spectral in FORMS:
        _, U, info = gpu_solve(fc, prob, prob.eps, prob.tol, prob.max_rank, precision, spectral, h)
        e = exact_error(prob, U)
        print(f"C3 precision {precision} spectral {spectral}: iters {info.iters} rank {U.rank} "
              f"err {e:.2e}")
        assert info.status == 0
        assert e <= 1e-6


def _one_per_class():
    seen, out = set(), []
    for i in range(512):
        p = fi.config4(i)
        if p.n not in seen:
            seen.add(p.n)
            out.append(p)
    return sorted(out, key=lambda p: p.n)


@pytest.mark.parametrize("precision,spectral", [(0, False), (2, True)])
def test_config4_batch_every_grid_class_meets_1e6(fc, precision, spectral):
    """The mixed batch (n in {127, 255, 511, 1023, 2047}, alpha ~ U[0.1, 0.9], gamma
    log-uniform in [1e-4, 1], rank 1-8 Gaussians): one problem of every grid class solved
    together by fc_solve_batched, each against its exact solution: error <= 1e-6."""
    probs = _one_per_class()
    assert [p.n for p in probs] == [127, 255, 511, 1023, 2047]
    hs = [fc.fc_setup(p.n, p.d, p.alpha, p.beta, p.gamma, p.eps, max_rank=p.max_rank,
                      max_tucker=p.max_tucker) for p in probs]
    Bs = [fc.CP.from_factors(*p.rhs()) for p in probs]
    Us = [fc.CP(p.d, p.n, p.max_rank) for p in probs]
    infos = fc.fc_solve_batched(hs, Bs, Us, tol=[p.tol for p in probs],
                                eps=[p.eps for p in probs], precision=precision,
                                spectral=spectral)
    for p, U, info in zip(probs, Us, infos):
        e = exact_error(p, U)
        print(f"{p.label}: iters {info.iters} rank {U.rank} err {e:.2e}")
        assert info.status == 0
        assert e <= 1e-6


@pytest.mark.parametrize("problem", [0, 1])
def test_config5_n8191_gaussians_against_the_exact_solution(fc, problem):
    """n = 8191 (5.5e11 points, no full format), gamma = 1e-4, alpha = 0.25 / 0.75, tensor-core
    form, with stall detection: the Gaussians of the workload's draw that vanish at the
    boundary (width <= 0.03), whose sine transforms decay fast enough for the exact error to be
    summed over a low-index box of the eigen-grid with the remainder bounded (oracle.eigerr).
    Widths down to 0.01 need more than the 56 Tucker directions and 256 CP terms the solver
    keeps: the iteration stalls with the error near 1e-3, which this test bounds (2e-3), so
    that the limit is measured on every run; it is not the 1e-6 of the smaller grids."""
    prob = fi.config5(problem, narrow_only=True)
    assert 2 <= len(prob.rhs()[0]) < 16
    h = fc.fc_setup(prob.n, prob.d, prob.alpha, prob.beta, prob.gamma, prob.eps,
                    max_rank=prob.max_rank, max_tucker=prob.max_tucker, precision=2)
    B = fc.CP.from_factors(*prob.rhs())
    U = fc.CP(prob.d, prob.n, prob.max_rank)
    info = fc.fc_solve(h, B, U, tol=prob.tol, eps=prob.eps, spectral=True, stall=8,
                       raise_on_fail=False)
    e = exact_error(prob, U)
    print(f"{prob.label}: terms {len(prob.rhs()[0])} status {info.status} iters {info.iters} "
          f"rank {U.rank} relres {info.relres:.1e} err {e:.2e}")
    assert info.status in (0, fc.fc.FC_ENOCONV)
    assert e <= 2e-3


@pytest.mark.parametrize("problem", [0, 1])
def test_config5_n8191_full_draw_keeps_its_best_iterate(fc, problem):
    """All 16 Gaussians of the n = 8191 workload (widths 0.01 ... 0.15), stall detection on:
    the solve ends at the iterate of the smallest residual (no divergence past it)."""
    prob = fi.config5(problem)
    h = fc.fc_setup(prob.n, prob.d, prob.alpha, prob.beta, prob.gamma, prob.eps,
                    max_rank=prob.max_rank, max_tucker=prob.max_tucker, precision=2)
    B = fc.CP.from_factors(*prob.rhs())
    U = fc.CP(prob.d, prob.n, prob.max_rank)
    info = fc.fc_solve(h, B, U, tol=prob.tol, eps=prob.eps, spectral=True, stall=8,
                       raise_on_fail=False)
    hist = [info.history[i] for i in range(min(info.iters, 128))]
    print(f"{prob.label}: status {info.status} iters {info.iters} rank {U.rank} "
          f"relres {info.relres:.1e} max rank {info.max_rank_seen} tucker max {info.tucker_max}")
    assert info.status in (0, fc.fc.FC_ENOCONV)
    assert info.relres == pytest.approx(min(hist)) and info.relres < 1e-2
