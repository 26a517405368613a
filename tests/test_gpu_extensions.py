"""State recovery (eqn:State), the directionally fractional Laplacian (Remark after
Lemma 4.1), the test operators of Section 6 (A^alpha, I + A^(2 alpha), A^alpha + A^-alpha
with their preconditioners) and separable variable coefficients (Remark on generalised
directionally fractional operators) through the C ABI, against the CPU FP64 oracle's
full-format definitions."""
import numpy as np
import pytest
import torch

import fc_inputs as fi
from oracle import cp, full

pytestmark = pytest.mark.gpu


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(np.asarray(b)))


@pytest.mark.parametrize("n,d,alpha", [(40, 3, 0.5), (63, 2, 0.25), (33, 3, 1.0)])
def test_state_matches_oracle(n, d, alpha):
    """y = trunc(beta A^-alpha u): the state symbol (beta rho^-alpha, R_minus terms) applied
    to a smooth CP tensor, against the full-format spectral definition."""
    import paper_1809_01971_gb300 as fc
    beta = 1.5
    h = fc.fc_setup(n, d, alpha, beta, 1e-2, 1e-10, max_rank=512)
    U = fi.gaussians_cp(n, d, 3, np.random.default_rng(fi.seed_for(11, n)))
    Y = fc.CP(d, n, 512)
    fc.fc_state(h, fc.CP.from_factors(*U), 1e-10, 512, Y)
    got = fc.fc_to_full(h, Y).cpu().numpy()
    ref = full.state_full(cp.to_full(U), alpha, beta)
    e = rel(got, ref)
    print(f"state n={n} d={d} alpha={alpha}: rank {Y.rank} (R_minus {h.info.rank_minus}) err {e:.2e}")
    assert e < 1e-8


def test_solve_then_state_2d():
    """Control u from the CP-PCG solve, then the state y = beta A^-alpha u (eqn:L_alp_state):
    both against the oracle's full-format solution."""
    import paper_1809_01971_gb300 as fc
    prob = fi.config1()
    h = fc.fc_setup(prob.n, prob.d, prob.alpha, prob.beta, prob.gamma, prob.eps)
    Ug = fc.CP(prob.d, prob.n, 32)
    fc.fc_solve(h, fc.CP.from_factors(*prob.rhs()), Ug, tol=prob.tol)
    Y = fc.CP(prob.d, prob.n, 32)
    fc.fc_state(h, Ug, 1e-10, 32, Y)
    u_ref = full.solve_full(cp.to_full(prob.rhs()), prob.alpha, prob.beta, prob.gamma)
    y_ref = full.state_full(u_ref, prob.alpha, prob.beta)
    e = rel(fc.fc_to_full(h, Y).cpu().numpy(), y_ref)
    print(f"state of the solved control: err {e:.2e}")
    assert e < 1e-6


@pytest.mark.parametrize("n,d,alpha,gamma_", [(31, 3, 0.3, 1e-2), (47, 3, 0.7, 1e-3),
                                              (63, 2, 0.5, 1e-1)])
def test_directional_operator_solve(n, d, alpha, gamma_):
    """(beta^2 A_(alpha)^-1 + gamma A_(alpha)) u = b with A_(alpha) = sum_l (-Delta_l)^alpha:
    the CP-PCG solve and the full-format eigenbasis solve against the oracle."""
    import paper_1809_01971_gb300 as fc
    y = fi.gaussians_cp(n, d, 3, np.random.default_rng(fi.seed_for(12, n)))
    b = cp.to_full(y)
    ref = full.solve_full_directional(b, alpha, 1.0, gamma_)
    h = fc.fc_setup(n, d, alpha, 1.0, gamma_, 1e-9, max_rank=128, directional=True)
    assert h.info.sym_err < 1e-9
    Ug = fc.CP(d, n, 128)
    info = fc.fc_solve(h, fc.CP.from_factors(*y), Ug, tol=1e-9, eps=1e-9)
    e_cp = rel(fc.fc_to_full(h, Ug).cpu().numpy(), ref)
    flat = torch.tensor(np.ascontiguousarray(b.transpose(*reversed(range(d)))).reshape(-1), device="cuda")
    u = torch.empty_like(flat)
    fc.fc_full_solve(h, flat, u, torch.empty_like(flat))
    got_full = u.cpu().numpy().reshape([n] * d).transpose(*reversed(range(d)))
    e_full = rel(got_full, ref)
    print(f"directional n={n} d={d} alpha={alpha} gamma={gamma_}: iters {info.iters} rank {Ug.rank} "
          f"CP err {e_cp:.2e} full err {e_full:.2e}")
    assert e_full < 1e-12
    assert e_cp < 1e-6


@pytest.mark.parametrize("kind,pkind,d,n,alpha", [
    (1, 0, 2, 255, 0.5), (1, 1, 2, 255, 0.5), (2, 0, 2, 255, 0.5), (0, 0, 2, 255, 0.5),
    (1, 1, 3, 64, 0.5), (2, 0, 3, 64, 0.1), (0, 0, 3, 64, 0.1), (1, 0, 3, 64, 0.1)])
def test_section6_operators_solve(kind, pkind, d, n, alpha):
    """L u = b for the operators of Tables 6.1-6.4: A^alpha (kind 1), I + A^(2 alpha) (kind 2)
    and A^alpha + A^-alpha (kind 0 at beta = gamma = 1), preconditioned by the least-squares
    exponential sum of 1/g (pkind 0) or by the exponential sum of rho^-alpha (pkind 1, the
    symbol g_1, exact for A^alpha).  CP-PCG vs the oracle's eigenbasis solve."""
    import paper_1809_01971_gb300 as fc
    y = fi.gaussians_cp(n, d, 3, np.random.default_rng(fi.seed_for(13, n + 10 * kind)))
    cap = 96 if d == 2 else 192
    h = fc.fc_setup(n, d, alpha, 1.0, 1.0, 1e-11, max_rank=cap, op_kind=kind,
                    precond_kind=pkind)
    U = fc.CP(d, n, cap)
    info = fc.fc_solve(h, fc.CP.from_factors(*y), U, tol=1e-10, eps=1e-11)
    ref = full.solve_full_op(cp.to_full(y), kind, alpha)
    e = rel(fc.fc_to_full(h, U).cpu().numpy(), ref)
    print(f"operator kind {kind} precond {pkind} d={d} n={n} alpha={alpha}: iters {info.iters} "
          f"rank {U.rank} err {e:.2e} (symbol err {h.info.sym_err:.1e}, precond max|pg-1| "
          f"{h.info.pc_err:.2f})")
    assert info.status == 0 and e < 1e-6
    if kind == 1 and pkind == 1 and info.max_rank_seen < cap:
        assert info.iters <= 2          # g_1 is the exact inverse symbol of A^alpha
    if kind != 0:                       # the state y = beta A^-alpha u needs the control operator
        with pytest.raises(fc.FCError) as ex:
            fc.fc_state(h, U, 1e-8, cap, fc.CP(d, n, cap))
        assert ex.value.code == fc.fc.FC_EINVAL


def test_section6_iterations_vs_preconditioner_rank():
    """Trend of Table 6.1 (2D, alpha = 1/2, A^alpha + A^-alpha, residual 1e-6): PCG iterations
    against the rank r of the exponential-sum preconditioner, r in {1, 5, 6, 10}.  The
    paper's right-hand side is not given, so only the trend is checked: ranks 5, 6 and 10
    converge within the paper's range of a few iterations and rank 10 needs the fewest.  Rank
    1 is a scaled identity (max |p g - 1| = 0.985 on the spectrum): its run takes ~70
    iterations, over which the truncations' perturbations stop further progress near 2e-6;
    with stall detection it returns its best iterate, which must be within 1e-5."""
    import paper_1809_01971_gb300 as fc
    n, d, alpha = 255, 2, 0.5
    y = fi.gaussians_cp(n, d, 3, np.random.default_rng(fi.seed_for(14, n)))
    ref = full.solve_full_op(cp.to_full(y), 0, alpha)
    its = {}
    for r in (1, 5, 6, 10):
        h = fc.fc_setup(n, d, alpha, 1.0, 1.0, 1e-8, max_rank=128, precond_rank=r)
        U = fc.CP(d, n, 128)
        info = fc.fc_solve(h, fc.CP.from_factors(*y), U, tol=1e-6, eps=1e-8, kmax=200,
                           stall=8, raise_on_fail=False)
        e = rel(fc.fc_to_full(h, U).cpu().numpy(), ref)
        its[r] = info.iters
        print(f"precond rank {r}: max|pg-1| {h.info.pc_err:.3f} status {info.status} "
              f"iters {info.iters} relres {info.relres:.1e} err {e:.1e}")
        if r == 1:
            assert info.relres <= 1e-5 and e < 1e-4
        else:
            assert info.status == 0 and info.iters <= 10 and e < 1e-5
    assert its[10] <= min(its[5], its[6]) <= its[1]


def _coef(n, kind):
    x = (np.arange(n + 1) + 0.5) / (n + 1)
    return {0: 1.0 + 0.5 * np.sin(2 * np.pi * x), 1: np.exp(x), 2: 0.3 + x**2}[kind]


@pytest.mark.parametrize("n,d,kinds,alpha,gamma_,precision", [
    (63, 2, (0, 1), 0.5, 1e-2, 0), (31, 3, (0, None, 2), 0.5, 1e-2, 0),
    (47, 3, (1, 2, 0), 0.75, 1e-3, 2)])
def test_variable_coefficients(n, d, kinds, alpha, gamma_, precision):
    """Mode l carries the stiffness matrix of -(a_l u')' (a_l = 1 + sin/2, e^x, 0.3 + x^2, or
    constant): the CP-PCG solve and the full-format solve against the oracle's per-mode
    eigenbasis solve."""
    import paper_1809_01971_gb300 as fc
    coeffs = [None if k is None else _coef(n, k) for k in kinds]
    y = fi.gaussians_cp(n, d, 3, np.random.default_rng(fi.seed_for(15, n)))
    b = cp.to_full(y)
    ref = full.solve_full_varcoef(b, coeffs, 0, alpha, 1.0, gamma_)
    h = fc.fc_setup(n, d, alpha, 1.0, gamma_, 1e-10, max_rank=128, precision=precision,
                    coeff=coeffs)
    U = fc.CP(d, n, 128)
    info = fc.fc_solve(h, fc.CP.from_factors(*y), U, tol=1e-9, eps=1e-10)
    e = rel(fc.fc_to_full(h, U).cpu().numpy(), ref)
    # full-format solve through the same per-mode bases
    flat = torch.tensor(np.ascontiguousarray(b.transpose(*reversed(range(d)))).reshape(-1),
                        device="cuda")
    u = torch.empty_like(flat)
    tmp = torch.empty_like(flat)
    fc.fc_full_solve(h, flat, u, tmp)
    ef = rel(u.cpu().numpy().reshape([n] * d).transpose(*reversed(range(d))), ref)
    print(f"variable coefficients n={n} d={d} kinds={kinds} precision {precision}: iters "
          f"{info.iters} rank {U.rank} CP err {e:.2e} full-format err {ef:.2e} "
          f"(rho in [{h.info.rho_min:.3g}, {h.info.rho_max:.3g}])")
    assert info.status == 0 and e < 1e-7
    assert ef < 1e-9
