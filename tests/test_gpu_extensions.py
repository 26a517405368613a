"""State recovery (eqn:State) and the directionally fractional Laplacian (Remark after
Lemma 4.1) through the C ABI, against the CPU FP64 oracle's full-format definitions."""
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
