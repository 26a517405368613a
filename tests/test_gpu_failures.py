"""Failure statuses of the C ABI, each provoked from the host, and the next call on the same
handle succeeding (Section 3.3: Algorithm 1 stops when k_max is reached; the paper's tables
mark solves that did not converge within 100 iterations).  No test faults, traps or hangs
the GPU: the expired-wait status comes from a lowered poll limit (fc_set_wait_limit), after
which the tensor-core kernel stops producing, drains the MMAs it issued and returns."""
import numpy as np
import pytest
import torch

import fc_inputs as fi

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def fc():
    import paper_1809_01971_gb300 as m
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    m.lib()
    return m


def _c1(fc, precision=0):
    prob = fi.config1()
    h = fc.fc_setup(prob.n, prob.d, prob.alpha, prob.beta, prob.gamma, prob.eps,
                    precision=precision)
    return prob, h, fc.CP.from_factors(*prob.rhs()), fc.CP(prob.d, prob.n, 32)


def _ok_solve(fc, prob, h, B, U):
    info = fc.fc_solve(h, B, U, tol=prob.tol, eps=prob.eps)
    assert info.status == fc.fc.FC_OK and info.relres <= prob.tol and U.rank > 0
    return info


def test_enoconv_at_kmax_then_the_handle_solves(fc):
    prob, h, B, U = _c1(fc)
    info = fc.fc_solve(h, B, U, tol=prob.tol, eps=prob.eps, kmax=1, raise_on_fail=False)
    assert info.status == fc.fc.FC_ENOCONV and info.iters == 1 and info.relres > prob.tol
    with pytest.raises(fc.FCError) as ex:
        fc.fc_solve(h, B, U, tol=prob.tol, eps=prob.eps, kmax=1)
    assert ex.value.code == fc.fc.FC_ENOCONV
    assert _ok_solve(fc, prob, h, B, U).iters > 1


def test_enan_from_a_non_finite_right_hand_side(fc):
    prob, h, B, U = _c1(fc)
    xi, Us = prob.rhs()
    bad = [u.copy() for u in Us]
    bad[1][7, 0] = np.nan
    Bn = fc.CP.from_factors(xi, bad)
    info = fc.fc_solve(h, Bn, U, tol=prob.tol, eps=prob.eps, raise_on_fail=False)
    assert info.status == fc.fc.FC_ENAN
    _ok_solve(fc, prob, h, B, U)


def test_etimeout_from_an_expired_wait_then_the_handle_solves(fc):
    """n = 255 3D in the tensor-core form: its large contractions run K ranges of several
    pipeline stages, whose producer waits give up at once with the limit at 0."""
    prob = fi.config2(0)
    h = fc.fc_setup(prob.n, prob.d, prob.alpha, prob.beta, prob.gamma, prob.eps,
                    max_rank=prob.max_rank, precision=2)
    B = fc.CP.from_factors(*prob.rhs())
    U = fc.CP(prob.d, prob.n, prob.max_rank)
    prev = fc.fc_set_wait_limit(0)
    try:
        with pytest.raises(fc.FCError) as ex:
            fc.fc_solve(h, B, U, tol=prob.tol, eps=prob.eps)
        assert ex.value.code == fc.fc.FC_ETIMEOUT
    finally:
        fc.fc_set_wait_limit(prev)
    assert prev > 0
    info = fc.fc_solve(h, B, U, tol=prob.tol, eps=prob.eps)
    assert info.status == fc.fc.FC_OK and info.relres <= prob.tol


def test_etimeout_in_the_contraction_entry_point(fc):
    """fc_dgemm in the tensor-core form: FC_ETIMEOUT with the limit at 0, the exact product
    again after the limit is restored."""
    # 1024 x 1024 output tiles over K = 4096: K ranges of 13 pipeline stages per CTA, so the
    # producers wait on the MMAs of earlier stages
    g = torch.Generator(device="cpu").manual_seed(5)
    A = torch.randn(1024, 4096, generator=g, dtype=torch.float64).cuda()
    Bm = torch.randn(4096, 1024, generator=g, dtype=torch.float64).cuda()
    prev = fc.fc_set_wait_limit(0)
    try:
        with pytest.raises(fc.FCError) as ex:
            fc.fc_dgemm(A, Bm, precision=2)
        assert ex.value.code == fc.fc.FC_ETIMEOUT
    finally:
        fc.fc_set_wait_limit(prev)
    C = fc.fc_dgemm(A, Bm, precision=2)
    ref = A.cpu() @ Bm.cpu()
    assert float((C.cpu() - ref).abs().max()) <= 4096 * 2.0**-52 * float(A.abs().max() * Bm.abs().max())


def test_argument_errors_leave_the_handle_usable(fc):
    prob, h, B, U = _c1(fc)
    small = fc.CP(prob.d, prob.n, 4)
    with pytest.raises(fc.FCError) as ex:
        fc.fc_solve(h, B, small, tol=prob.tol)
    assert ex.value.code == fc.fc.FC_ERANK
    with pytest.raises(fc.FCError) as ex:
        fc.fc_solve(h, B, U, tol=prob.tol, precision=7)
    assert ex.value.code == fc.fc.FC_EINVAL
    with pytest.raises(fc.FCError) as ex:
        fc.fc_set_wait_limit(-1)
    assert ex.value.code == fc.fc.FC_EINVAL
    _ok_solve(fc, prob, h, B, U)
