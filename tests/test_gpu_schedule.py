"""Launch schedules and the batched form's autotuner on the GPU, through the C ABI.

A schedule changes tile shapes, K splits, the tensor-core threshold and the batch policy, never
the arithmetic: the contraction kernel under extreme schedules against the exact product (in
extended precision on the host), CP-PCG solves under them against the full-format oracle, and the autotuner's own run
(every solution of its last batch against the exact solution over the whole grid)."""
import numpy as np
import pytest
import torch

import fc_inputs as fi
from oracle import cp, full

pytestmark = pytest.mark.gpu

# the two corners of the autotuner's search space, and the default
SPLIT_ALL = dict(gemm_cover=1, gemm_split=8, tc_split=1, tc_min_log2=20, workers=8, order=1)
SPLIT_NONE = dict(gemm_cover=16, gemm_split=0, tc_split=0, tc_min_log2=26, workers=32, order=0)
DEFAULT = dict(gemm_cover=8, gemm_split=4, tc_split=1, tc_min_log2=22, workers=16, order=0)


@pytest.fixture(scope="module")
def fc():
    import paper_1809_01971_gb300 as m
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    m.lib()
    return m


@pytest.fixture(autouse=True)
def _restore_schedule(fc):
    prev = fc.fc_get_schedule()
    yield
    fc.fc_set_schedule(prev)


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / max(np.linalg.norm(b), 1e-300))


def _bound(form, A, B, K):
    """Element-wise error bounds of the three forms (those of the contraction-kernel tests):
    FP64 2 K u |A||B|, double-float 4 K 2^-46 |A||B|, tensor-core digits
    2 K u max|A_i,:| max|B_:,j|."""
    if form == 2:
        return 2.0 * K * 2.0 ** -53 * np.outer(np.abs(A).max(axis=1), np.abs(B).max(axis=0))
    return (4.0 * K * 2.0 ** -46 if form == 1 else 2.0 * K * 2.0 ** -53) * (np.abs(A) @ np.abs(B))


@pytest.mark.parametrize("precision", [0, 1, 2])
@pytest.mark.parametrize("M,N,K", [(100, 100, 3000), (257, 61, 1500), (33, 700, 129)])
def test_dgemm_under_every_schedule(fc, precision, M, N, K):
    """fc_dgemm (the contraction kernel of every form) under the split-everything,
    split-nothing and default schedules, ragged sizes, K split into many ranges or none: each
    within its form's bound of the exact product (extended precision on the host)."""
    rng = np.random.default_rng(M * 7 + N * 3 + K)
    A = rng.standard_normal((M, K))
    B = rng.standard_normal((K, N))
    ref = A.astype(np.longdouble) @ B.astype(np.longdouble)
    bound = _bound(precision, A, B, K)
    Ad = torch.tensor(A, device="cuda")
    Bd = torch.tensor(B, device="cuda")
    for s in (SPLIT_ALL, SPLIT_NONE, DEFAULT):
        fc.fc_set_schedule(**s)
        C = fc.fc_dgemm(Ad, Bd, precision=precision).cpu().numpy()
        ratio = float(np.max(np.abs(C.astype(np.longdouble) - ref).astype(np.float64) / bound))
        print(f"prec {precision} {M}x{N}x{K} schedule {s}: err / bound {ratio:.2e}")
        assert ratio <= 1.0


@pytest.mark.parametrize("precision", [0, 2])
def test_solve_under_extreme_schedules(fc, precision):
    """A 3D n = 255 solve (4 Gaussians + a sine mode, eps = 1e-9) under both corners of the
    search space: each within 1e-6 of the full-format oracle, and within 2e-6 of each other."""
    prob = fi.config2(0)
    h = fc.fc_setup(prob.n, prob.d, prob.alpha, prob.beta, prob.gamma, prob.eps,
                    max_rank=prob.max_rank, precision=precision)
    B = fc.CP.from_factors(*prob.rhs())
    ref = full.solve_full(cp.to_full(prob.rhs()), prob.alpha, prob.beta, prob.gamma)
    got = []
    for s in (SPLIT_ALL, SPLIT_NONE):
        fc.fc_set_schedule(**s)
        U = fc.CP(prob.d, prob.n, prob.max_rank)
        info = fc.fc_solve(h, B, U, tol=prob.tol, eps=prob.eps)
        u = fc.fc_to_full(h, U).cpu().numpy()
        e = rel(u, ref)
        print(f"prec {precision} schedule {s}: iters {info.iters} rank {U.rank} err {e:.2e}")
        assert info.status == 0 and e < 1e-6
        got.append(u)
    assert rel(got[0], got[1]) < 2e-6


def _mixed(count, nmax):
    return [p for p in (fi.config4(i) for i in range(80)) if p.n <= nmax][:count]


def _setup_mixed(fc, probs):
    hs = [fc.fc_setup(p.n, p.d, p.alpha, p.beta, p.gamma, p.eps, max_rank=p.max_rank,
                      max_tucker=p.max_tucker, precision=2) for p in probs]
    Bs = [fc.CP.from_factors(*p.rhs()) for p in probs]
    Us = [fc.CP(p.d, p.n, p.max_rank) for p in probs]
    return hs, Bs, Us


def test_batched_largest_first_with_few_workers(fc):
    """Largest-first order with 3 workers for 10 mixed problems (n 127 and 255): every
    problem is solved (status 0) to within 1e-6 of its exact solution."""
    from oracle import eigerr
    probs = _mixed(10, 255)
    assert len({p.n for p in probs}) == 2
    hs, Bs, Us = _setup_mixed(fc, probs)
    fc.fc_set_schedule(workers=3, order=1)
    infos = fc.fc_solve_batched(hs, Bs, Us, tol=[p.tol for p in probs],
                                eps=[p.eps for p in probs], raise_on_fail=False, stall=8)
    for p, U, info in zip(probs, Us, infos):
        e = eigerr.control_error(U.factors(), p.rhs(), p.alpha, p.beta, p.gamma)[0]
        print(f"{p.label} status {info.status} iters {info.iters} err {e:.1e}")
        assert info.status == 0 and e <= 1e-6


def test_autotune_batched(fc):
    """The batched form's autotuner on 8 mixed problems: one pass evaluates the start and
    every other candidate of every field (17 runs), leaves the best as the process schedule,
    and the last run's solutions are all within 1e-6 of the exact solutions."""
    from oracle import eigerr
    probs = _mixed(8, 255)
    hs, Bs, Us = _setup_mixed(fc, probs)
    best, cost, evals = fc.fc_autotune_batched(hs, Bs, Us, tol=[p.tol for p in probs],
                                               eps=[p.eps for p in probs], stall=8, passes=1,
                                               min_gain=0.02)
    print(f"best {best.as_dict()} cost {cost * 1e3:.2f} ms per solve, {evals} evaluations")
    assert evals == 17
    assert fc.fc_get_schedule().as_dict() == best.as_dict()
    assert 0.0 < cost < 10.0
    for p, U in zip(probs, Us):
        e = eigerr.control_error(U.factors(), p.rhs(), p.alpha, p.beta, p.gamma)[0]
        assert e <= 1e-6, (p.label, e)


def test_autotune_batched_errors_restore_the_schedule(fc):
    """An argument error (the same handle twice) is reported, and the process schedule is the
    one from before the call."""
    probs = _mixed(2, 127)
    hs, Bs, Us = _setup_mixed(fc, probs[:1])
    fc.fc_set_schedule(workers=24)
    before = fc.fc_get_schedule().as_dict()
    with pytest.raises(fc.FCError) as e:
        fc.fc_autotune_batched([hs[0], hs[0]], Bs * 2, Us * 2)
    assert e.value.code == fc.fc.FC_EINVAL
    assert fc.fc_get_schedule().as_dict() == before
