"""fc_symeig, the small dense FP64 eigen-solves of the RHOSVD truncation (Section 5).

method 0 (Householder / bisection / inverse iteration) against LAPACK (numpy.linalg.eigh)
on random, graded, rank-deficient and degenerate matrices; method 1 (the truncation's graded
Jacobi solver) for orthonormality, eigenvalues, and the property the truncation relies on:
on a graded Gram matrix its eigen-directions order the energy so that the eps-rank found
from projected energies equals the optimal (SVD) rank."""
import numpy as np
import pytest
import scipy.linalg as sl
import torch

pytestmark = pytest.mark.gpu


def _cases(m, rng):
    A = rng.standard_normal((m, m))
    yield "sym", A + A.T
    Q, _ = np.linalg.qr(rng.standard_normal((m, m)))
    yield "graded", (Q * 10.0 ** (-16 * np.arange(m) / max(m - 1, 1))) @ Q.T
    B = rng.standard_normal((m, max(1, m // 3)))
    yield "rankdef", B @ B.T * 1e-30
    yield "identity", np.eye(m) * 3.0
    yield "zero", np.zeros((m, m))


@pytest.mark.parametrize("method", [0, 1])
@pytest.mark.parametrize("m", [1, 2, 3, 7, 33, 56, 64])
def test_symeig_matches_lapack(m, method):
    import paper_1809_01971_gb300 as fc
    rng = np.random.default_rng(100 + m)
    names, mats = zip(*_cases(m, rng))
    A = torch.tensor(np.stack(mats), device="cuda")
    w, V = fc.fc_symeig(A, method=method)
    torch.cuda.synchronize()
    w, V = w.cpu().numpy(), V.cpu().numpy()
    # method 0: FP64 accuracy.  method 1 resolves eigen-directions to FP32 precision relative
    # to the grading of the matrix (what the truncation needs; see the graded-rank test below)
    # and returns FP64 Rayleigh quotients: eigenvalues within ~(1e-7)^2 ... 1e-7 relative to
    # ||A|| depending on the gaps, eigenvectors orthonormal to FP64 precision.
    tol_w = 1e-13 if method == 0 else 1e-7
    for b, (name, M) in enumerate(zip(names, mats)):
        wn = np.linalg.eigvalsh(M)[::-1]
        nA = max(np.linalg.norm(M, 2), 1e-300)
        e_w = np.max(np.abs(np.sort(w[b])[::-1] - wn)) / nA
        e_o = np.linalg.norm(V[b].T @ V[b] - np.eye(m))
        e_r = np.linalg.norm(M @ V[b] - V[b] * w[b]) / max(np.linalg.norm(M), 1e-300)
        print(f"method {method} m={m} {name}: eig {e_w:.1e} orth {e_o:.1e} resid {e_r:.1e}")
        assert e_w <= tol_w
        assert e_o <= 1e-12
        if name != "zero":
            assert e_r <= (1e-12 if method == 0 else 1e-5)
        if method == 0:
            assert np.all(np.diff(w[b]) <= 0)


@pytest.mark.parametrize("seed", [5, 6])
def test_graded_gram_reaches_optimal_rank(seed):
    """Gram of a pivoted sketch basis (diagonal falling from ~1 to ~1e-22): the eps = 1e-9
    rank from projected energies along method-1 eigenvectors is the SVD rank of W."""
    import paper_1809_01971_gb300 as fc
    rng = np.random.default_rng(seed)
    n, K, c = 255, 2000, 56
    sv = 10.0 ** (-np.linspace(0, 12, 60))
    U, _ = np.linalg.qr(rng.standard_normal((n, 60)))
    Vk, _ = np.linalg.qr(rng.standard_normal((K, 60)))
    W = (U * sv) @ Vk.T
    Q, _, _ = sl.qr(W @ rng.standard_normal((K, c)), mode="economic", pivoting=True)
    B = Q.T @ W
    T = B @ B.T
    w, V = fc.fc_symeig(torch.tensor(T, device="cuda"), method=1)
    V = V[0].cpu().numpy()
    thr2 = (1e-9) ** 2 / 6 * np.sum(sv ** 2)
    rho = np.sum((V.T @ B) ** 2, axis=1)
    missed = max(np.sum(W ** 2) - np.sum(B ** 2), 0.0)
    tail = np.append(np.cumsum(rho[::-1])[::-1], 0.0)
    r = next(i for i in range(1, c + 1) if tail[i] + missed <= thr2)
    s = np.linalg.svd(W, compute_uv=False)
    t_opt = np.cumsum((s ** 2)[::-1])[::-1]
    r_opt = next(i for i in range(len(t_opt)) if t_opt[i] <= thr2)
    print(f"graded seed {seed}: rank {r}, optimal {r_opt}, orth {np.linalg.norm(V.T @ V - np.eye(c)):.1e}")
    assert r <= r_opt + 1
    assert np.linalg.norm(V.T @ V - np.eye(c)) <= 1e-12
