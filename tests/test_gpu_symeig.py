"""fc_symeig, the small dense FP64 eigen-solver of the RHOSVD truncation (Section 5), against
LAPACK's symmetric eigen-solver (numpy.linalg.eigh) on random, graded, rank-deficient and
degenerate matrices, with the sizes the truncation uses (up to 64, ragged)."""
import numpy as np
import pytest
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


@pytest.mark.parametrize("m", [1, 2, 3, 7, 33, 56, 64])
def test_symeig_matches_lapack(m):
    import paper_1809_01971_gb300 as fc
    rng = np.random.default_rng(100 + m)
    names, mats = zip(*_cases(m, rng))
    A = torch.tensor(np.stack(mats), device="cuda")
    w, V = fc.fc_symeig(A)
    torch.cuda.synchronize()
    w, V = w.cpu().numpy(), V.cpu().numpy()
    for b, (name, M) in enumerate(zip(names, mats)):
        wn = np.linalg.eigvalsh(M)[::-1]
        nA = max(np.linalg.norm(M, 2), 1e-300)
        e_w = np.max(np.abs(w[b] - wn)) / nA
        e_o = np.linalg.norm(V[b].T @ V[b] - np.eye(m))
        e_r = np.linalg.norm(M @ V[b] - V[b] * w[b]) / max(np.linalg.norm(M), 1e-300)
        print(f"m={m} {name}: eig {e_w:.1e} orth {e_o:.1e} resid {e_r:.1e}")
        assert e_w <= 1e-13
        assert e_o <= 1e-12
        assert e_r <= 1e-12 or name == "zero"
        assert np.all(np.diff(w[b]) <= 0)
