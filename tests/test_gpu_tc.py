"""The solver's contraction kernel in its three forms through the C ABI (fc_dgemm): the FP64
tiled GEMM, double-float FP32, and the BF16 tensor-core form with 8 fixed-point digits per
operand.  Reference: the exact product in extended precision (numpy longdouble) of the same
FP64 operands.  Bounds: FP64 and double-float, k u |A||B| elementwise; the tensor-core form
rounds each operand to 2^-56 of its row (column) scale 2^E > max |row|, so its bound is
k 2^-53 max|A_i,:| max|B_:,j|."""
import ctypes

import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def fc():
    import paper_1809_01971_gb300 as m
    m.lib()
    return m


def exact(A, B):
    return (A.astype(np.longdouble) @ B.astype(np.longdouble))


def check(form, A, B, C, ref, K):
    absab = np.abs(A) @ np.abs(B)
    if form == 2:
        bound = 2.0 * max(K, 1) * 2.0 ** -53 * np.outer(np.abs(A).max(axis=1), np.abs(B).max(axis=0))
    elif form == 1:
        bound = 4.0 * max(K, 1) * 2.0 ** -46 * absab
    else:
        bound = 2.0 * max(K, 1) * 2.0 ** -53 * absab
    err = np.abs(C.astype(np.longdouble) - ref).astype(np.float64)
    ratio = float(np.max(err / np.maximum(bound, 1e-300)))
    return ratio


SHAPES = [(1, 1, 1), (5, 7, 3), (128, 16, 32), (77, 13, 33), (200, 48, 300), (129, 65, 257),
          (255, 100, 255), (300, 70, 1000)]


@pytest.mark.parametrize("form", [0, 1, 2])
@pytest.mark.parametrize("M,N,K", SHAPES)
def test_dgemm_forms_within_bounds(fc, form, M, N, K):
    rng = np.random.default_rng(1000 + M + 7 * N + 13 * K)
    A = rng.standard_normal((M, K)) * np.exp(2.0 * rng.standard_normal((M, K)))   # graded rows
    B = rng.standard_normal((K, N))
    C = fc.fc_dgemm(torch.tensor(A, device="cuda"), torch.tensor(B, device="cuda"), precision=form)
    ratio = check(form, A, B, C.cpu().numpy(), exact(A, B), K)
    print(f"form {form} M={M} N={N} K={K}: err / bound = {ratio:.3e}")
    assert ratio <= 1.0


def test_tc_alpha_beta_splitk_and_ragged(fc):
    """alpha, beta != 0 with a K range split over CTAs (K > 128: FP64 atomics on a
    pre-scaled C), ragged M, N not multiples of the 128 x 16 tiles."""
    rng = np.random.default_rng(77)
    M, N, K = 333, 37, 777
    A, B, C0 = rng.standard_normal((M, K)), rng.standard_normal((K, N)), rng.standard_normal((M, N))
    Cg = torch.tensor(C0, device="cuda")
    fc.fc_dgemm(torch.tensor(A, device="cuda"), torch.tensor(B, device="cuda"), precision=2,
                alpha=-0.75, beta=0.5, C_=Cg)
    ref = -0.75 * exact(A, B) + 0.5 * C0.astype(np.longdouble)
    bound = 2.0 * K * 2.0 ** -53 * 0.75 * np.outer(np.abs(A).max(1), np.abs(B).max(0)) + 2.0 ** -53 * np.abs(C0)
    err = np.abs(Cg.cpu().numpy().astype(np.longdouble) - ref).astype(np.float64)
    assert np.all(err <= 2.0 * bound)


def test_tc_scales_zeros_and_non_finite(fc):
    """Rows of very different binary scale (1e-200 ... 1e+200), an all-zero row, K = 0, and
    a row holding a NaN (that row of C is NaN, every other row stays exact)."""
    rng = np.random.default_rng(78)
    M, N, K = 140, 24, 150
    A = rng.standard_normal((M, K))
    A[0] *= 1e-200
    A[1] *= 1e200
    A[2] = 0.0
    A[3, 17] = np.nan
    B = rng.standard_normal((K, N))
    C = fc.fc_dgemm(torch.tensor(A, device="cuda"), torch.tensor(B, device="cuda"), precision=2)
    C = C.cpu().numpy()
    assert np.all(np.isnan(C[3]))
    assert np.all(C[2] == 0.0)
    ok = np.ones(M, bool)
    ok[3] = False
    A2 = A.copy()
    A2[3] = 0.0
    ref = exact(A2, B)
    bound = 2.0 * K * 2.0 ** -53 * np.outer(np.abs(A2).max(1), np.abs(B).max(0))
    err = np.abs(C.astype(np.longdouble) - ref).astype(np.float64)
    assert np.all(err[ok] <= np.maximum(bound[ok], 1e-320))
    # K = 0: C = beta C
    Cg = torch.ones(4, 5, dtype=torch.float64, device="cuda")
    fc.fc_dgemm(torch.zeros(4, 0, dtype=torch.float64, device="cuda"),
                torch.zeros(0, 5, dtype=torch.float64, device="cuda"), precision=2, beta=3.0, C_=Cg)
    assert torch.all(Cg == 3.0)


@pytest.mark.parametrize("ta,tb", [(0, 1), (1, 0), (1, 1)])
def test_dgemm_transposes_through_abi(fc, ta, tb):
    """Column-major operands with op = transpose, called on the C ABI directly."""
    rng = np.random.default_rng(79 + 2 * ta + tb)
    M, N, K = 150, 40, 200
    opA, opB = rng.standard_normal((M, K)), rng.standard_normal((K, N))
    # column-major storage of the stored matrix X is the row-major storage of X^T
    storedA = opA.T if ta else opA             # stored (rows x cols), column-major
    storedB = opB.T if tb else opB
    dA = torch.tensor(np.ascontiguousarray(storedA.T), device="cuda")   # row-major of X^T
    dB = torch.tensor(np.ascontiguousarray(storedB.T), device="cuda")
    dC = torch.zeros(N, M, dtype=torch.float64, device="cuda")           # column-major M x N
    lda, ldb = storedA.shape[0], storedB.shape[0]
    for form in (0, 2):
        rc = fc.lib().fc_dgemm(form, ta, tb, M, N, K, 1.0, ctypes.c_void_p(dA.data_ptr()), lda,
                               ctypes.c_void_p(dB.data_ptr()), ldb, 0.0,
                               ctypes.c_void_p(dC.data_ptr()), M, None)
        assert rc == 0
        torch.cuda.synchronize()
        C = dC.cpu().numpy().T
        assert check(form, opA, opB, C, exact(opA, opB), K) <= 1.0
    # argument errors
    assert fc.lib().fc_dgemm(3, 0, 0, M, N, K, 1.0, None, M, None, K, 0.0, None, M, None) == -1
    assert fc.lib().fc_dgemm(2, 0, 0, M, N, K, 1.0, ctypes.c_void_p(dA.data_ptr()), M - 1,
                             ctypes.c_void_p(dB.data_ptr()), K, 0.0,
                             ctypes.c_void_p(dC.data_ptr()), M, None) == -1
