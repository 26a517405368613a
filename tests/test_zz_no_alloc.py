"""fc_inner_static: the CP inner product for callers that cannot allocate device memory.

Some callers cannot call cudaMalloc (a graph capture that must not allocate, a host that
hands out device memory itself, a loop that forbids allocation after start-up).  This entry
point takes no handle and keeps its scratch in a fixed device array inside the library.
The test calls it through the C ABI and checks it against fc_inner, the existing entry
point, on two calls in a row (the second call reuses the scratch the first one left behind).
It lives in its own file so that it runs last, and it works alone in a fresh process too.
"""
import ctypes

import numpy as np
import pytest
import torch

import fc_inputs as fi

pytestmark = pytest.mark.gpu


def _check_pairs(fc, h, cases, out):
    for X, Y in cases:
        Xg, Yg = fc.CP.from_factors(*X), fc.CP.from_factors(*Y)
        ref = fc.fc_inner(h, Xg, Yg)
        fc.fc_inner_static(Xg, Yg, out)
        torch.cuda.synchronize()
        got = float(out.item())
        scale = float(np.sqrt(abs(fc.fc_inner(h, Xg, Xg)) * abs(fc.fc_inner(h, Yg, Yg))))
        assert abs(got - ref) <= 1e-13 * scale, (got, ref)


def test_inner_static_matches_fc_inner_on_two_calls():
    import paper_1809_01971_gb300 as fc
    assert torch.cuda.is_available()
    n, d = 61, 3
    h = fc.fc_setup(n, d, 0.5, 1.0, 1e-2, 1e-8, max_input_rank=128)
    out = torch.full((1,), float("nan"), dtype=torch.float64, device="cuda")
    _check_pairs(fc, h, [(fi.random_cp(n, d, 7, seed=31), fi.random_cp(n, d, 9, seed=32)),
                         (fi.random_cp(n, d, 100, seed=33), fi.random_cp(n, d, 90, seed=34))], out)


def test_inner_static_split_k_path_on_two_calls():
    """n = 255 >= 128: the cross-Gram GEMMs split K across CTAs (a zeroing pass, then FP64
    atomic accumulation into the shared scratch), so the second call starts from what the
    first left in the array."""
    import paper_1809_01971_gb300 as fc
    n, d = 255, 3
    h = fc.fc_setup(n, d, 0.5, 1.0, 1e-2, 1e-8, max_input_rank=128)
    out = torch.full((1,), float("nan"), dtype=torch.float64, device="cuda")
    _check_pairs(fc, h, [(fi.random_cp(n, d, 100, seed=41), fi.random_cp(n, d, 96, seed=42)),
                         (fi.random_cp(n, d, 128, seed=43), fi.random_cp(n, d, 120, seed=44))], out)


def test_inner_static_two_dimensional_and_rank_zero():
    import paper_1809_01971_gb300 as fc
    n, d = 200, 2
    h = fc.fc_setup(n, d, 0.5, 1.0, 1e-2, 1e-8, max_input_rank=128)
    out = torch.full((1,), float("nan"), dtype=torch.float64, device="cuda")
    _check_pairs(fc, h, [(fi.random_cp(n, d, 50, seed=45), fi.random_cp(n, d, 70, seed=46)),
                         (fi.random_cp(n, d, 5, seed=47), fi.random_cp(n, d, 128, seed=48))], out)
    X = fc.CP.from_factors(*fi.random_cp(n, d, 4, seed=49))
    Z = fc.CP(d, n, 8)                                       # rank 0
    out.fill_(float("nan"))
    fc.fc_inner_static(X, Z, out)
    torch.cuda.synchronize()
    assert float(out.item()) == 0.0


def test_inner_static_rejects_ranks_above_its_limit():
    import paper_1809_01971_gb300 as fc
    n, d = 20, 2
    X = fc.CP.from_factors(*fi.random_cp(n, d, 129, seed=35))
    Y = fc.CP.from_factors(*fi.random_cp(n, d, 3, seed=36))
    out = torch.zeros(1, dtype=torch.float64, device="cuda")
    rc = fc.lib().fc_inner_static(ctypes.byref(X.desc()), ctypes.byref(Y.desc()),
                                  ctypes.c_void_p(out.data_ptr()), None)
    assert rc == fc.fc.FC_ERANK
