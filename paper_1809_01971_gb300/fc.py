"""Thin Python binding of libfc (ctypes): argument marshalling only.

Every entry point of ``include/fc.h`` has a function of the same name here; each one
converts its arguments to the C types, calls the library and raises :class:`FCError`
on a non-zero status.  All arithmetic runs in the CUDA library.  PyTorch supplies the
device memory (factor matrices, weights, workspace) and the current CUDA stream.

The library must have been built (``python -m paper_1809_01971_gb300.build``); loading
fails loudly otherwise.  There is no CPU fallback.

A canonical (CP) tensor (Section 5, eqn:CP_form of the paper)
    T = sum_{r < rank} xi[r] U_1[:, r] (x) ... (x) U_d[:, r]
is held by :class:`CP`: ``xi`` of shape (cap,) and ``U`` of shape (d, cap, ld), FP64,
so ``U[l, r, :n]`` is column r of the column-major n x cap factor matrix U_l.
"""
from __future__ import annotations

import ctypes as C
import os
from typing import Optional

import numpy as np
import torch

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libfc.so")

FC_OK = 0
FC_EINVAL = -1
FC_ERANK = -2
FC_ENOCONV = -3
FC_EBREAKDOWN = -4
FC_ENAN = -5
FC_ECUDA = -6
FC_EWORKSPACE = -7
FC_ESETUP = -8
FC_ETIMEOUT = -9


class fc_cp(C.Structure):
    _fields_ = [("d", C.c_int), ("n", C.c_int), ("rank", C.c_int), ("cap", C.c_int),
                ("ld", C.c_int), ("xi", C.c_void_p), ("U", C.c_void_p * 3)]


class fc_setup_opts(C.Structure):
    _fields_ = [("delta_sym", C.c_double), ("precond_rank", C.c_int), ("max_rank", C.c_int),
                ("max_tucker", C.c_int), ("max_input_rank", C.c_int), ("directional", C.c_int),
                ("precision", C.c_int), ("op_kind", C.c_int), ("precond_kind", C.c_int),
                ("coeff", C.c_void_p * 3)]


class fc_setup_info(C.Structure):
    _fields_ = [("n", C.c_int), ("d", C.c_int), ("rank_symbol", C.c_int),
                ("rank_minus", C.c_int), ("rank_plus", C.c_int), ("rank_precond", C.c_int),
                ("rho_min", C.c_double), ("rho_max", C.c_double), ("sym_err", C.c_double),
                ("pc_err", C.c_double), ("workspace_bytes", C.c_size_t)]


class fc_solve_opts(C.Structure):
    _fields_ = [("tol", C.c_double), ("eps", C.c_double), ("kmax", C.c_int),
                ("max_rank", C.c_int), ("spectral", C.c_int), ("precision", C.c_int),
                ("stall", C.c_int)]


class fc_solve_info(C.Structure):
    _fields_ = [("status", C.c_int), ("iters", C.c_int), ("relres", C.c_double),
                ("rank_x", C.c_int), ("max_rank_seen", C.c_int), ("trunc_calls", C.c_int),
                ("tucker_max", C.c_int), ("tucker_mean", C.c_double), ("basis_max", C.c_int),
                ("history", C.c_double * 128)]


class fc_schedule(C.Structure):
    _fields_ = [("gemm_cover", C.c_int), ("gemm_split", C.c_int), ("tc_split", C.c_int),
                ("tc_min_log2", C.c_int), ("workers", C.c_int), ("order", C.c_int)]

    def as_dict(self) -> dict:
        return {k: getattr(self, k) for k, _ in self._fields_}


# cost callback of fc_autotune: double (*)(const fc_schedule*, void*)
TUNE_COST = C.CFUNCTYPE(C.c_double, C.POINTER(fc_schedule), C.c_void_p)


class FCError(RuntimeError):
    def __init__(self, fn: str, code: int, msg: str):
        super().__init__(f"{fn}: {msg} ({code})")
        self.code = code


_LIB = None


def lib() -> C.CDLL:
    """Load libfc.so (built in-tree); raises if it is missing."""
    global _LIB
    if _LIB is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"libfc.so not built: {LIB_PATH} missing; run "
                               "python -m paper_1809_01971_gb300.build")
        L = C.CDLL(LIB_PATH)
        P, I, D, V = C.c_void_p, C.c_int, C.c_double, C.c_void_p
        cp_p = C.POINTER(fc_cp)
        sig = {
            "fc_setup": (I, [I, I, D, D, D, D, C.POINTER(fc_setup_opts), C.POINTER(P)]),
            "fc_get_info": (I, [P, C.POINTER(fc_setup_info)]),
            "fc_workspace_size": (I, [P, C.POINTER(C.c_size_t)]),
            "fc_set_workspace": (I, [P, V, C.c_size_t]),
            "fc_get_symbol": (I, [P, I, cp_p, V]),
            "fc_apply": (I, [P, cp_p, cp_p, V]),
            "fc_precond": (I, [P, cp_p, cp_p, V]),
            "fc_truncate": (I, [P, cp_p, D, I, I, cp_p, V]),
            "fc_inner": (I, [P, cp_p, cp_p, C.POINTER(D), V]),
            "fc_apply_trunc": (I, [P, I, cp_p, D, I, cp_p, V]),
            "fc_state": (I, [P, cp_p, D, I, cp_p, V]),
            "fc_solve": (I, [P, cp_p, cp_p, C.POINTER(fc_solve_opts), C.POINTER(fc_solve_info), V]),
            "fc_solve_batched": (I, [I, C.POINTER(P), cp_p, cp_p, C.POINTER(fc_solve_opts),
                                     C.POINTER(fc_solve_info), V]),
            "fc_set_wait_limit": (I, [I, C.POINTER(I)]),
            "fc_to_full": (I, [P, cp_p, V, V]),
            "fc_full_solve": (I, [P, V, V, V, V]),
            "fc_destroy": (None, [P]),
            "fc_strerror": (C.c_char_p, [I]),
            "fc_last_cuda_error": (C.c_char_p, []),
            "fc_launch_count": (C.c_ulonglong, []),
            "fc_inner_static": (I, [cp_p, cp_p, V, V]),
            "fc_prof_enable": (I, [I]),
            "fc_symeig": (I, [I, I, I, V, I, C.c_longlong, V, C.c_longlong, V, I, C.c_longlong, V]),
            "fc_prof_read": (I, [C.POINTER(C.c_longlong), C.POINTER(D), C.POINTER(D)]),
            "fc_dgemm": (I, [I, I, I, I, I, I, D, V, I, V, I, D, V, I, V]),
            "fc_get_schedule": (I, [C.POINTER(fc_schedule)]),
            "fc_set_schedule": (I, [C.POINTER(fc_schedule)]),
            "fc_autotune": (I, [C.POINTER(fc_schedule), I, D, TUNE_COST, V,
                                C.POINTER(fc_schedule), C.POINTER(D), C.POINTER(I)]),
            "fc_autotune_batched": (I, [I, C.POINTER(P), cp_p, cp_p, C.POINTER(fc_solve_opts), I,
                                        D, C.POINTER(fc_schedule), C.POINTER(D), C.POINTER(I),
                                        V]),
        }
        for name, (res, args) in sig.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _LIB = L
    return _LIB


def _check(fn: str, rc: int) -> int:
    if rc != FC_OK:
        L = lib()
        msg = L.fc_strerror(rc).decode()
        if rc == FC_ECUDA:
            msg += ": " + L.fc_last_cuda_error().decode()
        raise FCError(fn, rc, msg)
    return rc


def _stream(stream) -> Optional[int]:
    if stream is None:
        return torch.cuda.current_stream().cuda_stream
    if isinstance(stream, torch.cuda.Stream):
        return stream.cuda_stream
    return int(stream)


class CP:
    """Device CP tensor with capacity ``cap`` (weights and factor matrices in FP64)."""

    def __init__(self, d: int, n: int, cap: int, device="cuda", ld: Optional[int] = None):
        self.d, self.n, self.cap = d, n, cap
        self.ld = ld if ld is not None else n
        self.rank = 0
        self.xi = torch.zeros(max(cap, 1), dtype=torch.float64, device=device)
        self.U = torch.zeros(d, max(cap, 1), self.ld, dtype=torch.float64, device=device)

    @classmethod
    def from_factors(cls, xi, U, cap: Optional[int] = None, device="cuda", ld=None) -> "CP":
        """From weights (R,) and d factor matrices (n, R) (numpy or torch, host or device)."""
        xi = torch.as_tensor(xi, dtype=torch.float64)
        d = len(U)
        n = int(U[0].shape[0])
        R = int(xi.shape[0])
        t = cls(d, n, cap if cap is not None else R, device=device, ld=ld)
        if R > t.cap:
            raise ValueError("rank exceeds capacity")
        t.xi[:R].copy_(xi)
        for l in range(d):
            t.U[l, :R, :n].copy_(torch.as_tensor(U[l], dtype=torch.float64).T)
        t.rank = R
        return t

    def factors(self):
        """(xi, [U_l]) on the host as numpy arrays, U_l of shape (n, rank)."""
        R = self.rank
        xi = self.xi[:R].detach().cpu().numpy().copy()
        U = [self.U[l, :R, :self.n].detach().cpu().numpy().T.copy() for l in range(self.d)]
        return xi, U

    def desc(self) -> fc_cp:
        c = fc_cp()
        c.d, c.n, c.rank, c.cap, c.ld = self.d, self.n, self.rank, self.cap, self.ld
        c.xi = self.xi.data_ptr()
        base = self.U.data_ptr()
        stride = self.U.stride(0) * 8
        for l in range(3):
            c.U[l] = base + (l if l < self.d else 0) * stride
        return c


class Handle:
    """A set-up problem (fc_setup) with its torch-allocated workspace bound."""

    def __init__(self, ptr: int, device):
        self.device = device
        self.ptr = C.c_void_p(ptr)
        info = fc_setup_info()
        _check("fc_get_info", lib().fc_get_info(self.ptr, C.byref(info)))
        self.info = info
        nbytes = C.c_size_t()
        _check("fc_workspace_size", lib().fc_workspace_size(self.ptr, C.byref(nbytes)))
        self.workspace = torch.empty(nbytes.value + 256, dtype=torch.uint8, device=device)
        base = self.workspace.data_ptr()
        aligned = (base + 255) & ~255
        _check("fc_set_workspace", lib().fc_set_workspace(self.ptr, C.c_void_p(aligned), nbytes.value))

    @property
    def n(self):
        return self.info.n

    @property
    def d(self):
        return self.info.d

    def destroy(self):
        if self.ptr:
            lib().fc_destroy(self.ptr)
            self.ptr = C.c_void_p(0)

    def __del__(self):
        try:
            self.destroy()
        except Exception:
            pass


def fc_get_info(h: Handle) -> fc_setup_info:
    """Sizes and ranks of a set-up (fc_get_info)."""
    info = fc_setup_info()
    _check("fc_get_info", lib().fc_get_info(h.ptr, C.byref(info)))
    return info


def fc_workspace_size(h: Handle) -> int:
    """Bytes of device scratch the handle needs (fc_workspace_size)."""
    nbytes = C.c_size_t()
    _check("fc_workspace_size", lib().fc_workspace_size(h.ptr, C.byref(nbytes)))
    return nbytes.value


def fc_set_workspace(h: Handle, buf: torch.Tensor) -> None:
    """Bind caller-owned device scratch (fc_set_workspace): a CUDA tensor of at least
    fc_workspace_size(h) bytes whose data pointer is 256-byte aligned.  The handle keeps a
    reference to it in place of the workspace fc_setup allocated."""
    nbytes = buf.numel() * buf.element_size()
    _check("fc_set_workspace", lib().fc_set_workspace(h.ptr, C.c_void_p(buf.data_ptr()), nbytes))
    h.workspace = buf


def fc_destroy(h: Handle) -> None:
    """Release the handle's set-up tables (fc_destroy); the handle is unusable afterwards."""
    h.destroy()


def fc_strerror(code: int) -> str:
    """Text of a status code (fc_strerror)."""
    return lib().fc_strerror(int(code)).decode()


def fc_last_cuda_error() -> str:
    """Text of the last CUDA error the library recorded (fc_last_cuda_error)."""
    return lib().fc_last_cuda_error().decode()


def fc_setup(n, d, alpha, beta, gamma, eps, delta_sym=0.0, precond_rank=0, max_rank=0,
             max_tucker=0, max_input_rank=0, directional=False, precision=0, op_kind=0,
             precond_kind=0, coeff=None, device="cuda") -> Handle:
    """precision: 0 FP64 contractions, 1 double-float FP32 contractions, 2 FP64-accurate
    digit products on the BF16 tensor cores for the large contractions.  op_kind: 0 the
    control operator, 1 A^alpha, 2 I + A^(2 alpha); precond_kind: 0 least-squares fit of 1/g,
    1 the exponential sum of rho^-alpha; coeff: per mode None or the n+1 values a_l((i+1/2)h)
    of a variable coefficient (fc_setup_opts)."""
    o = fc_setup_opts(delta_sym, precond_rank, max_rank, max_tucker, max_input_rank,
                      1 if directional else 0, int(precision), int(op_kind), int(precond_kind))
    keep = []                    # coefficient arrays stay alive through the call
    if coeff is not None:
        for l, a in enumerate(list(coeff)[:3]):
            if a is None:
                continue
            arr = np.ascontiguousarray(np.asarray(a, dtype=np.float64))
            if arr.shape != (int(n) + 1,):
                raise ValueError(f"coeff[{l}] needs n+1 = {int(n) + 1} values a((i+1/2)h)")
            keep.append(arr)
            o.coeff[l] = arr.ctypes.data
    out = C.c_void_p()
    _check("fc_setup", lib().fc_setup(int(n), int(d), float(alpha), float(beta), float(gamma),
                                      float(eps), C.byref(o), C.byref(out)))
    return Handle(out.value, device)


def fc_get_symbol(h: Handle, which: int, out: CP, stream=None) -> CP:
    c = out.desc()
    _check("fc_get_symbol", lib().fc_get_symbol(h.ptr, which, C.byref(c), _stream(stream)))
    out.rank = c.rank
    return out


def _apply(fn: str, h: Handle, x: CP, y: CP, stream) -> CP:
    cx, cy = x.desc(), y.desc()
    rc = getattr(lib(), fn)(h.ptr, C.byref(cx), C.byref(cy), _stream(stream))
    y.rank = cy.rank
    _check(fn, rc)
    return y


def fc_apply(h: Handle, x: CP, y: CP, stream=None) -> CP:
    return _apply("fc_apply", h, x, y, stream)


def fc_precond(h: Handle, x: CP, y: CP, stream=None) -> CP:
    return _apply("fc_precond", h, x, y, stream)


def fc_truncate(h: Handle, x: CP, eps: float, max_rank: int, y: CP, normalize: bool = True,
                stream=None) -> CP:
    cx, cy = x.desc(), y.desc()
    rc = lib().fc_truncate(h.ptr, C.byref(cx), float(eps), int(max_rank), 1 if normalize else 0,
                           C.byref(cy), _stream(stream))
    y.rank = cy.rank
    _check("fc_truncate", rc)
    return y


def fc_apply_trunc(h: Handle, which: int, x: CP, eps: float, max_rank: int, y: CP,
                   stream=None) -> CP:
    cx, cy = x.desc(), y.desc()
    rc = lib().fc_apply_trunc(h.ptr, int(which), C.byref(cx), float(eps), int(max_rank),
                              C.byref(cy), _stream(stream))
    y.rank = cy.rank
    _check("fc_apply_trunc", rc)
    return y


def fc_state(h: Handle, u: CP, eps: float, max_rank: int, y: CP, stream=None) -> CP:
    """y = trunc(beta A^-alpha u, eps): the state of the control problem (eqn:State)."""
    cu, cy = u.desc(), y.desc()
    rc = lib().fc_state(h.ptr, C.byref(cu), float(eps), int(max_rank), C.byref(cy), _stream(stream))
    y.rank = cy.rank
    _check("fc_state", rc)
    return y


def fc_inner(h: Handle, x: CP, y: CP, stream=None) -> float:
    out = C.c_double()
    _check("fc_inner", lib().fc_inner(h.ptr, C.byref(x.desc()), C.byref(y.desc()), C.byref(out),
                                      _stream(stream)))
    return out.value


def _form(precision):
    """fc_solve_opts.precision: None -> 0 (the handle's form), else the setup code + 1."""
    return 0 if precision is None else int(precision) + 1


def fc_solve(h: Handle, rhs: CP, u: CP, tol=1e-8, eps=0.0, kmax=100, max_rank=0, stream=None,
             raise_on_fail: bool = True, spectral: bool = False, precision=None,
             stall: int = 0) -> fc_solve_info:
    """Algorithm 1; spectral=True keeps every iterate in the DST-I eigenbasis (one transform
    at entry and exit instead of two per mat-vec: the same result).  precision: None for the
    handle's contraction form, else 0 FP64 / 1 double-float / 2 tensor-core digits for this
    solve.  stall > 0: stop after that many iterations without a 10% residual decrease and
    return the best iterate (fc_solve_opts.stall)."""
    o = fc_solve_opts(float(tol), float(eps), int(kmax), int(max_rank), 1 if spectral else 0,
                      _form(precision), int(stall))
    info = fc_solve_info()
    cr, cu = rhs.desc(), u.desc()
    rc = lib().fc_solve(h.ptr, C.byref(cr), C.byref(cu), C.byref(o), C.byref(info), _stream(stream))
    u.rank = cu.rank
    if raise_on_fail or rc not in (FC_ENOCONV, FC_EBREAKDOWN, FC_ENAN):
        _check("fc_solve", rc)
    return info


def _batch_args(handles, rhs, us, tol, eps, kmax, max_rank, spectral, precision, stall):
    count = len(handles)

    def per(v):
        return list(v) if isinstance(v, (list, tuple)) else [v] * count

    tols, epss, kms, mrs, prs = per(tol), per(eps), per(kmax), per(max_rank), per(precision)
    H = (C.c_void_p * count)(*[h.ptr.value for h in handles])
    R = (fc_cp * count)(*[x.desc() for x in rhs])
    Uc = (fc_cp * count)(*[x.desc() for x in us])
    O = (fc_solve_opts * count)(*[fc_solve_opts(float(tols[i]), float(epss[i]), int(kms[i]),
                                                int(mrs[i]), 1 if spectral else 0, _form(prs[i]),
                                                int(stall))
                                  for i in range(count)])
    return count, H, R, Uc, O


def fc_solve_batched(handles, rhs, us, tol=1e-8, eps=0.0, kmax=100, max_rank=0,
                     raise_on_fail: bool = True, spectral: bool = False, precision=None,
                     stream=None, stall: int = 0):
    """Independent solves run concurrently (a pool of host threads, fc_schedule.workers, each
    on a worker stream of the library that starts after the work queued on ``stream`` and
    joins it).  tol / eps / kmax / max_rank / precision are scalars or per-problem sequences."""
    count, H, R, Uc, O = _batch_args(handles, rhs, us, tol, eps, kmax, max_rank, spectral,
                                     precision, stall)
    infos = (fc_solve_info * count)()
    rc = lib().fc_solve_batched(count, H, R, Uc, O, infos, _stream(stream))
    for i in range(count):
        us[i].rank = Uc[i].rank
    if raise_on_fail or rc not in (FC_ENOCONV, FC_EBREAKDOWN, FC_ENAN):
        _check("fc_solve_batched", rc)
    return list(infos)


def fc_get_schedule() -> fc_schedule:
    """The process launch schedule (tile and split rules, batch policy)."""
    s = fc_schedule()
    _check("fc_get_schedule", lib().fc_get_schedule(C.byref(s)))
    return s


def fc_set_schedule(s=None, **fields) -> fc_schedule:
    """Replace the process schedule by ``s`` (default: the current one) with ``fields``
    changed; returns the previous schedule."""
    prev = fc_get_schedule()
    new = fc_schedule(*[getattr(s if s is not None else prev, k) for k, _ in fc_schedule._fields_])
    for k, v in fields.items():
        if k not in dict(fc_schedule._fields_):
            raise TypeError(f"no schedule field {k!r}")
        setattr(new, k, int(v))
    _check("fc_set_schedule", lib().fc_set_schedule(C.byref(new)))
    return prev


def fc_autotune(cost, start=None, passes: int = 1, min_gain: float = 0.02):
    """The autotuner's coordinate descent on a Python cost ``cost(schedule_dict) -> float``;
    returns (best schedule, best cost, evaluations).  The process schedule is not changed."""
    def _cb(cand, _ctx):
        try:
            return float(cost(cand.contents.as_dict()))
        except Exception:       # a failed candidate
            return float("nan")

    cb = TUNE_COST(_cb)
    best, bc, ev = fc_schedule(), C.c_double(), C.c_int()
    _check("fc_autotune", lib().fc_autotune(C.byref(start) if start is not None else None,
                                            int(passes), float(min_gain), cb, None,
                                            C.byref(best), C.byref(bc), C.byref(ev)))
    return best, bc.value, ev.value


def fc_autotune_batched(handles, rhs, us, tol=1e-8, eps=0.0, kmax=100, max_rank=0,
                        spectral: bool = False, precision=None, stall: int = 0, passes: int = 1,
                        min_gain: float = 0.02, stream=None):
    """The batched form's autotuner: every candidate schedule timed on one fc_solve_batched run
    of these problems (seconds per converged solve); leaves the best as the process schedule
    and returns (best schedule, its cost, evaluations)."""
    count, H, R, Uc, O = _batch_args(handles, rhs, us, tol, eps, kmax, max_rank, spectral,
                                     precision, stall)
    best, bc, ev = fc_schedule(), C.c_double(), C.c_int()
    rc = lib().fc_autotune_batched(count, H, R, Uc, O, int(passes), float(min_gain),
                                   C.byref(best), C.byref(bc), C.byref(ev), _stream(stream))
    for i in range(count):
        us[i].rank = Uc[i].rank
    _check("fc_autotune_batched", rc)
    return best, bc.value, ev.value


def fc_set_wait_limit(iterations: int) -> int:
    """Test hook: the producer-side wait limit of the tensor-core kernel (fc_set_wait_limit);
    returns the previous limit."""
    prev = C.c_int()
    _check("fc_set_wait_limit", lib().fc_set_wait_limit(int(iterations), C.byref(prev)))
    return prev.value


def fc_to_full(h: Handle, x: CP, out: Optional[torch.Tensor] = None, stream=None) -> torch.Tensor:
    """Full n^d array; returned with shape (n,)*d in numpy axis order (i_1 is axis 0)."""
    n, d = h.n, h.d
    if out is None:
        out = torch.empty(n ** d, dtype=torch.float64, device=x.xi.device)
    _check("fc_to_full", lib().fc_to_full(h.ptr, C.byref(x.desc()), C.c_void_p(out.data_ptr()),
                                          _stream(stream)))
    # column-major with i_1 fastest -> numpy axis order reversed
    return out.view(*([n] * d)).permute(*reversed(range(d)))


def fc_inner_static(x: CP, y: CP, out: torch.Tensor, stream=None) -> torch.Tensor:
    """<x, y> into the device scalar ``out`` without a handle or any allocation."""
    if out.dtype != torch.float64 or not out.is_cuda:
        raise ValueError("out must be a CUDA float64 tensor")
    if x.xi.device != out.device or y.xi.device != out.device:
        raise ValueError("x, y and out must be on the same CUDA device")
    with torch.cuda.device(out.device):
        _check("fc_inner_static", lib().fc_inner_static(C.byref(x.desc()), C.byref(y.desc()),
                                                        C.c_void_p(out.data_ptr()),
                                                        _stream(stream)))
    return out


def fc_symeig(A: torch.Tensor, method: int = 0, stream=None):
    """Eigen-decomposition of a batch (b, m, m) of symmetric FP64 CUDA matrices:
    (w descending (b, m), V (b, m, m) with eigenvectors as columns).  method 0: Householder /
    bisection / inverse iteration; method 1: the truncation's graded Jacobi solver."""
    if A.dim() == 2:
        A = A.unsqueeze(0)
    A = A.contiguous()
    bsz, m, _ = A.shape
    w = torch.empty(bsz, m, dtype=torch.float64, device=A.device)
    Vt = torch.empty(bsz, m, m, dtype=torch.float64, device=A.device)   # column-major V = Vt^T
    _check("fc_symeig", lib().fc_symeig(int(method), bsz, m, C.c_void_p(A.data_ptr()), m, m * m,
                                        C.c_void_p(w.data_ptr()), m, C.c_void_p(Vt.data_ptr()), m,
                                        m * m, _stream(stream)))
    return w, Vt.transpose(1, 2)


def fc_dgemm(A: torch.Tensor, B: torch.Tensor, precision: int = 2, alpha: float = 1.0,
             beta: float = 0.0, C_: torch.Tensor = None, stream=None) -> torch.Tensor:
    """C = alpha A B + beta C for FP64 CUDA matrices in a contraction form of the solver
    (0 FP64, 1 double-float FP32, 2 BF16 tensor-core digit products).  A torch matrix in
    row-major storage is the column-major transpose, so op(A) = A is passed as transA with
    the row-major leading dimension."""
    assert A.dtype == torch.float64 and B.dtype == torch.float64 and A.dim() == 2 and B.dim() == 2
    A = A.contiguous()
    B = B.contiguous()
    M, K = A.shape
    K2, N = B.shape
    assert K == K2
    if C_ is None:
        C_ = torch.zeros(M, N, dtype=torch.float64, device=A.device)
    assert C_.shape == (M, N) and C_.is_contiguous() and C_.dtype == torch.float64
    # row-major C (M x N) is the column-major C^T (N x M, ld N) = B^T A^T, where the row-major
    # B (K x N) is the column-major B^T (N x K, ld N) and A the column-major A^T (K x M, ld K)
    _check("fc_dgemm", lib().fc_dgemm(int(precision), 0, 0, N, M, K, float(alpha),
                                      C.c_void_p(B.data_ptr()), max(N, 1),
                                      C.c_void_p(A.data_ptr()), max(K, 1), float(beta),
                                      C.c_void_p(C_.data_ptr()), max(N, 1), _stream(stream)))
    out = C_
    return out


PROF_JACOBI = 1
PROF_TC = 2
PROF_F64 = 3


def fc_prof_enable(kclass: int) -> None:
    _check("fc_prof_enable", lib().fc_prof_enable(int(kclass)))


def fc_prof_read():
    """(launches, summed event time in ms, algorithmic flops) of the instrumented class."""
    n, ms, work = C.c_longlong(), C.c_double(), C.c_double()
    _check("fc_prof_read", lib().fc_prof_read(C.byref(n), C.byref(ms), C.byref(work)))
    return n.value, ms.value, work.value


def fc_launch_count() -> int:
    """Kernels libfc has launched in this process so far."""
    return int(lib().fc_launch_count())


def fc_full_solve(h: Handle, rhs: torch.Tensor, u: torch.Tensor, tmp: torch.Tensor,
                  stream=None) -> torch.Tensor:
    """rhs, u, tmp: contiguous device arrays of n^d doubles, column-major (i_1 fastest)."""
    for t in (rhs, u, tmp):
        if t.dtype != torch.float64 or not t.is_contiguous() or t.numel() != h.n ** h.d:
            raise ValueError("full arrays must be contiguous float64 with n^d elements")
    _check("fc_full_solve", lib().fc_full_solve(h.ptr, C.c_void_p(rhs.data_ptr()),
                                                C.c_void_p(u.data_ptr()), C.c_void_p(tmp.data_ptr()),
                                                _stream(stream)))
    return u
