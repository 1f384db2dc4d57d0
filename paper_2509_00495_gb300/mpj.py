"""Thin ctypes binding of libmpjacobi (same entry-point names as include/mpjacobi.h).

Argument marshalling only: every step of the solve runs in the library's CUDA
kernels.  Device memory and streams come from PyTorch: inputs are CUDA
float64 tensors, outputs are allocated with torch and filled by the library
on ``torch.cuda.current_stream()``.  There is no CPU fallback: if the library
is missing or a tensor is not on a CUDA device, the call raises.

Layout: the library is column-major.  A row-major (n, n) torch tensor ``T``
seen column-major is ``T.T``; for a symmetric A this is A itself.  Returned
eigenvector matrices are ``Q`` with ``Q[:, j]`` the eigenvector of ``W[j]``.
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass

import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
_LIBPATH = os.path.join(_HERE, "libmpjacobi.so")

MPJ_OK = 0
MPJ_NOT_CONVERGED = 1
MPJ_EINVAL = -1
MPJ_ENOTSYM = -2
MPJ_ENONFINITE = -3
MPJ_ECUDA = -4
MPJ_ENOMEM = -5
MPJ_EDEGENERATE = -6
MPJ_EWORKSPACE = -7
MPJ_ETIMEOUT = -8
MPJ_ETOOLARGE = -9
MPJ_EPREMISE = -10

ORDER_CYCLIC = 0
ORDER_ROUND_ROBIN = 1
ORDER_BLOCK = 2
METHOD_MIXED = 0
METHOD_PLAIN = 1

_vp = ctypes.c_void_p
_i = ctypes.c_int
_d = ctypes.c_double
_ip = ctypes.POINTER(ctypes.c_int)
_dp = ctypes.POINTER(ctypes.c_double)


class Opts(ctypes.Structure):
    _fields_ = [("tol", _d), ("tol32", _d), ("max_sweeps64", _i), ("max_sweeps32", _i), ("ns_steps", _i),
                ("ordering", _i), ("method", _i), ("polish", _i), ("sort", _i), ("check_symmetry", _i),
                ("threshold", _i), ("precond_passes", _i), ("stage1_half", _i), ("max_sweeps32_pass2", _i)]


class Info(ctypes.Structure):
    _fields_ = [("status", _i), ("sweeps32", _i), ("sweeps32_pass2", _i), ("sweeps64", _i), ("ns_steps", _i),
                ("norm_fro", _d),
                ("tol", _d), ("off32", _d), ("off_cond", _d), ("off_final", _d), ("ms_stage", ctypes.c_float * 6),
                ("ns_e0", _d), ("rotated_blocks64", ctypes.c_longlong)]

    def as_dict(self) -> dict:
        d = {k: getattr(self, k) for k, _ in self._fields_ if k != "ms_stage"}
        d["ms_stage"] = list(self.ms_stage)
        return d


class MPJError(RuntimeError):
    def __init__(self, status: int, where: str):
        self.status = status
        msg = f"{where}: {status_str(status)}"
        if status == MPJ_ECUDA:
            msg += f" ({lib().mpj_last_cuda_error().decode()})"
        super().__init__(msg)


_lib = None


def lib():
    """Load libmpjacobi.so (built in place by build.py); raise if it is missing."""
    global _lib
    if _lib is None:
        if not os.path.exists(_LIBPATH):
            raise RuntimeError(f"libmpjacobi.so not built ({_LIBPATH}); run paper_2509_00495_gb300/build.py")
        L = ctypes.CDLL(_LIBPATH)
        L.mpj_opts_default.argtypes = [ctypes.POINTER(Opts)]
        L.mpj_status_str.argtypes = [_i]
        L.mpj_status_str.restype = ctypes.c_char_p
        L.mpj_last_cuda_error.restype = ctypes.c_char_p
        L.mpj_kernel_launches.restype = ctypes.c_longlong
        L.mpj_device_allocations.restype = ctypes.c_longlong
        L.mpj_syev_workspace.argtypes = [_i, ctypes.POINTER(Opts)]
        L.mpj_syev_workspace.restype = ctypes.c_size_t
        L.mpj_syev.argtypes = [_i, _vp, _i, _vp, _vp, _d, _vp]
        L.mpj_syev_ex.argtypes = [_i, _vp, _i, _vp, _vp, _i, ctypes.POINTER(Opts), ctypes.POINTER(Info), _vp,
                                  ctypes.c_size_t, _vp]
        L.mpj_stage1.argtypes = [_i, _vp, _i, _vp, _i, _d, _i, _ip, _dp, _vp]
        L.mpj_newton_schulz.argtypes = [_i, _vp, _i, _i, _vp]
        L.mpj_precondition.argtypes = [_i, _vp, _i, _vp, _i, _vp, _i, _vp]
        L.mpj_jacobi64.argtypes = [_i, _vp, _i, _vp, _i, _d, _i, _i, _ip, _dp, _vp]
        L.mpj_dgemm.argtypes = [ctypes.c_char, ctypes.c_char, _i, _i, _i, _d, _vp, _i, _vp, _i, _d, _vp, _i, _vp]
        L.mpj_stage1_panel.argtypes = [_i, _i, _vp, _vp, _vp, _i, _vp]
        L.mpj_dgemm_tc.argtypes = [ctypes.c_char, ctypes.c_char, _i, _i, _i, _d, _vp, _i, _vp, _i, _d, _vp, _i, _vp]
        if hasattr(L, "mpj_syev_batched"):
            L.mpj_syev_batched.argtypes = [_i, _ip, _vp, _vp, _vp, _d, _ip, _vp]
            L.mpj_batched_group_size.argtypes = [_i, _ip]
            L.mpj_release_plans.argtypes = []
        if hasattr(L, "mpj_syev_backward"):
            L.mpj_syev_backward.argtypes = [_i, _i, _vp, _vp, _i, _vp, _vp, _i, _vp, _i, _vp]
        _lib = L
    return _lib


def status_str(st: int) -> str:
    return lib().mpj_status_str(st).decode()


def _stream():
    return _vp(torch.cuda.current_stream().cuda_stream)


def _dev(t: torch.Tensor, name: str) -> torch.Tensor:
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError(f"{name} must be a CUDA tensor (libmpjacobi has no CPU path)")
    if t.dtype != torch.float64:
        raise TypeError(f"{name} must be float64")
    return t


def _ptr(t):
    return _vp(t.data_ptr()) if t is not None else _vp(0)


def _check(st: int, where: str, allow_not_converged=True):
    if st < 0 or (st == MPJ_NOT_CONVERGED and not allow_not_converged):
        raise MPJError(st, where)
    return st


def default_opts(**kw) -> Opts:
    o = Opts()
    lib().mpj_opts_default(ctypes.byref(o))
    for k, v in kw.items():
        if v is None:
            continue
        if k == "ordering" and isinstance(v, str):
            v = {"cyclic": ORDER_CYCLIC, "round_robin": ORDER_ROUND_ROBIN, "block": ORDER_BLOCK}[v]
        if k == "method" and isinstance(v, str):
            v = {"mixed": METHOD_MIXED, "plain": METHOD_PLAIN}[v]
        setattr(o, k, int(v) if isinstance(v, bool) else v)
    return o


@dataclass
class SolveResult:
    W: torch.Tensor
    Q: torch.Tensor
    info: dict
    status: int


def syev_ex(A: torch.Tensor, *, workspace: torch.Tensor | None = None, **opts) -> SolveResult:
    """mpj_syev_ex on a symmetric CUDA float64 (n, n) tensor.  Options as in mpj_opts."""
    A = _dev(A, "A")
    n = A.shape[0]
    if A.dim() != 2 or A.shape[1] != n:
        raise ValueError("A must be square")
    if not A.is_contiguous():
        A = A.contiguous()
    W = torch.empty(n, dtype=torch.float64, device=A.device)
    Qt = torch.empty(n, n, dtype=torch.float64, device=A.device)
    o = default_opts(**opts)
    info = Info()
    wp, wb = (_ptr(workspace), workspace.numel() * workspace.element_size()) if workspace is not None else (_vp(0), 0)
    st = lib().mpj_syev_ex(n, _ptr(A), max(n, 1), _ptr(W), _ptr(Qt), max(n, 1), ctypes.byref(o), ctypes.byref(info),
                           wp, ctypes.c_size_t(wb), _stream())
    _check(st, "mpj_syev_ex")
    return SolveResult(W, Qt.T, info.as_dict(), st)


def syev(A: torch.Tensor, tol: float = 0.0):
    """mpj_syev (mixed method, default options): returns (W ascending, Q)."""
    A = _dev(A, "A").contiguous()
    n = A.shape[0]
    W = torch.empty(n, dtype=torch.float64, device=A.device)
    Qt = torch.empty(n, n, dtype=torch.float64, device=A.device)
    st = lib().mpj_syev(n, _ptr(A), max(n, 1), _ptr(W), _ptr(Qt), tol, _stream())
    _check(st, "mpj_syev")
    return W, Qt.T


def syev_workspace(n: int, **opts) -> int:
    o = default_opts(**opts)
    return int(lib().mpj_syev_workspace(n, ctypes.byref(o)))


def stage1(A: torch.Tensor, tol32: float = 0.0, max_sweeps: int = 0):
    """mpj_stage1: returns (Q_l, sweeps, off32)."""
    A = _dev(A, "A").contiguous()
    n = A.shape[0]
    Qt = torch.empty(n, n, dtype=torch.float64, device=A.device)
    sw, of = ctypes.c_int(), ctypes.c_double()
    st = lib().mpj_stage1(n, _ptr(A), n, _ptr(Qt), n, tol32, max_sweeps, ctypes.byref(sw), ctypes.byref(of),
                          _stream())
    _check(st, "mpj_stage1")
    return Qt.T.contiguous(), sw.value, of.value


def newton_schulz(X: torch.Tensor, steps: int = 2) -> torch.Tensor:
    """mpj_newton_schulz on a copy of X (column-major semantics handled here)."""
    X = _dev(X, "X")
    n = X.shape[0]
    Xt = X.T.contiguous()  # column-major buffer of X
    st = lib().mpj_newton_schulz(n, _ptr(Xt), n, steps, _stream())
    _check(st, "mpj_newton_schulz")
    return Xt.T


def precondition(A: torch.Tensor, Qd: torch.Tensor) -> torch.Tensor:
    """mpj_precondition: A_cond = Q_d^T A Q_d."""
    A = _dev(A, "A")
    n = A.shape[0]
    At = A.T.contiguous()
    Qt = _dev(Qd, "Qd").T.contiguous()
    Ct = torch.empty(n, n, dtype=torch.float64, device=A.device)
    st = lib().mpj_precondition(n, _ptr(At), n, _ptr(Qt), n, _ptr(Ct), n, _stream())
    _check(st, "mpj_precondition")
    return Ct.T


def jacobi64(A: torch.Tensor, V: torch.Tensor | None = None, *, tol: float = 0.0, ordering=ORDER_ROUND_ROBIN,
             max_sweeps: int = 0):
    """mpj_jacobi64 on copies of A and V: returns (A_final, V, sweeps, off_final, status)."""
    A = _dev(A, "A")
    n = A.shape[0]
    if isinstance(ordering, str):
        ordering = {"cyclic": ORDER_CYCLIC, "round_robin": ORDER_ROUND_ROBIN, "block": ORDER_BLOCK}[ordering]
    At = A.T.contiguous()
    Vt = (torch.eye(n, dtype=torch.float64, device=A.device) if V is None else _dev(V, "V")).T.contiguous()
    sw, of = ctypes.c_int(), ctypes.c_double()
    st = lib().mpj_jacobi64(n, _ptr(At), n, _ptr(Vt), n, tol, ordering, max_sweeps, ctypes.byref(sw),
                            ctypes.byref(of), _stream())
    _check(st, "mpj_jacobi64")
    return At.T, Vt.T, sw.value, of.value, st


def dgemm(transa: str, transb: str, alpha: float, A: torch.Tensor, B: torch.Tensor, beta: float = 0.0,
          C: torch.Tensor | None = None) -> torch.Tensor:
    """mpj_dgemm with numpy-like semantics: alpha op(A) op(B) + beta C (row-major tensors in and out)."""
    A = _dev(A, "A")
    B = _dev(B, "B")
    At, Bt = A.T.contiguous(), B.T.contiguous()  # column-major buffers
    m = A.shape[1] if transa == "T" else A.shape[0]
    k = A.shape[0] if transa == "T" else A.shape[1]
    n = B.shape[0] if transb == "T" else B.shape[1]
    Ct = (torch.zeros(n, m, dtype=torch.float64, device=A.device) if C is None else _dev(C, "C").T.contiguous())
    st = lib().mpj_dgemm(transa.encode(), transb.encode(), m, n, k, alpha, _ptr(At), max(A.shape[0], 1), _ptr(Bt),
                         max(B.shape[0], 1), beta, _ptr(Ct), max(m, 1), _stream())
    _check(st, "mpj_dgemm")
    return Ct.T


def dgemm_tc(transa: str, transb: str, alpha: float, A: torch.Tensor, B: torch.Tensor, beta: float = 0.0,
             C: torch.Tensor | None = None) -> torch.Tensor:
    """mpj_dgemm_tc (FP64 product on the tensor cores from exact bf16 slices),
    with the numpy-like semantics of dgemm."""
    A = _dev(A, "A")
    B = _dev(B, "B")
    At, Bt = A.T.contiguous(), B.T.contiguous()  # column-major buffers
    m = A.shape[1] if transa == "T" else A.shape[0]
    k = A.shape[0] if transa == "T" else A.shape[1]
    n = B.shape[0] if transb == "T" else B.shape[1]
    Ct = (torch.zeros(n, m, dtype=torch.float64, device=A.device) if C is None else _dev(C, "C").T.contiguous())
    st = lib().mpj_dgemm_tc(transa.encode(), transb.encode(), m, n, k, alpha, _ptr(At), max(A.shape[0], 1),
                            _ptr(Bt), max(B.shape[0], 1), beta, _ptr(Ct), max(m, 1), _stream())
    _check(st, "mpj_dgemm_tc")
    return Ct.T


def stage1_panel(R: int, U: torch.Tensor, In: torch.Tensor, transpose_out: bool = False,
                 _test_no_commit: bool = False) -> torch.Tensor:
    """mpj_stage1_panel: the tensor-core block product of block round R.
    In: N x N float32 holding the column-major matrix (In[j, i] = element
    (i, j), i.e. the transpose of the logical matrix, as stored); U: (N/32,
    32, 32) float32 with U[q, j, i] = U_q(i, j).  Returns Out in the same
    storage convention."""
    for t, name in ((In, "In"), (U, "U")):
        if not isinstance(t, torch.Tensor) or not t.is_cuda or t.dtype != torch.float32:
            raise TypeError(f"{name} must be a float32 CUDA tensor")
    In, U = In.contiguous(), U.contiguous()
    N = In.shape[0]
    Out = torch.zeros_like(In)
    mode = int(transpose_out) | (2 if _test_no_commit else 0)
    st = lib().mpj_stage1_panel(N, R, _ptr(U), _ptr(In), _ptr(Out), mode, _stream())
    _check(st, "mpj_stage1_panel")
    return Out


# ------------------------------------------------------------------ batched
class BatchedSolver:
    """Repeated mpj_syev_batched calls on fixed device buffers (the planned,
    graph-replayed path): inputs are copied into the solver's own matrices,
    so every call after the first replays the same CUDA graph."""

    def __init__(self, sizes, device="cuda"):
        self.sizes = [int(n) for n in sizes]
        self.A = [torch.empty(n, n, dtype=torch.float64, device=device) for n in self.sizes]
        self.W = [torch.empty(n, dtype=torch.float64, device=device) for n in self.sizes]
        self.Qt = [torch.empty(n, n, dtype=torch.float64, device=device) for n in self.sizes]
        self.pa = torch.tensor([a.data_ptr() for a in self.A], dtype=torch.int64, device=device)
        self.pw = torch.tensor([w.data_ptr() for w in self.W], dtype=torch.int64, device=device)
        self.pq = torch.tensor([q.data_ptr() for q in self.Qt], dtype=torch.int64, device=device)
        self.ns = (ctypes.c_int * len(self.sizes))(*self.sizes)

    def solve(self, mats=None, tol: float = 0.0):
        if mats is not None:
            for dst, src in zip(self.A, mats):
                dst.copy_(src)
        sweeps = (ctypes.c_int * len(self.sizes))()
        st = lib().mpj_syev_batched(len(self.sizes), self.ns, _ptr(self.pa), _ptr(self.pw), _ptr(self.pq), tol,
                                    sweeps, _stream())
        _check(st, "mpj_syev_batched")
        return self.W, [q.T for q in self.Qt], list(sweeps), st

    def group_size(self) -> int:
        return int(lib().mpj_batched_group_size(len(self.sizes), self.ns))


def syev_batched(mats: list[torch.Tensor], tol: float = 0.0):
    """mpj_syev_batched over a list of symmetric CUDA float64 matrices (n_i <= 256).
    Returns (list of W, list of Q, sweeps per matrix, status)."""
    L = lib()
    if not hasattr(L, "mpj_syev_batched"):
        raise RuntimeError("libmpjacobi built without mpj_syev_batched")
    mats = [_dev(a, "A").contiguous() for a in mats]
    b = len(mats)
    dev = mats[0].device
    ns = (ctypes.c_int * b)(*[a.shape[0] for a in mats])
    Ws = [torch.empty(a.shape[0], dtype=torch.float64, device=dev) for a in mats]
    Qts = [torch.empty_like(a) for a in mats]
    pa = torch.tensor([a.data_ptr() for a in mats], dtype=torch.int64, device=dev)
    pw = torch.tensor([w.data_ptr() for w in Ws], dtype=torch.int64, device=dev)
    pq = torch.tensor([q.data_ptr() for q in Qts], dtype=torch.int64, device=dev)
    sweeps = (ctypes.c_int * b)()
    st = L.mpj_syev_batched(b, ns, _ptr(pa), _ptr(pw), _ptr(pq), tol, sweeps, _stream())
    _check(st, "mpj_syev_batched")
    return Ws, [q.T for q in Qts], list(sweeps), st


# ------------------------------------------------------------------ backward
def syev_backward(W: torch.Tensor, Q: torch.Tensor, dW: torch.Tensor | None, dQ: torch.Tensor | None):
    """mpj_syev_backward for a batch (leading dim) or one matrix: returns dA (symmetric)."""
    L = lib()
    if not hasattr(L, "mpj_syev_backward"):
        raise RuntimeError("libmpjacobi built without mpj_syev_backward")
    single = W.dim() == 1
    if single:
        W, Q = W[None], Q[None]
        dW = None if dW is None else dW[None]
        dQ = None if dQ is None else dQ[None]
    W = _dev(W, "W").contiguous()
    b, n = W.shape
    Qt = _dev(Q, "Q").transpose(1, 2).contiguous()
    dWc = None if dW is None else _dev(dW, "dW").contiguous()
    dQt = None if dQ is None else _dev(dQ, "dQ").transpose(1, 2).contiguous()
    dAt = torch.empty(b, n, n, dtype=torch.float64, device=W.device)
    st = L.mpj_syev_backward(b, n, _ptr(W), _ptr(Qt), n, _ptr(dWc), _ptr(dQt), n, _ptr(dAt), n, _stream())
    _check(st, "mpj_syev_backward")
    dA = dAt.transpose(1, 2)
    return dA[0] if single else dA


class EighFunction(torch.autograd.Function):
    """(W, Q) = eigh(A) through mpj_syev_ex; backward through mpj_syev_backward."""

    @staticmethod
    def forward(ctx, A, opts):
        r = syev_ex(A, **(opts or {}))
        ctx.save_for_backward(r.W, r.Q)
        return r.W, r.Q

    @staticmethod
    def backward(ctx, dW, dQ):
        W, Q = ctx.saved_tensors
        return syev_backward(W, Q, dW, dQ), None


def eigh(A: torch.Tensor, **opts):
    """Differentiable mixed precision eigh of a symmetric CUDA float64 matrix."""
    return EighFunction.apply(A, opts)
