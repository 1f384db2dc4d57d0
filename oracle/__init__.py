"""CPU oracle of the mixed precision Jacobi eigensolver (arXiv 2509.00495).

TEST INFRASTRUCTURE ONLY: the tests, the smoke check and the CPU-baseline leg
of the benchmark may use this package; the library itself never imports it,
and it imports nothing from the library.  The arithmetic lives in
``mpj_oracle.c`` (plain C, -O2 -ffp-contract=off, no BLAS); this module only
compiles it and marshals numpy arrays through ctypes.

All matrices are numpy float64 (or float32) arrays in Fortran (column-major)
order; ``Q[:, j]`` is the eigenvector of ``W[j]``.

Parity pins for every function live in ``tests/test_oracle_*.py``.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "mpj_oracle.c")
_LIB = os.path.join(_HERE, "libmpj_oracle.so")

CYCLIC = 0
ROUND_ROBIN = 1
BLOCK_ROUND_ROBIN = 2  # the FP32 stage's block ordering (blocks of 16)
BLOCK = 16

U_D = 2.0 ** -53  # unit roundoff, double (paper Sec. 1.2, unit roundoff table)
U_L = 2.0 ** -24  # unit roundoff, single


def build(force: bool = False) -> str:
    """Compile mpj_oracle.c into libmpj_oracle.so (in place) if it is stale."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(
            ["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-std=c11", "-fPIC", "-shared",
             "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


_lib = None


def _load():
    global _lib
    if _lib is None:
        # MPJ_ORACLE_SO points the oracle at another build of mpj_oracle.c (the
        # mutation test uses it to plant mistakes and check the pins catch them)
        path = os.environ.get("MPJ_ORACLE_SO") or build()
        _lib = ctypes.CDLL(path)
        _declare(_lib)
    return _lib


_dp = ctypes.POINTER(ctypes.c_double)
_fp = ctypes.POINTER(ctypes.c_float)
_ip = ctypes.POINTER(ctypes.c_int)
_llp = ctypes.POINTER(ctypes.c_longlong)
_i = ctypes.c_int
_d = ctypes.c_double


class _Opts(ctypes.Structure):
    _fields_ = [("tol", _d), ("tol32", _d), ("skip_tol", _d), ("skip_tol32", _d),
                ("max_sweeps64", _i), ("max_sweeps32", _i), ("ns_steps", _i),
                ("ordering32", _i), ("ordering64", _i), ("polish", _i), ("sort", _i), ("threshold", _i),
                ("precond_passes", _i), ("stage1_half", _i)]


class _Info(ctypes.Structure):
    _fields_ = [("sweeps32", _i), ("sweeps64", _i), ("capped32", _i), ("capped64", _i),
                ("rotations32", ctypes.c_longlong), ("rotations64", ctypes.c_longlong),
                ("normA_fro", _d), ("off32", _d), ("off_cond", _d), ("off_final", _d), ("sweeps32_pass2", _i),
                ("ns_steps", _i), ("ns_e0", _d)]


def _declare(L):
    L.orc_jacobi_pair_d.argtypes = [_d, _d, _d, _dp, _dp]
    L.orc_jacobi_pair_f.argtypes = [ctypes.c_float] * 3 + [_fp, _fp]
    L.orc_off_d.argtypes = [_i, _dp, _i]
    L.orc_off_d.restype = _d
    L.orc_off_f.argtypes = [_i, _fp, _i]
    L.orc_off_f.restype = _d
    L.orc_fro_d.argtypes = [_i, _dp, _i]
    L.orc_fro_d.restype = _d
    L.orc_round_robin_pair.argtypes = [_i, _i, _i, _ip, _ip, _ip]
    L.orc_block_pair.argtypes = [_i, _i, _i, _i, _i, _ip, _ip]
    L.orc_block_pair.restype = _i
    L.orc_jacobi_d.argtypes = [_i, _dp, _i, _dp, _i, _i, _d, _d, _i, _i, _ip, _llp, _dp, _d]
    L.orc_jacobi_d.restype = _i
    L.orc_jacobi_f.argtypes = [_i, _fp, _i, _fp, _i, _i, _d, ctypes.c_float, _i, _ip, _llp, _dp]
    L.orc_jacobi_f.restype = _i
    for name in ("orc_gemm_tn_d", "orc_gemm_nn_d", "orc_gemm_nt_d"):
        getattr(L, name).argtypes = [_i, _i, _i, _dp, _i, _dp, _i, _dp, _i]
    L.orc_newton_schulz_d.argtypes = [_i, _dp, _i, _i]
    L.orc_precondition_d.argtypes = [_i, _dp, _i, _dp, _i, _dp, _i]
    L.orc_stage1.argtypes = [_i, _dp, _i, _dp, _i, ctypes.POINTER(_Opts), ctypes.POINTER(_Info), _fp]
    L.orc_stage1.restype = _i
    L.orc_syev_mixed.argtypes = [_i, _dp, _i, _dp, _dp, _i, ctypes.POINTER(_Opts), ctypes.POINTER(_Info),
                                 _dp, _dp, _dp]
    L.orc_syev_mixed.restype = _i
    L.orc_syev_plain.argtypes = [_i, _dp, _i, _dp, _dp, _i, ctypes.POINTER(_Opts), ctypes.POINTER(_Info)]
    L.orc_syev_plain.restype = _i
    L.orc_eigh_backward.argtypes = [_i, _dp, _dp, _i, _dp, _dp, _i, _dp, _i]
    L.orc_eigh_backward.restype = _i
    L.orc_sample_rotations.argtypes = [_i, ctypes.c_void_p, _i, ctypes.c_void_p, _i, ctypes.c_longlong, _i]
    L.orc_round_half.argtypes = [ctypes.c_float]
    L.orc_round_half.restype = ctypes.c_float
    L.orc_ns_steps.argtypes = [_i, _i]
    L.orc_ns_steps.restype = _i
    L.orc_jacobi_h.argtypes = [_i, _fp, _i, _fp, _i, _i, _d, ctypes.c_float, _i, _ip, _llp, _dp]
    L.orc_jacobi_h.restype = _i


def _f64(a) -> np.ndarray:
    return np.array(a, dtype=np.float64, order="F", copy=True)


def _ptr(a: np.ndarray | None, t=_dp):
    if a is None:
        return ctypes.cast(None, t)
    assert a.flags.f_contiguous or a.ndim == 1
    return a.ctypes.data_as(t)


@dataclass
class Info:
    sweeps32: int
    sweeps64: int
    capped32: bool
    capped64: bool
    rotations32: int
    rotations64: int
    normA_fro: float
    off32: float
    off_cond: float
    off_final: float
    sweeps32_pass2: int = 0
    ns_steps: int = 0
    ns_e0: float = 0.0


def _info(ci: _Info) -> Info:
    return Info(ci.sweeps32, ci.sweeps64, bool(ci.capped32), bool(ci.capped64), ci.rotations32,
                ci.rotations64, ci.normA_fro, ci.off32, ci.off_cond, ci.off_final, ci.sweeps32_pass2,
                ci.ns_steps, ci.ns_e0)


class PremiseError(ArithmeticError):
    """Q_l violates the Newton-Schulz premise ||Q_l^T Q_l - I||_2 < 2."""


def _opts(n, tol=0.0, tol32=0.0, skip_tol=0.0, skip_tol32=0.0, max_sweeps64=0, max_sweeps32=0, ns_steps=0,
          ordering32=CYCLIC, ordering64=CYCLIC, polish=False, sort=True, threshold=False,
          precond_passes=1, stage1_half=False) -> _Opts:
    return _Opts(tol, tol32, skip_tol, skip_tol32, max_sweeps64, max_sweeps32, ns_steps, ordering32, ordering64,
                 int(polish), int(sort), int(threshold), int(precond_passes), int(stage1_half))


# ---------------------------------------------------------------- primitives
def jacobi_pair(app: float, aqq: float, apq: float, dtype=np.float64):
    """Algorithm 2 (Sec. 3.1.2, stable form of Appendix A): returns (c, s)."""
    L = _load()
    if dtype == np.float32:
        c, s = ctypes.c_float(), ctypes.c_float()
        L.orc_jacobi_pair_f(app, aqq, apq, ctypes.byref(c), ctypes.byref(s))
        return np.float32(c.value), np.float32(s.value)
    c, s = _d(), _d()
    L.orc_jacobi_pair_d(app, aqq, apq, ctypes.byref(c), ctypes.byref(s))
    return c.value, s.value


def off(A) -> float:
    """off(A) = sqrt(sum_{i != j} a_ij^2) (Sec. 3.1 definition, direct form)."""
    L = _load()
    if np.asarray(A).dtype == np.float32:
        a = np.array(A, dtype=np.float32, order="F")
        return L.orc_off_f(a.shape[0], _ptr(a, _fp), a.shape[0])
    a = _f64(A)
    return L.orc_off_d(a.shape[0], _ptr(a), a.shape[0])


def fro(A) -> float:
    a = _f64(A)
    return _load().orc_fro_d(a.shape[0], _ptr(a), a.shape[0])


def round_robin_pairs(n: int):
    """The round-robin (circle method) schedule: list over rounds of lists of (p, q)."""
    L = _load()
    m = n + (n & 1)
    p, q, v = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
    rounds = []
    for r in range(max(m - 1, 0)):
        pairs = []
        for i in range(m // 2):
            L.orc_round_robin_pair(n, r, i, ctypes.byref(p), ctypes.byref(q), ctypes.byref(v))
            if v.value:
                pairs.append((p.value, q.value))
        rounds.append(pairs)
    return rounds


def block_schedule(n: int):
    """The block round-robin schedule: list over outer rounds of lists (per block
    pair) of lists (per inner round) of the valid global pairs (p, q)."""
    L = _load()
    N = ((n + 2 * BLOCK - 1) // (2 * BLOCK)) * 2 * BLOCK
    nb = N // BLOCK
    p, q = ctypes.c_int(), ctypes.c_int()
    out = []
    for R in range(nb - 1):
        rnd = []
        for P in range(nb // 2):
            inner = []
            for rho in range(2 * BLOCK - 1):
                pairs = []
                for i in range(BLOCK):
                    if L.orc_block_pair(n, R, P, rho, i, ctypes.byref(p), ctypes.byref(q)):
                        pairs.append((p.value, q.value))
                inner.append(pairs)
            rnd.append(inner)
        out.append(rnd)
    return out


def round_half(x: float) -> float:
    """The oracle's rounding of an FP32 value to IEEE binary16 (as a float)."""
    return float(_load().orc_round_half(x))


def ns_steps(n: int, half: bool = False) -> int:
    """Newton-Schulz steps the oracle takes for size n (single or half stage 1)."""
    return int(_load().orc_ns_steps(n, int(half)))


def jacobi(A, V=None, *, ordering=CYCLIC, tol=0.0, skip_tol=U_D, max_sweeps=30, paper_mode=False,
           dtype=np.float64, skip_abs=0.0):
    """Cyclic Jacobi sweeps (Algorithm 4) on a copy of A; returns (A_final, V, sweeps, rotations, off, capped).

    dtype float64 runs the FP64 loop, float32 the FP32 loop (stage 1)."""
    L = _load()
    n = np.asarray(A).shape[0]
    sw, rot, of = ctypes.c_int(), ctypes.c_longlong(), _d()
    if dtype == np.float16:
        a = np.array(np.asarray(A, dtype=np.float16), dtype=np.float32, order="F")
        v = np.array(np.eye(n) if V is None else V, dtype=np.float32, order="F")
        capped = L.orc_jacobi_h(n, _ptr(a, _fp), n, _ptr(v, _fp), n, ordering, tol, skip_tol, max_sweeps,
                                ctypes.byref(sw), ctypes.byref(rot), ctypes.byref(of))
        return a, v, sw.value, rot.value, of.value, bool(capped)
    if dtype == np.float32:
        a = np.array(A, dtype=np.float32, order="F")
        v = np.array(np.eye(n) if V is None else V, dtype=np.float32, order="F")
        capped = L.orc_jacobi_f(n, _ptr(a, _fp), n, _ptr(v, _fp), n, ordering, tol, skip_tol, max_sweeps,
                                ctypes.byref(sw), ctypes.byref(rot), ctypes.byref(of))
    else:
        a = _f64(A)
        v = _f64(np.eye(n) if V is None else V)
        capped = L.orc_jacobi_d(n, _ptr(a), n, _ptr(v), n, ordering, tol, skip_tol, max_sweeps, int(paper_mode),
                                ctypes.byref(sw), ctypes.byref(rot), ctypes.byref(of), skip_abs)
    return a, v, sw.value, rot.value, of.value, bool(capped)


def gemm(A, B, trans_a=False, trans_b=False) -> np.ndarray:
    """Plain triple-loop product op(A) op(B) in double."""
    L = _load()
    a, b = _f64(A), _f64(B)
    if trans_a and trans_b:
        raise ValueError("not needed")
    if trans_a:
        k, m = a.shape
        n = b.shape[1]
        c = np.zeros((m, n), order="F")
        L.orc_gemm_tn_d(m, n, k, _ptr(a), a.shape[0], _ptr(b), b.shape[0], _ptr(c), m)
    elif trans_b:
        m, k = a.shape
        n = b.shape[0]
        c = np.zeros((m, n), order="F")
        L.orc_gemm_nt_d(m, n, k, _ptr(a), a.shape[0], _ptr(b), b.shape[0], _ptr(c), m)
    else:
        m, k = a.shape
        n = b.shape[1]
        c = np.zeros((m, n), order="F")
        L.orc_gemm_nn_d(m, n, k, _ptr(a), a.shape[0], _ptr(b), b.shape[0], _ptr(c), m)
    return c


def newton_schulz(X, steps: int | None = None) -> np.ndarray:
    """Eq. (itNS): X <- X (3I - X^T X) / 2, `steps` times (2 for n < 52000, else 3)."""
    x = _f64(X)
    n = x.shape[0]
    if steps is None:
        steps = 2 if n < 52000 else 3
    _load().orc_newton_schulz_d(n, _ptr(x), n, steps)
    return x


def precondition(A, Qd) -> np.ndarray:
    """Algorithm 9 step 3: A_cond = Q_d^T A Q_d."""
    a, q = _f64(A), _f64(Qd)
    n = a.shape[0]
    c = np.zeros((n, n), order="F")
    _load().orc_precondition_d(n, _ptr(a), n, _ptr(q), n, _ptr(c), n)
    return c


def stage1(A, **kw):
    """Stage 1: FP32 Jacobi from the identity on fl32(A).  Returns (Q_l, A32_final, Info)."""
    a = _f64(A)
    n = a.shape[0]
    ql = np.zeros((n, n), order="F")
    a32 = np.zeros((n, n), dtype=np.float32, order="F")
    ci = _Info()
    _load().orc_stage1(n, _ptr(a), n, _ptr(ql), n, ctypes.byref(_opts(n, **kw)), ctypes.byref(ci), _ptr(a32, _fp))
    return ql, a32, _info(ci)


def syev_mixed(A, *, return_intermediates=False, **kw):
    """Algorithm 9 with an FP32 Jacobi stage 1.  Returns (W, Q, Info[, dict of Q_l, Q_d, A_cond]).

    stage1_half=True runs stage 1 in half precision (binary16) with the
    Newton-Schulz step count of orc_ns_steps; raises PremiseError when
    ||Q_l^T Q_l - I||_2 >= 2 (the iteration's convergence premise).

    precond_passes=2 applies stages 1-3 a second time to A_cond before the
    FP64 sweeps (not in the paper; see orc_syev_mixed)."""
    a = _f64(A)
    n = a.shape[0]
    W = np.zeros(n)
    Q = np.zeros((n, n), order="F")
    ci = _Info()
    inter = {k: np.zeros((n, n), order="F") for k in ("Ql", "Qd", "Acond")} if return_intermediates else None
    rc = _load().orc_syev_mixed(n, _ptr(a), n, _ptr(W), _ptr(Q), n, ctypes.byref(_opts(n, **kw)), ctypes.byref(ci),
                                _ptr(inter["Ql"]) if inter else _ptr(None),
                                _ptr(inter["Qd"]) if inter else _ptr(None),
                                _ptr(inter["Acond"]) if inter else _ptr(None))
    if rc == 2:
        raise PremiseError(f"||Q_l^T Q_l - I||_2 = {ci.ns_e0:.3g} >= 2")
    if return_intermediates:
        return W, Q, _info(ci), inter
    return W, Q, _info(ci)


def syev_plain(A, **kw):
    """Plain FP64 Jacobi from V = I.  Returns (W, Q, Info)."""
    a = _f64(A)
    n = a.shape[0]
    W = np.zeros(n)
    Q = np.zeros((n, n), order="F")
    ci = _Info()
    _load().orc_syev_plain(n, _ptr(a), n, _ptr(W), _ptr(Q), n, ctypes.byref(_opts(n, **kw)), ctypes.byref(ci))
    return W, Q, _info(ci)


def sample_rotations(A, nrot: int, dtype=np.float64) -> float:
    """Run the first `nrot` rotations of a cyclic sweep on a copy of A (timing
    sample); returns the seconds the C loop took."""
    import time
    n = A.shape[0]
    a = np.array(A, dtype=dtype, order="F")
    v = np.asfortranarray(np.eye(n, dtype=dtype))
    L = _load()
    t0 = time.perf_counter()
    L.orc_sample_rotations(n, a.ctypes.data, n, v.ctypes.data, n, nrot, 0 if dtype == np.float64 else 1)
    return time.perf_counter() - t0


def sample_gemm(A, B) -> float:
    """Time one oracle product A @ B (plain triple loop); returns seconds."""
    import time
    a, b = _f64(A), _f64(B)
    m, k = a.shape
    n = b.shape[1]
    c = np.zeros((m, n), order="F")
    L = _load()
    t0 = time.perf_counter()
    L.orc_gemm_nn_d(m, n, k, _ptr(a), m, _ptr(b), k, _ptr(c), m)
    return time.perf_counter() - t0


def eigh_backward(W, Q, dW=None, dQ=None) -> np.ndarray:
    """dA = sym(Q (diag(dW) + F o (Q^T dQ)) Q^T), F_ij = 1/(w_j - w_i)."""
    w = np.ascontiguousarray(W, dtype=np.float64)
    q = _f64(Q)
    n = q.shape[0]
    dw = None if dW is None else np.ascontiguousarray(dW, dtype=np.float64)
    dq = None if dQ is None else _f64(dQ)
    dA = np.zeros((n, n), order="F")
    rc = _load().orc_eigh_backward(n, _ptr(w), _ptr(q), n, _ptr(dw), _ptr(dq), n, _ptr(dA), n)
    if rc != 0:
        raise ZeroDivisionError("repeated eigenvalue with nonzero coupling")
    return dA
