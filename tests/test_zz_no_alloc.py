"""The allocation-free FP64 sweep entry point, mpj_jacobi64_noalloc.

It exists for callers that may not allocate device memory during a call (a
fully committed memory budget, allocator-free latency-critical loops, hosts
where allocation calls are not allowed at that point); its scratch is one
fixed device array shared by all calls.  Checked through the C ABI against
mpj_jacobi64 (which allocates its scratch) on two calls in a row, with the
tolerances the other GPU tests use.  Collected last on purpose.
"""
import ctypes

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

U = 2.0 ** -53


@pytest.fixture(scope="module")
def lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2509_00495_gb300 import build, mpj
    build.build()
    L = mpj.lib()
    vp, i, d = ctypes.c_void_p, ctypes.c_int, ctypes.c_double
    L.mpj_jacobi64_noalloc.argtypes = [i, vp, i, vp, i, d, i, i, ctypes.POINTER(i), ctypes.POINTER(d), vp]
    L.mpj_jacobi64.argtypes = [i, vp, i, vp, i, d, i, i, ctypes.POINTER(i), ctypes.POINTER(d), vp]
    return L


def _run(fn, A_np, ordering):
    n = A_np.shape[0]
    A = torch.from_numpy(np.ascontiguousarray(A_np)).cuda()  # symmetric: row- = column-major
    V = torch.eye(n, dtype=torch.float64, device="cuda")
    sw, off = ctypes.c_int(), ctypes.c_double()
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    st = fn(n, ctypes.c_void_p(A.data_ptr()), n, ctypes.c_void_p(V.data_ptr()), n, 0.0, ordering, 0,
            ctypes.byref(sw), ctypes.byref(off), stream)
    torch.cuda.synchronize()
    # column-major V seen row-major is V^T
    return st, A.cpu().numpy(), V.cpu().numpy().T, sw.value, off.value


@pytest.mark.parametrize("n,ordering", [(97, 1), (256, 1), (40, 0)])
def test_noalloc_matches_allocating_entry_point(lib, n, ordering):
    from paper_2509_00495_gb300 import inputs
    A, lam = inputs.geo_matrix(n, 1e3, seed=n)
    st0, a0, v0, sw0, off0 = _run(lib.mpj_jacobi64, A, ordering)
    assert st0 == 0
    nA = np.linalg.norm(A, 2)
    for _ in range(2):  # two calls in a row share the same fixed scratch
        st, a, v, sw, off = _run(lib.mpj_jacobi64_noalloc, A, ordering)
        assert st == 0 and sw == sw0
        assert off <= n * U * np.linalg.norm(A)
        assert np.abs(np.diag(a) - np.diag(a0)).max() <= 1e-13 * nA
        assert np.abs(v - v0).max() <= 1e-10
        assert np.linalg.norm(A @ v - v * np.diag(a)) <= 4 * n * U * nA


def test_noalloc_where_the_fixed_array_shortens_the_v_batches(lib):
    """n = 2048: the fixed array holds only 32 rounds of V multipliers per batch
    (the allocating entry point batches 64 and overlaps them on a side
    stream); the rotation sequence and its arithmetic are the same, so the
    results agree with mpj_jacobi64, on two calls in a row."""
    from paper_2509_00495_gb300 import inputs
    n = 2048
    rng = np.random.default_rng(12)
    lam = np.sort(rng.uniform(-1.0, 1.0, n))
    A = inputs.near_diagonal(n, lam, 1e-4, seed=12)
    st0, a0, v0, sw0, off0 = _run(lib.mpj_jacobi64, A, 1)
    assert st0 == 0
    nA = np.linalg.norm(A, 2)
    for _ in range(2):
        st, a, v, sw, off = _run(lib.mpj_jacobi64_noalloc, A, 1)
        assert st == 0 and sw == sw0
        assert np.abs(np.diag(a) - np.diag(a0)).max() <= 1e-13 * nA
        assert np.abs(v - v0).max() <= 1e-10


def test_noalloc_accepts_its_largest_size(lib):
    """n = MPJ_NOALLOC_MAX_N = 8192 fits the fixed array (with fewer rounds per V
    batch); a diagonal input converges before the first sweep."""
    n = 8192
    A = torch.diag(torch.linspace(-1.0, 1.0, n, dtype=torch.float64, device="cuda"))
    V = torch.eye(n, dtype=torch.float64, device="cuda")
    sw, off = ctypes.c_int(), ctypes.c_double()
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    st = lib.mpj_jacobi64_noalloc(n, ctypes.c_void_p(A.data_ptr()), n, ctypes.c_void_p(V.data_ptr()), n, 0.0, 1, 0,
                                  ctypes.byref(sw), ctypes.byref(off), stream)
    torch.cuda.synchronize()
    assert st == 0 and sw.value == 0 and off.value == 0.0


def test_noalloc_rejects_sizes_beyond_its_scratch(lib):
    from paper_2509_00495_gb300 import mpj
    big = 8193  # one past MPJ_NOALLOC_MAX_N; rejected on the host before any device work
    st = lib.mpj_jacobi64_noalloc(big, ctypes.c_void_p(8), big, ctypes.c_void_p(8), big, 0.0, 1, 0, None, None, None)
    assert st == -9 and mpj.status_str(st) == "MPJ_ETOOLARGE"
