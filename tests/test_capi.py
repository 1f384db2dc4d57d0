"""The C ABI: the library builds, loads and exports every entry point that
include/*.h declares; host-side argument checks need no GPU."""
import ctypes
import glob
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="session")
def libpath():
    from paper_2509_00495_gb300 import build
    return build.build()


def declared_functions():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        src = open(h).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        for m in re.finditer(r"^\s*(?:const\s+)?[A-Za-z_][\w\s\*]*?\b(mpj_\w+)\s*\(", src, flags=re.M):
            names.add(m.group(1))
    return sorted(names)


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ["mpj_syev", "mpj_syev_ex", "mpj_syev_workspace", "mpj_syev_batched", "mpj_syev_backward",
                     "mpj_status_str", "mpj_stage1", "mpj_newton_schulz", "mpj_precondition", "mpj_jacobi64",
                     "mpj_dgemm", "mpj_opts_default", "mpj_last_cuda_error"]:
        assert required in names


def test_library_exports_every_declared_symbol(libpath):
    L = ctypes.CDLL(libpath)
    missing = [n for n in declared_functions() if not hasattr(L, n)]
    assert not missing, missing


def test_host_side_helpers_without_gpu(libpath):
    from paper_2509_00495_gb300 import mpj
    L = mpj.lib()
    assert mpj.status_str(0) == "MPJ_OK"
    assert mpj.status_str(-3) == "MPJ_ENONFINITE"
    o = mpj.default_opts()
    assert o.ordering == mpj.ORDER_BLOCK and o.method == mpj.METHOD_MIXED and o.sort == 1
    # workspace grows like n^2 and is zero for n = 0
    assert mpj.syev_workspace(0) == 0
    w1, w2 = mpj.syev_workspace(512), mpj.syev_workspace(1024)
    assert 3.5 < w2 / w1 < 4.5
    # argument errors are caught on the host before any CUDA call
    assert L.mpj_syev(-1, None, 1, None, None, 0.0, None) == mpj.MPJ_EINVAL
    assert L.mpj_syev(4, None, 4, None, None, 0.0, None) == mpj.MPJ_EINVAL
    assert L.mpj_dgemm(b"X", b"N", 2, 2, 2, 1.0, None, 2, None, 2, 0.0, None, 2, None) == mpj.MPJ_EINVAL
    assert L.mpj_jacobi64(4, ctypes.c_void_p(8), 2, ctypes.c_void_p(8), 4, 0.0, 1, 0, None, None, None) == mpj.MPJ_EINVAL
    bad = mpj.default_opts(ordering=7)
    assert L.mpj_syev_ex(4, ctypes.c_void_p(8), 4, ctypes.c_void_p(8), ctypes.c_void_p(8), 4, ctypes.byref(bad), None,
                         None, 0, None) == mpj.MPJ_EINVAL


def test_binding_refuses_cpu_tensors(libpath):
    import torch
    from paper_2509_00495_gb300 import mpj
    with pytest.raises(TypeError):
        mpj.syev(torch.eye(3, dtype=torch.float64))


def test_more_host_side_argument_checks(libpath):
    """Entry points added later reject bad arguments on the host as well."""
    from paper_2509_00495_gb300 import mpj
    L = mpj.lib()
    p = ctypes.c_void_p(256)
    # stage-1 panel: N a multiple of 32, R in range, known mode bits, test mode only for N <= 256
    assert L.mpj_stage1_panel(48, 0, p, p, p, 0, None) == mpj.MPJ_EINVAL
    assert L.mpj_stage1_panel(64, 3, p, p, p, 0, None) == mpj.MPJ_EINVAL
    assert L.mpj_stage1_panel(64, 0, p, p, p, 4, None) == mpj.MPJ_EINVAL
    assert L.mpj_stage1_panel(512, 0, p, p, p, 2, None) == mpj.MPJ_EINVAL
    assert L.mpj_stage1_panel(64, 0, p, p, p, 1, None) == mpj.MPJ_EINVAL  # transposing in place
    # allocation-free sweeps: too large before any device work
    big = 8193
    z = ctypes.c_double(0.0)
    assert L.mpj_jacobi64_noalloc(big, p, big, p, big, z, 1, 0, None, None, None) == -9  # MPJ_ETOOLARGE
    assert L.mpj_jacobi64_noalloc(4, p, 4, p, 4, z, 5, 0, None, None, None) == mpj.MPJ_EINVAL
    # batched: sizes outside [1, 256]
    n_bad = (ctypes.c_int * 2)(3, 300)
    assert L.mpj_syev_batched(2, n_bad, p, p, p, 0.0, None, None) == mpj.MPJ_EINVAL
    assert L.mpj_syev_batched(0, None, None, None, None, 0.0, None, None) == 0


def test_bench_reference_arm_contract():
    """bench.py --impl reference prints one JSON line with the contract's keys
    (the oracle timed on bounded samples; no GPU involved)."""
    import json
    import subprocess
    import sys
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                          "--warmup", "0", "--ref-step-seconds", "0.5"], capture_output=True, text=True,
                         timeout=600, cwd=ROOT)
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [l for l in out.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for k in ["metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better", "scaling",
              "dtype", "data", "config", "impl", "cpu_baseline", "e2e"]:
        assert k in d, k
    assert d["impl"] == "reference" and d["value"] > 0 and d["higher_is_better"] is True
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["cores"] >= 1
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["e2e"]["value"] == d["value"]


def test_allocation_counter_is_exported(libpath):
    from paper_2509_00495_gb300 import mpj
    L = mpj.lib()
    L.mpj_device_allocations.restype = ctypes.c_longlong
    assert L.mpj_device_allocations() >= 0


def test_noalloc_size_limit_on_the_host(libpath):
    """The fixed scratch of mpj_jacobi64_noalloc holds n = MPJ_NOALLOC_MAX_N:
    8192 passes the host-side size check (and then fails at the first CUDA call,
    there being no device here), 8193 is refused with MPJ_ETOOLARGE.  Never run
    with a device present: the pointers are placeholders."""
    import torch
    if torch.cuda.is_available():
        pytest.skip("host-only check (placeholder pointers)")
    from paper_2509_00495_gb300 import mpj
    L = mpj.lib()
    p = ctypes.c_void_p(256)
    fn = L.mpj_jacobi64_noalloc
    fn.argtypes = [ctypes.c_int, ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p, ctypes.c_int, ctypes.c_double,
                   ctypes.c_int, ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]
    assert fn(8193, p, 8193, p, 8193, 1.0, 1, 1, None, None, None) == -9
    assert fn(8192, p, 8192, p, 8192, 1.0, 1, 1, None, None, None) == mpj.MPJ_ECUDA
