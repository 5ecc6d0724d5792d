"""The C-ABI library builds, loads and exports every symbol include/nefe.h declares (no GPU)."""
import ctypes
import os
import re

import pytest

from paper_2103_10449_gb300 import build as B
from paper_2103_10449_gb300 import nefe as N

HEADER = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include", "nefe.h")


def declared_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"NEFE_API\s+(?:const\s+)?\w+\s*\*?\s*(nefe_\w+)\s*\(", src)))


def test_library_builds_and_exports_every_declared_symbol():
    path = B.build()
    assert os.path.exists(path)
    lib = ctypes.CDLL(path)
    names = declared_functions()
    assert len(names) >= 25
    missing = [n for n in names if not hasattr(lib, n)]
    assert missing == []
    # and the binding wraps every one of them
    assert set(names) == set(N.SIGNATURES) | {"nefe_last_error"}


def test_debug_bounds_library_builds_and_exports_every_declared_symbol():
    """The debug flavour (index checks on every atom index read from device data) is the same
    sources with NEFE_DEBUG_BOUNDS: it builds beside the normal library and exports the same
    C ABI."""
    path = B.build(debug=True)
    assert os.path.basename(path) == "libnefe_debug.so" and os.path.exists(path)
    lib = ctypes.CDLL(path)
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert missing == []


def test_host_only_calls_work_without_gpu():
    p = N.nefe_sw_params_silicon()
    assert (p.eps, p.sigma, p.A, p.B, p.p, p.q, p.a, p.lambda3, p.gamma) == (
        2.1683, 2.0951, 7.049556277, 0.6022245584, 4.0, 0.0, 1.80, 21.0, 1.20)
    assert p.cos0 == pytest.approx(-1.0 / 3.0)


def test_invalid_arguments_are_rejected_before_any_device_work():
    L = N.load()
    rc = L.nefe_neighbor_build(None, -1, (ctypes.c_double * 3)(10, 10, 10), 4.0, 48, None, None, None, None)
    assert rc == N.NEFE_EINVAL
    assert b"bad argument" in L.nefe_last_error()
    rc = L.nefe_create(None, 0, None, 0, 0.001, 0.5, 48)
    assert rc == N.NEFE_EINVAL
    h = ctypes.c_void_p()
    rc = L.nefe_create(ctypes.byref(h), 0, None, 7, 0.001, 0.5, 48)
    assert rc == N.NEFE_EINVAL
    assert L.nefe_destroy(None) == N.NEFE_OK
    # context-level tuning calls reject a missing context; the barrier check rejects its limit
    # before touching a device
    assert L.nefe_set_rebuild_policy(None, 1) == N.NEFE_EINVAL
    assert L.nefe_set_cooperative_rebuild(None, 1) == N.NEFE_EINVAL
    assert L.nefe_check_barrier_timeout(0, 0.0) == N.NEFE_EINVAL
    assert L.nefe_check_barrier_timeout(0, 5000.0) == N.NEFE_EINVAL
    assert b"limit_ms" in L.nefe_last_error()


def test_product_path_has_no_oracle_dependency():
    pkg = os.path.dirname(B.__file__)
    for root, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".h", ".cuh")):
                txt = open(os.path.join(root, f)).read()
                assert not re.search(r"^\s*(import|from)\s+oracle", txt, flags=re.M), f
                assert "liboracle" not in txt and "nefe_oracle" not in txt, f
