"""The C-ABI library builds for sm_103a, loads without a GPU and exports every entry point
declared in include/wect.h (no compute call is made here)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    with open(os.path.join(ROOT, "include", "wect.h")) as fh:
        text = fh.read()
    return sorted(set(re.findall(r"^WECT_API\s+[^;(]*?\b([a-z_][a-z0-9_]*)\s*\(", text, flags=re.M)))


@pytest.fixture(scope="module")
def lib_path():
    from paper_2511_03909_gb300 import _build

    return _build.build()


def test_header_declares_the_boundary():
    names = declared_symbols()
    for must in ("wect_complex_create_cubical", "wect_complex_create_simplicial", "wect_compute", "ecf_compute",
                 "wect_backward", "wect_batch_create", "wect_batch_compute", "wect_complex_destroy", "wect_last_error"):
        assert must in names


def test_library_exports_every_declared_symbol(lib_path):
    lib = ctypes.CDLL(lib_path)
    missing = [n for n in declared_symbols() if not hasattr(lib, n)]
    assert not missing, f"not exported: {missing}"


def test_binding_matches_header(lib_path):
    import paper_2511_03909_gb300 as P

    assert sorted(P.exported_symbols()) == declared_symbols()
    L = P.load()
    assert L.wect_version().decode().startswith("wect-gb300")
    assert L.wect_last_error().decode() == ""


def test_argument_errors_need_no_gpu(lib_path):
    """Argument checks run on the host before any CUDA call."""
    import paper_2511_03909_gb300 as P

    L = P.load()
    h = ctypes.c_void_p()
    dims = (ctypes.c_int64 * 2)(4, 4)
    assert L.wect_complex_create_cubical(0, dims, None, P.W_ONE, 0, None, ctypes.byref(h)) == 1
    assert L.wect_complex_create_cubical(4, dims, None, P.W_ONE, 0, None, ctypes.byref(h)) == 1
    bad = (ctypes.c_int64 * 2)(0, 4)
    assert L.wect_complex_create_cubical(2, bad, None, P.W_ONE, 0, None, ctypes.byref(h)) == 1
    assert L.wect_complex_create_cubical(2, dims, None, 9, 0, None, ctypes.byref(h)) == 1
    assert L.wect_complex_create_cubical(2, dims, None, P.W_F32, 99, None, ctypes.byref(h)) == 1
    assert L.wect_compute(None, None, 1, 8, 0.0, 1.0, None, None) == 1
    assert L.wect_compute_host(None, None, None, 1, 8, 0.0, 1.0, None, None) == 1
    assert b"NULL" in L.wect_last_error()
