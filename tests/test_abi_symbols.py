"""The C-ABI library builds for sm_103a, loads, and exports every function
include/*.h declares (no GPU needed: nothing here launches a kernel)."""
import ctypes
import glob
import os
import re

import pytest

from paper_2402_17794_gb300 import _build, _lib

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = []
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        names += re.findall(r"^\s*(?:const\s+)?[\w\s\*]*?\b(rsvd_\w+)\s*\(", text, flags=re.M)
    return sorted(set(names))


@pytest.fixture(scope="module")
def lib():
    try:
        _build.nvcc_path()
    except RuntimeError:
        pytest.skip("nvcc not available")
    path = _build.build()
    return ctypes.CDLL(path)


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("rsvd_plan_create", "rsvd_solve", "rsvd_gaussian", "rsvd_apply_a",
                     "rsvd_apply_at", "rsvd_orth", "rsvd_small_svd", "rsvd_plan_status"):
        assert required in names


def test_every_declared_symbol_is_exported(lib):
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_covers_every_symbol():
    assert set(declared_functions()) <= set(_lib.SIGNATURES)


def test_status_strings_and_argument_checks_without_gpu(lib):
    lib.rsvd_status_string.restype = ctypes.c_char_p
    assert lib.rsvd_status_string(0) == b"ok"
    assert lib.rsvd_status_string(-3) == b"invalid argument"
    assert b"Cholesky" in lib.rsvd_status_string(1)
    # argument validation happens before any CUDA call
    h = ctypes.c_void_p()
    f = lib.rsvd_plan_create
    f.argtypes = [ctypes.POINTER(ctypes.c_void_p), ctypes.c_int64, ctypes.c_int64, ctypes.c_int,
                  ctypes.c_int, ctypes.c_int, ctypes.c_void_p]
    assert f(None, 10, 10, 4, 0, 0, None) == -1
    assert f(ctypes.byref(h), 0, 10, 4, 0, 0, None) == -2
    assert f(ctypes.byref(h), 10, 0, 4, 0, 0, None) == -3
    assert f(ctypes.byref(h), 10, 10, 0, 0, 0, None) == -4
    assert f(ctypes.byref(h), 10, 10, 289, 0, 0, None) == -4
    assert f(ctypes.byref(h), 10, 10, 4, 9, 0, None) == -5
    assert f(ctypes.byref(h), 10, 10, 4, 0, 1, None) == -6   # plain FP64 only
    lib.rsvd_solve.argtypes = [ctypes.c_void_p] * 1 + [ctypes.c_void_p, ctypes.c_int64,
                                                        ctypes.c_int64, ctypes.c_int64, ctypes.c_int,
                                                        ctypes.c_int, ctypes.c_int, ctypes.c_uint64,
                                                        ctypes.c_void_p, ctypes.c_int64,
                                                        ctypes.c_void_p, ctypes.c_void_p,
                                                        ctypes.c_int64]
    assert lib.rsvd_solve(None, None, 1, 1, 1, 1, 0, 0, 0, None, 1, None, None, 1) == -1


def test_library_source_never_touches_the_oracle():
    pkg = os.path.join(ROOT, "paper_2402_17794_gb300")
    for path in glob.glob(os.path.join(pkg, "**", "*.*"), recursive=True):
        if path.endswith((".py", ".cu", ".h", ".cuh")):
            text = open(path).read()
            assert "import oracle" not in text and "from oracle" not in text, path
