"""ctypes loader for ``librsvd_gb300.so`` (the C ABI of include/rsvd.h).

Argument marshalling only.  If the shared object is missing this raises:
the library has no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os

from ._build import LIB_PATH

c_int, c_int64, c_uint32, c_uint64 = ctypes.c_int, ctypes.c_int64, ctypes.c_uint32, ctypes.c_uint64
c_void_p, c_size_t = ctypes.c_void_p, ctypes.c_size_t
P_double = ctypes.c_void_p

class RsvdProblem(ctypes.Structure):
    """rsvd_problem_t of include/rsvd.h."""
    _fields_ = [("A", c_void_p), ("m", c_int64), ("n", c_int64), ("lda", c_int64),
                ("k", c_int), ("p", c_int), ("q", c_int), ("seed", c_uint64),
                ("U", c_void_p), ("ldu", c_int64), ("S", c_void_p), ("VT", c_void_p),
                ("ldvt", c_int64)]


class RsvdGemm(ctypes.Structure):
    """rsvd_gemm_t of include/rsvd.h."""
    _fields_ = [("A", c_void_p), ("lda", c_int64), ("X", c_void_p), ("ldx", c_int64),
                ("C", c_void_p), ("ldc", c_int64), ("M", c_int64), ("K", c_int64),
                ("N", c_int), ("x_upper", c_int)]


# name -> (restype, argtypes), in the order of include/rsvd.h
SIGNATURES = {
    "rsvd_plan_create": (c_int, [ctypes.POINTER(c_void_p), c_int64, c_int64, c_int, c_int, c_int,
                                 c_void_p]),
    "rsvd_workspace_size": (c_int, [c_void_p, ctypes.POINTER(c_size_t)]),
    "rsvd_set_workspace": (c_int, [c_void_p, c_void_p, c_size_t]),
    "rsvd_plan_status": (c_int, [c_void_p]),
    "rsvd_plan_set_stream": (c_int, [c_void_p, c_void_p]),
    "rsvd_plan_set_wait_limit": (c_int, [c_void_p, c_int64]),
    "rsvd_plan_prepare_a": (c_int, [c_void_p, c_void_p, c_int64, c_int64, c_int64]),
    "rsvd_plan_release_a": (c_int, [c_void_p]),
    "rsvd_set_tile_scales": (c_int, [c_void_p, c_void_p, c_int64, c_int64, c_int64]),
    "rsvd_plan_diagnostics": (c_int, [c_void_p, ctypes.POINTER(c_int), ctypes.POINTER(c_int)]),
    "rsvd_plan_destroy": (c_int, [c_void_p]),
    "rsvd_status_string": (ctypes.c_char_p, [c_int]),
    "rsvd_kernel_launches": (c_uint64, []),
    "rsvd_solve": (c_int, [c_void_p, c_void_p, c_int64, c_int64, c_int64, c_int, c_int, c_int,
                           c_uint64, c_void_p, c_int64, P_double, c_void_p, c_int64]),
    "rsvd_solve_algorithm": (c_int, [c_void_p, c_int, c_void_p, c_int64, c_int64, c_int64, c_int,
                                     c_int, c_int, c_uint64, c_void_p, c_int64, c_void_p, c_void_p,
                                     c_int64]),
    "rsvd_solve_singlepass": (c_int, [c_void_p, c_void_p, c_int64, c_int64, c_int64, c_int, c_int,
                                      c_uint64, c_void_p, c_int64, c_void_p, c_void_p, c_int64]),
    "rsvd_solve_hermitian": (c_int, [c_void_p, c_void_p, c_int64, c_int64, c_int, c_int,
                                     c_uint64, c_void_p, c_int64, c_void_p]),
    "rsvd_range_adaptive": (c_int, [c_void_p, c_void_p, c_int64, c_int64, c_int64, ctypes.c_double,
                                    c_int, c_int, c_uint64, c_void_p, c_int64,
                                    ctypes.POINTER(c_int)]),
    "rsvd_solve_adaptive": (c_int, [c_void_p, c_void_p, c_int64, c_int64, c_int64, ctypes.c_double,
                                    c_int, c_int, c_uint64, c_void_p, c_int64, c_void_p,
                                    c_void_p, c_int64, ctypes.POINTER(c_int)]),
    "rsvd_range_srft": (c_int, [c_void_p, c_void_p, c_int64, c_int64, c_int64, c_int, c_uint64,
                                c_void_p, c_int64]),
    "rsvd_solve_srft": (c_int, [c_void_p, c_void_p, c_int64, c_int64, c_int64, c_int, c_int,
                                c_uint64, c_void_p, c_int64, c_void_p, c_void_p, c_int64]),
    "rsvd_srft_sketch": (c_int, [c_void_p, c_void_p, c_int64, c_int64, c_int64, c_int, c_uint64,
                                 c_void_p, c_int64]),
    "rsvd_gaussian": (c_int, [c_void_p, c_int64, c_int, c_uint64, c_uint32, c_int, c_void_p,
                              c_int64]),
    "rsvd_apply_a": (c_int, [c_void_p, c_void_p, c_int64, c_int64, c_int64, c_void_p, c_int64,
                             c_int, c_void_p, c_int64]),
    "rsvd_apply_at": (c_int, [c_void_p, c_void_p, c_int64, c_int64, c_int64, c_void_p, c_int64,
                              c_int, c_void_p, c_int64]),
    "rsvd_apply_split": (c_int, [c_void_p, c_void_p, c_int64, c_int64, c_int64, c_int, c_void_p,
                                 c_int64, c_int, c_int, c_void_p, c_int64]),
    "rsvd_orth": (c_int, [c_void_p, P_double, c_int64, c_int, c_int64, P_double, c_int64,
                          P_double, c_int64]),
    "rsvd_small_svd": (c_int, [c_void_p, P_double, c_int, c_int64, P_double, P_double, c_int64,
                               P_double, c_int64]),
    "rsvd_batch_plan_create": (c_int, [ctypes.POINTER(c_void_p), c_int, c_int64, c_int64, c_int,
                                       c_int, c_void_p]),
    "rsvd_solve_batched": (c_int, [c_void_p, c_int, ctypes.POINTER(RsvdProblem)]),
    "rsvd_batch_status": (c_int, [c_void_p, c_int, ctypes.POINTER(c_int)]),
    "rsvd_batch_set_engine": (c_int, [c_void_p, c_int]),
    "rsvd_batch_set_graphs": (c_int, [c_void_p, c_int]),
    "rsvd_batch_set_sm_limit": (c_int, [c_void_p, c_int]),
    "rsvd_batch_autotune": (c_int, [c_void_p, c_int, ctypes.POINTER(RsvdProblem)]),
    "rsvd_grouped_gemm_f32": (c_int, [c_void_p, c_int, ctypes.POINTER(RsvdGemm), c_int]),
    "rsvd_grouped_schedule": (c_int, [c_int, ctypes.POINTER(c_int64), c_int, c_int,
                                      ctypes.POINTER(c_int), c_int, ctypes.POINTER(c_int),
                                      ctypes.POINTER(c_int)]),
    "rsvd_apply_a_f64_static": (c_int, [c_void_p, c_int64, c_int64, c_int64, c_void_p, c_int64,
                                        c_int, c_void_p, c_int64, c_void_p]),
}

_LIB = None


def load(path: str | None = None) -> ctypes.CDLL:
    """Load the shared object (once) and attach the C signatures."""
    global _LIB
    if _LIB is not None and path is None:
        return _LIB
    path = path or LIB_PATH
    if not os.path.exists(path):
        raise RuntimeError(
            f"CUDA library {path} is not built; run "
            "`python -c 'import __graft_entry__ as g; g.build()'` first")
    lib = ctypes.CDLL(path)
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    if path == LIB_PATH:
        _LIB = lib
    return lib
