"""ctypes declarations of the C ABI in include/wq.h (argument marshalling only)."""
from __future__ import annotations

import ctypes
import os

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libwq.so")

c_int, c_i64, c_vp, c_dp = ctypes.c_int, ctypes.c_int64, ctypes.c_void_p, ctypes.POINTER(ctypes.c_double)

STATUS = {0: "WQ_OK", 1: "WQ_ERR_INVALID_ARG", 2: "WQ_ERR_UNSUPPORTED", 3: "WQ_ERR_SINGULAR_RULE",
          4: "WQ_ERR_BAD_GEOMETRY", 5: "WQ_ERR_OOM", 6: "WQ_ERR_CUDA", 7: "WQ_ERR_TIMEOUT",
          8: "WQ_ERR_INJECTED", 9: "WQ_ERR_NONFINITE"}

# void* alloc(size_t bytes, void* stream, void* ctx); void free(void* ptr, void* stream, void* ctx)
ALLOC_FN = ctypes.CFUNCTYPE(c_vp, ctypes.c_size_t, c_vp, c_vp)
FREE_FN = ctypes.CFUNCTYPE(None, c_vp, c_vp, c_vp)


class Options(ctypes.Structure):
    """struct wq_options of include/wq.h."""
    _fields_ = [("size", ctypes.c_size_t), ("value_dtype", c_int), ("precision", c_int), ("algorithm", c_int),
                ("tile", c_int * 2), ("checked", c_int), ("tune_cache", ctypes.c_char_p),
                ("alloc", ALLOC_FN), ("free", FREE_FN), ("alloc_ctx", c_vp), ("scratch_limit", ctypes.c_size_t)]

# name -> (restype, argtypes)
SIGNATURES = {
    "wq_options_init": (c_int, [ctypes.POINTER(Options)]),
    "wq_plan_create": (c_int, [ctypes.POINTER(c_vp), c_int, c_int, ctypes.POINTER(c_i64),
                               ctypes.POINTER(c_vp), c_vp, ctypes.POINTER(Options), c_vp]),
    "wq_destroy": (c_int, [c_vp]),
    "wq_plan_destroy": (c_int, [c_vp]),
    "wq_plan_reserve": (c_int, [c_vp, c_int, c_int, c_int, c_vp]),
    "wq_plan_info": (c_int, [c_vp, ctypes.POINTER(c_int), ctypes.POINTER(c_i64), ctypes.POINTER(c_i64),
                             ctypes.POINTER(c_i64), ctypes.POINTER(c_i64)]),
    "wq_plan_pattern": (c_int, [c_vp, ctypes.POINTER(c_vp), ctypes.POINTER(c_vp)]),
    "wq_plan_set_geometry": (c_int, [c_vp, c_vp, c_int, c_vp]),
    "wq_plan_refresh": (c_int, [c_vp, c_vp, c_int, c_vp]),
    "wq_plan_set_weights": (c_int, [c_vp, c_vp, c_int, c_int, c_vp]),
    "wq_plan_set_tensor": (c_int, [c_vp, c_vp, c_vp]),
    "wq_assemble_stiffness": (c_int, [c_vp, c_vp, c_vp, c_int, c_int, c_vp]),
    "wq_assemble_mass": (c_int, [c_vp, c_vp, c_vp, c_int, c_int, c_vp]),
    "wq_assemble_host": (c_int, [c_vp, c_int, c_vp, c_vp, c_vp, c_vp]),
    "wq_assemble_load": (c_int, [c_vp, c_vp, c_vp, c_vp]),
    "wq_host_alloc": (c_int, [ctypes.c_size_t, ctypes.POINTER(c_vp)]),
    "wq_host_free": (c_int, [c_vp]),
    "wq_sync_check": (c_int, [c_vp, c_vp]),
    "wq_last_error": (ctypes.c_char_p, []),
    "wq_status_string": (ctypes.c_char_p, [c_int]),
    "wq_launch_count": (c_i64, []),
    "wq_get_nq_max": (c_int, [c_vp, ctypes.POINTER(c_int)]),
    "wq_get_points": (c_int, [c_vp, c_int, c_vp]),
    "wq_get_rules": (c_int, [c_vp, c_int, c_int, c_int, c_vp, c_vp, c_vp]),
    "wq_get_coefficients": (c_int, [c_vp, c_vp]),
    "wq_adjoint": (c_int, [c_vp, c_int, c_vp, c_vp, c_vp, c_vp, c_vp, c_vp, c_vp]),
    "wq_batch_create": (c_int, [ctypes.POINTER(c_vp), c_int, c_vp, c_vp, c_vp, c_vp]),
    "wq_batch_launch": (c_int, [c_vp, c_vp]),
    "wq_batch_assemble": (c_int, [c_vp, c_vp]),
    "wq_batch_info": (c_int, [c_vp, ctypes.POINTER(c_i64), ctypes.POINTER(c_i64), ctypes.POINTER(c_int)]),
    "wq_batch_destroy": (c_int, [c_vp]),
    "wq_plan_set_algorithm": (c_int, [c_vp, c_int]),
    "wq_plan_set_tiles": (c_int, [c_vp, c_int, c_int]),
    "wq_plan_get_tiles": (c_int, [c_vp, ctypes.POINTER(c_int), ctypes.POINTER(c_int)]),
    "wq_rules_noalloc": (c_int, [c_int, c_i64, c_vp, c_vp, c_vp, c_vp, c_int, c_vp]),
}

_lib = None


class WqError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


def load(path: str = LIB_PATH):
    """Load libwq.so; raises if it has not been built (there is no fallback)."""
    global _lib
    if _lib is None:
        if not os.path.exists(path):
            raise ImportError(f"libwq.so is not built ({path}); run __graft_entry__.build()")
        lib = ctypes.CDLL(path)
        for name, (res, args) in SIGNATURES.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
    return _lib


def check(status: int) -> None:
    if status != 0:
        raise WqError(status, load().wq_last_error().decode())
