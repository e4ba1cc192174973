"""ctypes binding of libboys.so: the same names as include/boys.h.

Argument marshalling only.  There is no CPU fallback: if the library cannot
be loaded, every call raises.
"""
from __future__ import annotations

import ctypes
import os
import threading

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libboys.so")
_lock = threading.Lock()
_lib = None

vp, i64, i32, c_int, c_double, c_size = (
    ctypes.c_void_p,
    ctypes.c_int64,
    ctypes.c_int32,
    ctypes.c_int,
    ctypes.c_double,
    ctypes.c_size_t,
)

# name -> (restype, argtypes); kept in the order of include/boys.h
SIGNATURES = {
    "boys_status_string": (ctypes.c_char_p, [c_int]),
    "boys_max_n": (c_int, [c_int]),
    "boys_cutoff": (c_double, [c_int, c_int]),
    "boys_top_order_f64": (c_int, [c_int]),
    "boys_eval_f64": (c_int, [vp, i64, c_int, vp, vp]),
    "boys_top_order_f32": (c_int, [c_int]),
    "boys_eval_f32": (c_int, [vp, i64, c_int, vp, vp]),
    "boys_eval_backward_f64": (c_int, [vp, vp, i64, vp, i64, i64, i64, c_int, vp, vp]),
    "boys_eval_f64_two_point": (c_int, [vp, i64, c_int, vp, vp]),
    "boys_eval_contract_f64": (c_int, [vp, i64, c_int, vp, i64, i64, vp, vp]),
    "boys_eval_contract_f32": (c_int, [vp, i64, c_int, vp, i64, i64, vp, vp]),
    "boys_eval_f64_host_workspace": (c_size, [c_int, i64]),
    "boys_eval_f64_host": (c_int, [vp, i64, c_int, vp, vp, c_size, vp]),
    "boys_ragged_workspace_bytes": (c_size, [i32]),
    "boys_ragged_max_n": (c_int, []),
    "boys_ragged_num_variants": (c_int, []),
    "boys_ragged_variant_info": (c_int, [c_int, vp, vp]),
    "boys_eval_ragged_f64": (c_int, [vp, i64, vp, vp, vp, i32, vp, i64, vp, c_size, c_int, vp]),
    "boys_ragged_errors": (c_int, [vp, vp, vp]),
    "boys_eval_ragged_f64_noalloc": (c_int, [vp, i64, vp, vp, vp, i32, vp, i64, c_int, vp]),
    "boys_eval_f32_host_workspace": (c_size, [c_int, i64]),
    "boys_eval_f32_host": (c_int, [vp, i64, c_int, vp, vp, c_size, vp]),
    # include/boys_microbench.h
    "boys_microbench_launch": (c_int, [c_int, i64, vp, c_int, vp]),
    "boys_microbench_ops_per_thread_iter": (c_int, []),
    "boys_microbench_dfma": (c_int, [c_int, i64, vp, c_int, vp]),
    "boys_microbench_int": (c_int, [c_int, i64, vp, c_int, vp]),
    "boys_microbench_int_insts_per_chain_iter": (c_int, [c_int]),
    "boys_debug_exp_neg": (c_int, [vp, i64, vp, vp]),
}


class BoysError(RuntimeError):
    """A non-zero boys_status returned by the library."""

    def __init__(self, fn: str, code: int):
        self.code = code
        super().__init__(f"{fn} failed: {status_string(code)} (code {code})")


def load(build_if_missing: bool = True):
    """Load libboys.so (building it in-tree first if it is absent)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if not os.path.exists(LIB_PATH) and build_if_missing:
            from .build import build_library

            build_library()
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: build it with paper_2504_07637_gb300.build")
        lib = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in SIGNATURES.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
        return lib


def status_string(code: int) -> str:
    return load().boys_status_string(code).decode()


def call(name: str, *args) -> None:
    """Call an entry point returning boys_status; raise BoysError on failure."""
    rc = getattr(load(), name)(*args)
    if rc != 0:
        raise BoysError(name, rc)

