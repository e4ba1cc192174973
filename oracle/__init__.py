"""CPU oracle for the Boys functions (test infrastructure only).

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The library under
``paper_2504_07637_gb300`` never does, and shares no code with it.

The arithmetic lives in ``boys_oracle.c`` (long double); this module only
compiles it with gcc and marshals numpy arrays through ctypes.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "boys_oracle.c")
_LIB = os.path.join(_HERE, "libboys_oracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle into ``libboys_oracle.so`` next to its source."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".{os.getpid()}.tmp"
        subprocess.check_call(
            ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fno-fast-math", _SRC, "-o", tmp, "-lm"]
        )
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        lib = ctypes.CDLL(build())
        i64, c_int, vp = ctypes.c_int64, ctypes.c_int, ctypes.c_void_p
        for name, args in {
            "boys_oracle_eval": [vp, i64, c_int, vp],
            "boys_oracle_eval_ld": [vp, i64, c_int, vp],
            "boys_oracle_series_ld": [vp, i64, c_int, vp],
            "boys_oracle_erf_upward_ld": [vp, i64, c_int, vp],
            "boys_oracle_quad_ld": [vp, i64, c_int, vp],
            "boys_oracle_grad": [vp, vp, i64, i64, i64, c_int, vp],
            "boys_oracle_grad_ld": [vp, vp, i64, i64, i64, c_int, vp, vp],
        }.items():
            fn = getattr(lib, name)
            fn.argtypes = args
            fn.restype = c_int
        lib.boys_oracle_cutoff.argtypes = [c_int, c_int]
        lib.boys_oracle_cutoff.restype = ctypes.c_double
        lib.boys_oracle_upper_ratio_ld.argtypes = [c_int, vp, i64, vp]
        lib.boys_oracle_upper_ratio_ld.restype = c_int
        lib.boys_oracle_c_ld.argtypes = [c_int, vp]
        lib.boys_oracle_c_ld.restype = c_int
        lib.boys_oracle_precision_bits.argtypes = []
        lib.boys_oracle_precision_bits.restype = c_int
        _lib = lib
        return lib


def _check(rc: int) -> None:
    if rc != 0:
        raise ValueError(f"oracle rejected its arguments (code {rc})")


def precision_bits() -> int:
    """Significand bits of the oracle's long double (64 on x86-64, 113 on AArch64)."""
    return _load().boys_oracle_precision_bits()


def boys(x, n_max: int) -> np.ndarray:
    """F_0..F_{n_max} at float64 arguments, as float64 [count, n_max+1]."""
    x = np.ascontiguousarray(x, dtype=np.float64).ravel()
    out = np.empty((x.size, n_max + 1), dtype=np.float64)
    _check(_load().boys_oracle_eval(x.ctypes.data, x.size, n_max, out.ctypes.data))
    return out


def boys_threaded(x, n_max: int, threads: int) -> np.ndarray:
    """``boys`` split into contiguous chunks over ``threads`` host threads.

    ctypes releases the GIL during the foreign call, so the chunks run in
    parallel; the arithmetic is the same single-threaded oracle.
    """
    x = np.ascontiguousarray(x, dtype=np.float64).ravel()
    out = np.empty((x.size, n_max + 1), dtype=np.float64)
    lib = _load()
    bounds = np.linspace(0, x.size, max(1, threads) + 1).astype(np.int64)
    rcs = []

    def work(a: int, b: int) -> None:
        if b > a:
            rcs.append(lib.boys_oracle_eval(x[a:b].ctypes.data, b - a, n_max, out[a:b].ctypes.data))

    ts = [threading.Thread(target=work, args=(int(bounds[k]), int(bounds[k + 1]))) for k in range(len(bounds) - 1)]
    for t in ts:
        t.start()
    for t in ts:
        t.join()
    for rc in rcs:
        _check(rc)
    return out


def boys_ld(x, n_max: int) -> np.ndarray:
    """F_0..F_{n_max} in long double, [count, n_max+1]."""
    x = np.ascontiguousarray(x, dtype=np.longdouble).ravel()
    out = np.empty((x.size, n_max + 1), dtype=np.longdouble)
    _check(_load().boys_oracle_eval_ld(x.ctypes.data, x.size, n_max, out.ctypes.data))
    return out


def series_ld(x, n: int) -> np.ndarray:
    """F_n by the positive series alone (long double)."""
    x = np.ascontiguousarray(x, dtype=np.longdouble).ravel()
    out = np.empty(x.size, dtype=np.longdouble)
    _check(_load().boys_oracle_series_ld(x.ctypes.data, x.size, n, out.ctypes.data))
    return out


def erf_upward_ld(x, n_max: int) -> np.ndarray:
    """F_0..F_{n_max} by erf and the upward recursion alone (long double)."""
    x = np.ascontiguousarray(x, dtype=np.longdouble).ravel()
    out = np.empty((x.size, n_max + 1), dtype=np.longdouble)
    _check(_load().boys_oracle_erf_upward_ld(x.ctypes.data, x.size, n_max, out.ctypes.data))
    return out


def quad_ld(x, n: int) -> np.ndarray:
    """F_n by Gauss-Legendre quadrature of the definition (long double)."""
    x = np.ascontiguousarray(x, dtype=np.longdouble).ravel()
    out = np.empty(x.size, dtype=np.longdouble)
    _check(_load().boys_oracle_quad_ld(x.ctypes.data, x.size, n, out.ctypes.data))
    return out


def grad(x, g, n_max: int) -> np.ndarray:
    """-sum_m g[i, m] F_{m+1}(x_i) for g of shape [count, n_max+1] (any strides)."""
    x = np.ascontiguousarray(x, dtype=np.float64).ravel()
    g = np.asarray(g, dtype=np.float64)
    if g.shape != (x.size, n_max + 1):
        g = np.broadcast_to(g, (x.size, n_max + 1))
    rs, cs = (s // 8 for s in g.strides)
    if g.strides[0] % 8 or g.strides[1] % 8:
        g = np.ascontiguousarray(g)
        rs, cs = n_max + 1, 1
    out = np.empty(x.size, dtype=np.float64)
    _check(_load().boys_oracle_grad(x.ctypes.data, g.ctypes.data, rs, cs, x.size, n_max, out.ctypes.data))
    return out


def grad_ld(x, g, n_max: int):
    """Long-double gradient and its normaliser sum_m |g_m| F_{m+1}."""
    x = np.ascontiguousarray(x, dtype=np.longdouble).ravel()
    g = np.ascontiguousarray(np.broadcast_to(np.asarray(g, dtype=np.longdouble), (x.size, n_max + 1)))
    out = np.empty(x.size, dtype=np.longdouble)
    scale = np.empty(x.size, dtype=np.longdouble)
    _check(
        _load().boys_oracle_grad_ld(
            x.ctypes.data, g.ctypes.data, n_max + 1, 1, x.size, n_max, out.ctypes.data, scale.ctypes.data
        )
    )
    return out, scale


def cutoff(n: int, bits: int) -> float:
    """z_nb: the root of R(n+1/2, z) = 2^-b (Sec. 2 cut-off)."""
    return float(_load().boys_oracle_cutoff(n, bits))


def upper_ratio_ld(n: int, x) -> np.ndarray:
    """R(n+1/2, x) = Gamma(n+1/2, x)/Gamma(n+1/2) in long double."""
    x = np.ascontiguousarray(x, dtype=np.longdouble).ravel()
    out = np.empty(x.size, dtype=np.longdouble)
    _check(_load().boys_oracle_upper_ratio_ld(n, x.ctypes.data, x.size, out.ctypes.data))
    return out


def c_ld(n_max: int) -> np.ndarray:
    """c_0..c_{n_max}, c_n = Gamma(n+1/2)/2, in long double."""
    out = np.empty(n_max + 1, dtype=np.longdouble)
    _check(_load().boys_oracle_c_ld(n_max, out.ctypes.data))
    return out
