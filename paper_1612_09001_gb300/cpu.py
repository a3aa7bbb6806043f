"""ctypes binding of the portable SIMD + OpenMP CPU filter (include/dpd_cpu.h).

A CPU product path beside the GPU library, for like-for-like CPU comparisons;
it fails loudly when lib/libdpd_cpu.so is missing."""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "lib", "libdpd_cpu.so")
_lib = None


def load(path: str | None = None):
    global _lib
    if _lib is None or path:
        p = path or LIB_PATH
        if not os.path.exists(p):
            raise RuntimeError(f"{p} is missing: run paper_1612_09001_gb300.build.build_cpu()")
        lib = ctypes.CDLL(p)
        lib.dpd_cpu_apply.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p,
                                      ctypes.c_void_p, ctypes.c_int64, ctypes.c_int]
        lib.dpd_cpu_apply.restype = ctypes.c_int
        lib.dpd_cpu_max_threads.argtypes = []
        lib.dpd_cpu_max_threads.restype = ctypes.c_int
        if path:
            return lib
        _lib = lib
    return _lib


def max_threads() -> int:
    return load().dpd_cpu_max_threads()


def apply(x, h, P: int, Q: int, M: int, threads: int = 0, out=None) -> np.ndarray:
    """y = DPD(x) on the host cores (complex64 numpy arrays)."""
    x = np.ascontiguousarray(x, dtype=np.complex64)
    h = np.ascontiguousarray(h, dtype=np.complex64)
    y = np.empty_like(x) if out is None else out
    if y.dtype != np.complex64 or not y.flags.c_contiguous or y.shape != x.shape:
        raise ValueError("out must be a contiguous complex64 array like x")
    rc = load().dpd_cpu_apply(P, Q, M, h.ctypes.data, x.ctypes.data, y.ctypes.data, x.shape[0], threads)
    if rc != 0:
        raise ValueError("dpd_cpu_apply: invalid arguments")
    return y
