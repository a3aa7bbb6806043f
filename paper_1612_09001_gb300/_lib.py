"""ctypes binding of libdpd.so (include/dpd.h).  Argument marshalling only.

The library is built in-tree by ``paper_1612_09001_gb300.build``.  There is no
fallback: if the shared library is missing or cannot be loaded, every call
raises.
"""
from __future__ import annotations

import ctypes
import os
import threading

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "lib", "libdpd.so")

STATUS = {
    0: "DPD_OK",
    1: "DPD_ERR_INVALID_ARGUMENT",
    2: "DPD_ERR_UNSUPPORTED",
    3: "DPD_ERR_NO_COEFFS",
    4: "DPD_ERR_CUDA",
    5: "DPD_ERR_ALLOC",
    6: "DPD_ERR_NOT_SPD",
    7: "DPD_ERR_TIMEOUT",
}
DPD_HOST, DPD_DEVICE = 0, 1
DPD_PREC_FP32, DPD_PREC_TF32X3, DPD_PREC_BF16X3 = 0, 1, 2
DPD_HOST_PIPELINED, DPD_HOST_ZERO_COPY = 0, 1
DPD_BASIS_MONOMIAL, DPD_BASIS_ORTHOGONAL = 0, 1


class DPDError(RuntimeError):
    def __init__(self, func: str, code: int):
        self.code = code
        super().__init__(f"{func} failed: {STATUS.get(code, code)}")


_lock = threading.Lock()
_lib = None

_i = ctypes.c_int
_i64 = ctypes.c_int64
_vp = ctypes.c_void_p
_pi = ctypes.POINTER(ctypes.c_int)

# name -> argtypes; every function returns dpd_status (int) unless listed in _RESTYPE.
SIGNATURES = {
    "dpd_create": [_i, _i, _i, ctypes.POINTER(_vp)],
    "dpd_destroy": [_vp],
    "dpd_num_coeffs": [_vp, _pi],
    "dpd_set_coeffs": [_vp, _vp, _i, _i, _vp],
    "dpd_apply": [_vp, _vp, _vp, _i64, _vp],
    "dpd_apply_host": [_vp, _vp, _vp, _i64, _i, _vp],
    "dpd_apply_stream": [_vp, _vp, _vp, _i64, _vp],
    "dpd_set_estimate_basis": [_vp, _i],
    "dpd_sq_error": [_vp, _vp, _vp, _i64, ctypes.c_float, ctypes.c_float, ctypes.c_double, _vp, _vp, _vp],
    "dpd_reset_stream": [_vp, _vp],
    "dpd_set_fwd_launch": [_vp, _i, _i, _i, _i, _i, _i, _i],
    "dpd_grad": [_vp, _vp, _vp, _i64, _vp, _vp, _vp],
    "dpd_set_adj_launch": [_vp, _i, _i],
    "dpd_grad_coeffs_noalloc": [_i, _i, _i, _vp, _vp, _i64, _vp, _vp],
    "dpd_probe_fma": [_i, _i, _i, _vp, _vp],
    "dpd_sync_status": [_vp, _vp],
    "dpd_gram": [_vp, _vp, _vp, _i64, _i, _vp, _vp, ctypes.POINTER(ctypes.c_double), _vp],
    "dpd_estimate": [_vp, _vp, _vp, _i64, _i, _i, _vp, ctypes.POINTER(ctypes.c_double), _vp],
    "dpd_estimate_batched": [_vp, _vp, _vp, _vp, _i, _i, _i, _vp, _pi, _vp],
    "dpd_plan_batched": [_vp, _i, _i, ctypes.POINTER(_vp)],
    "dpd_exec_batched": [_vp, _vp],
    "dpd_plan_set_launch": [_vp, _i, _i, _i, _i, _i],
    "dpd_plan_sync_status": [_vp, _vp],
    "dpd_plan_destroy": [_vp],
    "dpd_status_string": [_i],
    "dpd_kernel_launches": [],
}
class StreamDesc(ctypes.Structure):
    """dpd_stream_desc of include/dpd.h."""
    _fields_ = [("x", _vp), ("y", _vp), ("n", _i64), ("P", _i), ("Q", _i), ("M", _i), ("h", _vp)]


_RESTYPE = {"dpd_status_string": ctypes.c_char_p, "dpd_kernel_launches": ctypes.c_uint64}


def load(path: str | None = None):
    """Load libdpd.so (raises if it has not been built)."""
    global _lib
    with _lock:
        if _lib is not None and path is None:
            return _lib
        p = path or LIB_PATH
        if not os.path.exists(p):
            raise RuntimeError(f"libdpd.so not found at {p}; build it with "
                               "paper_1612_09001_gb300.build.build()")
        lib = ctypes.CDLL(p)
        for name, args in SIGNATURES.items():
            fn = getattr(lib, name)
            fn.argtypes = args
            fn.restype = _RESTYPE.get(name, _i)
        if path is None:
            _lib = lib
        return lib


def check(func: str, code: int):
    if code != 0:
        raise DPDError(func, code)
