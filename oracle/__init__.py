"""FP64 CPU oracle for the augmented-parallel-Hammerstein DPD filter.

TEST INFRASTRUCTURE ONLY.  The test suite, the smoke check and the benchmark's
CPU-baseline leg are the only callers allowed; the CUDA library never imports,
links or executes anything here, and this package imports nothing from it.

Two independent formulations are provided:

* ``apply`` / ``grad`` / ``gram`` / ``chol_solve`` / ``ls``: plain C loops in
  double precision (``dpd_oracle.c``) that follow Eq. 1 and Algorithm 1 term by
  term, the normal equations of Sec. 2.2, and a textbook Cholesky solve.
* ``basis.basis_matrix`` / ``basis.apply`` / ``basis.lstsq``: the basis matrix of
  Eq. 2 built with numpy, used to cross-check the loops.

Inputs may be complex64 (they are upcast exactly) or complex128.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

from . import basis  # noqa: F401
from .build import build as _build, LIB_PATH

__all__ = ["apply", "grad", "gram", "chol_solve", "ls", "num_coeffs", "threads", "basis", "load"]

_lock = threading.Lock()
_lib = None

_c_double_p = ctypes.POINTER(ctypes.c_double)


def load(path: str | None = None):
    """Load (building first if needed) the oracle shared library."""
    global _lib
    with _lock:
        if path is not None:
            return _bind(ctypes.CDLL(path))
        if _lib is None:
            if not os.path.exists(LIB_PATH):
                _build()
            _lib = _bind(ctypes.CDLL(LIB_PATH))
        return _lib


def _bind(lib):
    i64 = ctypes.c_int64
    ci = ctypes.c_int
    vp = ctypes.c_void_p
    lib.oracle_num_coeffs.argtypes = [ci, ci, ci]
    lib.oracle_num_coeffs.restype = ci
    lib.oracle_apply.argtypes = [ci, ci, ci, vp, vp, i64, vp, ci]
    lib.oracle_apply.restype = ci
    lib.oracle_grad.argtypes = [ci, ci, ci, vp, vp, vp, i64, vp, vp, ci]
    lib.oracle_grad.restype = ci
    lib.oracle_gram.argtypes = [ci, ci, ci, vp, vp, i64, vp, vp, ci]
    lib.oracle_gram.restype = ci
    lib.oracle_chol_solve.argtypes = [ci, vp, vp, vp]
    lib.oracle_chol_solve.restype = ci
    lib.oracle_threads.argtypes = [ci]
    lib.oracle_threads.restype = ci
    return lib


def _c128(a):
    a = np.ascontiguousarray(np.asarray(a).astype(np.complex128, copy=False))
    return a


def _ptr(a):
    return a.ctypes.data if a is not None and a.size else None


def num_coeffs(P, Q, M, lib=None):
    lib = lib or load()
    return lib.oracle_num_coeffs(P, Q, M)


def threads(nthreads=0, lib=None):
    lib = lib or load()
    return lib.oracle_threads(nthreads)


def apply(x, h, P, Q, M, nthreads=0, lib=None):
    """y_n = sum_p sum_k h_{p,k} psi_p(x_{n-k}) + sum_q sum_k hbar_{q,k} psibar_q(x_{n-k}) + c."""
    lib = lib or load()
    x = _c128(x)
    h = _c128(h)
    K = lib.oracle_num_coeffs(P, Q, M)
    if K < 0 or h.shape[0] != K:
        raise ValueError(f"bad model or coefficient count (P={P}, Q={Q}, M={M}, len(h)={h.shape[0]})")
    y = np.empty_like(x)
    rc = lib.oracle_apply(P, Q, M, _ptr(h), _ptr(x), x.shape[0], _ptr(y), nthreads)
    if rc:
        raise RuntimeError(f"oracle_apply failed: {rc}")
    return y


def grad(x, h, gy, P, Q, M, want_h=True, want_x=True, nthreads=0, lib=None):
    """(gh, gx) for a real loss with dL/dy = gy, gradients as dL/dRe + j dL/dIm."""
    lib = lib or load()
    x = _c128(x)
    h = _c128(h)
    gy = _c128(gy)
    K = lib.oracle_num_coeffs(P, Q, M)
    if K < 0 or h.shape[0] != K or gy.shape != x.shape:
        raise ValueError("bad arguments")
    gh = np.zeros(K, np.complex128) if want_h else None
    gx = np.zeros_like(x) if want_x else None
    rc = lib.oracle_grad(P, Q, M, _ptr(h), _ptr(x), _ptr(gy), x.shape[0],
                         _ptr(gh) if want_h else None, _ptr(gx) if want_x else None, nthreads)
    if rc:
        raise RuntimeError(f"oracle_grad failed: {rc}")
    return gh, gx


def gram(u, t, P, Q, M, nthreads=0, lib=None):
    """(G, b) = (Psi^H Psi, Psi^H t), Psi = Psi(u) of Eq. 2.  t may be None."""
    lib = lib or load()
    u = _c128(u)
    K = lib.oracle_num_coeffs(P, Q, M)
    if K < 0:
        raise ValueError("bad model")
    tt = _c128(t) if t is not None else None
    G = np.zeros((K, K), np.complex128)
    b = np.zeros(K, np.complex128)
    rc = lib.oracle_gram(P, Q, M, _ptr(u), _ptr(tt) if tt is not None else None, u.shape[0],
                         _ptr(G), _ptr(b), nthreads)
    if rc:
        raise RuntimeError(f"oracle_gram failed: {rc}")
    return G, (b if t is not None else None)


def chol_solve(G, b, lib=None):
    """Solve G h = b for Hermitian positive definite G (raises on a non-positive pivot)."""
    lib = lib or load()
    G = _c128(G)
    b = _c128(b)
    K = b.shape[0]
    h = np.zeros(K, np.complex128)
    rc = lib.oracle_chol_solve(K, _ptr(G), _ptr(b), _ptr(h))
    if rc == 6:
        raise np.linalg.LinAlgError("matrix is not positive definite")
    if rc:
        raise RuntimeError(f"oracle_chol_solve failed: {rc}")
    return h


def ls(u, t, P, Q, M, nthreads=0, lib=None):
    """Least-squares estimate of Sec. 2.2: h = (Psi^H Psi)^{-1} Psi^H t."""
    G, b = gram(u, t, P, Q, M, nthreads=nthreads, lib=lib)
    return chol_solve(G, b, lib=lib)
