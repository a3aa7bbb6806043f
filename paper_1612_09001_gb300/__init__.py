"""GB300-native augmented-parallel-Hammerstein (APH) digital predistortion.

Python face of ``libdpd.so`` (C ABI in ``include/dpd.h``).  Every step of the
filter runs in the library's CUDA kernels; this module only checks tensor
types and passes pointers, sizes and the current CUDA stream.  PyTorch supplies
device memory and streams.

    import torch, paper_1612_09001_gb300 as dpd
    f = dpd.DPD(P=9, Q=9, M=4)
    f.set_coeffs(h)                 # complex64, K values, stacking order of Sec. 2.2
    y = f.apply(x)                  # x: complex64 CUDA tensor
"""
from __future__ import annotations

import ctypes

from . import _lib
from ._lib import DPDError, DPD_HOST, DPD_DEVICE, DPD_PREC_FP32, DPD_PREC_TF32X3, DPD_PREC_BF16X3  # noqa: F401

PRECISIONS = {"fp32": DPD_PREC_FP32, "tf32x3": DPD_PREC_TF32X3, "bf16x3": DPD_PREC_BF16X3}
BASES = {"monomial": _lib.DPD_BASIS_MONOMIAL, "orthogonal": _lib.DPD_BASIS_ORTHOGONAL}

__all__ = ["DPD", "BatchedPlan", "DPDError", "num_coeffs", "kernel_launches", "lib"]


def lib():
    return _lib.load()


def num_coeffs(P: int, Q: int, M: int) -> int:
    bp = (P + 1) // 2 if P > 0 else 0
    bq = (Q + 1) // 2 if Q > 0 else 0
    return (bp + bq) * (M + 1) + 1


def kernel_launches() -> int:
    """Kernels launched by libdpd in this process so far."""
    return int(lib().dpd_kernel_launches())


def _stream_ptr(stream):
    import torch
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream)


def _check_samples(t, name):
    import torch
    if not isinstance(t, torch.Tensor):
        raise TypeError(f"{name} must be a torch.Tensor")
    if t.dtype != torch.complex64:
        raise TypeError(f"{name} must be complex64, got {t.dtype}")
    if not t.is_cuda:
        raise ValueError(f"{name} must be a CUDA tensor")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")


def _batch_pointers(xs, name):
    """Device addresses (uint64) and lengths (int64) of a batch of sample
    vectors given as a list of 1-D complex64 CUDA tensors, or as one contiguous
    2-D tensor of equal-length problems (problems x samples; its rows are the
    vectors).  Returns (addresses, lengths, device)."""
    import numpy as np
    import torch
    if isinstance(xs, torch.Tensor):
        _check_samples(xs, name)
        if xs.dim() != 2 or xs.shape[0] < 1 or xs.shape[1] < 1:
            raise ValueError(f"{name} must be a non-empty 2-D tensor (problems x samples) or a list of tensors")
        cnt, n = xs.shape
        addr = np.arange(cnt, dtype=np.uint64) * np.uint64(n * 8) + np.uint64(xs.data_ptr())
        return addr, np.full(cnt, n, dtype=np.int64), xs.device
    c64 = torch.complex64
    addr, lens = [], []
    for x in xs:   # one pass: the checks, the address and the length of each tensor
        if not (isinstance(x, torch.Tensor) and x.dtype is c64 and x.is_cuda and x.is_contiguous()):
            _check_samples(x, name)   # raises the specific error
        addr.append(x.data_ptr())
        lens.append(x.numel())
    if not addr:
        raise ValueError(f"{name} must not be empty")
    return np.array(addr, dtype=np.uint64), np.array(lens, dtype=np.int64), xs[0].device


class DPD:
    """One APH predistorter: orders P (main) and Q (conjugate), memory depth M."""

    def __init__(self, P: int, Q: int, M: int):
        self._lib = lib()
        h = ctypes.c_void_p()
        _lib.check("dpd_create", self._lib.dpd_create(P, Q, M, ctypes.byref(h)))
        self._h = h
        self.P, self.Q, self.M = P, Q, M
        k = ctypes.c_int()
        _lib.check("dpd_num_coeffs", self._lib.dpd_num_coeffs(self._h, ctypes.byref(k)))
        self.K = k.value
        self.fwd_launch = dict(mode=3, V=8, warps=16, stages=4, ctas_per_sm=0, use_tma=1, group=4)

    # -- lifetime
    def close(self):
        if getattr(self, "_h", None):
            self._lib.dpd_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    @property
    def handle(self):
        return self._h

    # -- coefficients
    def set_coeffs(self, h, stream=None):
        """Install K complex64 coefficients from a CUDA tensor, a CPU tensor or a numpy array."""
        import numpy as np
        import torch
        if isinstance(h, np.ndarray):
            h = torch.from_numpy(np.ascontiguousarray(h.astype(np.complex64)))
        if not isinstance(h, torch.Tensor) or h.dtype != torch.complex64 or h.numel() != self.K:
            raise ValueError(f"coefficients must be {self.K} complex64 values")
        h = h.contiguous()
        where = DPD_DEVICE if h.is_cuda else DPD_HOST
        self._coef_ref = h   # keep a device source alive until the kernel that reads it has run
        self._installed = None   # autograd's record of the installed tensor
        _lib.check("dpd_set_coeffs", self._lib.dpd_set_coeffs(
            self._h, ctypes.c_void_p(h.data_ptr()), self.K, where, _stream_ptr(stream)))

    # -- forward
    def apply(self, x, out=None, stream=None):
        """y = DPD(x) for a complex64 CUDA tensor (1-D or any shape, filtered as one stream)."""
        import torch
        _check_samples(x, "x")
        if out is None:
            out = torch.empty_like(x)
        else:
            _check_samples(out, "out")
            if out.numel() != x.numel():
                raise ValueError("out must have as many elements as x")
        _lib.check("dpd_apply", self._lib.dpd_apply(
            self._h, ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(out.data_ptr()),
            x.numel(), _stream_ptr(stream)))
        return out

    # -- adjoint
    def grad(self, x, gy, gh=None, gx=None, stream=None):
        """Gradients of a real loss through y = DPD(x) given gy = dL/dy (dL/dRe + j dL/dIm).

        Writes into gh (K complex64, CUDA) and/or gx (like x) when given; returns (gh, gx)."""
        _check_samples(x, "x")
        _check_samples(gy, "gy")
        if gy.numel() != x.numel():
            raise ValueError("gy must have as many elements as x")
        if gh is not None:
            _check_samples(gh, "gh")
            if gh.numel() != self.K:
                raise ValueError(f"gh must have {self.K} elements")
        if gx is not None:
            _check_samples(gx, "gx")
            if gx.numel() != x.numel():
                raise ValueError("gx must have as many elements as x")
        _lib.check("dpd_grad", self._lib.dpd_grad(
            self._h, ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(gy.data_ptr()), x.numel(),
            ctypes.c_void_p(gh.data_ptr() if gh is not None else None),
            ctypes.c_void_p(gx.data_ptr() if gx is not None else None), _stream_ptr(stream)))
        return gh, gx

    # -- least squares (Sec. 2.2)
    def gram(self, u, t=None, precision="tf32x3", stream=None, want_tt=True):
        """(G, g, tt): G = Psi^H Psi (K x K complex128 CUDA tensor), g = Psi^H t, tt = t^H t.

        tt is read back to the host (the call synchronises the stream) unless
        want_tt is False, in which case it is None and the call is asynchronous."""
        import torch
        _check_samples(u, "u")
        if t is not None:
            _check_samples(t, "t")
        G = torch.empty((self.K, self.K), dtype=torch.complex128, device=u.device)
        g = torch.empty(self.K, dtype=torch.complex128, device=u.device) if t is not None else None
        tt = ctypes.c_double(0.0)
        _lib.check("dpd_gram", self._lib.dpd_gram(
            self._h, ctypes.c_void_p(u.data_ptr()), ctypes.c_void_p(t.data_ptr() if t is not None else None),
            u.numel(), PRECISIONS[precision], ctypes.c_void_p(G.data_ptr()),
            ctypes.c_void_p(g.data_ptr() if g is not None else None),
            ctypes.byref(tt) if (t is not None and want_tt) else None, _stream_ptr(stream)))
        return G, g, (tt.value if (t is not None and want_tt) else None)

    def set_estimate_basis(self, basis):
        """Basis of the least-squares estimates: "monomial" or "orthogonal" (Sec. 2.1)."""
        _lib.check("dpd_set_estimate_basis", self._lib.dpd_set_estimate_basis(self._h, BASES[basis]))

    def estimate(self, u, t, precision="tf32x3", refine_iters=2, stream=None, basis=None):
        """Least-squares coefficients (complex64 CUDA tensor of K, monomial stacking order) and
        stats (condition estimate of the equilibrated Gram matrix of the basis used, relative
        residual).  basis: "monomial" or "orthogonal" sets the handle's estimate basis first."""
        import torch
        if basis is not None:
            self.set_estimate_basis(basis)
        _check_samples(u, "u")
        _check_samples(t, "t")
        h = torch.empty(self.K, dtype=torch.complex64, device=u.device)
        stats = (ctypes.c_double * 2)()
        _lib.check("dpd_estimate", self._lib.dpd_estimate(
            self._h, ctypes.c_void_p(u.data_ptr()), ctypes.c_void_p(t.data_ptr()), u.numel(),
            PRECISIONS[precision], refine_iters, ctypes.c_void_p(h.data_ptr()), stats, _stream_ptr(stream)))
        return h, {"cond_est": stats[0], "rel_residual": stats[1]}

    def estimate_batched(self, us, ts, precision="tf32x3", refine_iters=2, stream=None, basis=None):
        """Independent estimates of (u, t) pairs given as two lists of 1-D
        tensors, or as two 2-D tensors of equal-length problems (problems x
        samples); returns (count x K complex64 tensor, info list)."""
        import numpy as np
        import torch
        if basis is not None:
            self.set_estimate_basis(basis)
        up, ns, dev = _batch_pointers(us, "u")
        tp, nt, _ = _batch_pointers(ts, "t")
        if len(up) != len(tp) or not np.array_equal(ns, nt):
            raise ValueError("us and ts must hold the same number of problems, each t as long as its u")
        cnt = len(up)
        info = (ctypes.c_int * cnt)()
        h = torch.empty((cnt, self.K), dtype=torch.complex64, device=dev)
        rc = self._lib.dpd_estimate_batched(self._h, ctypes.c_void_p(up.ctypes.data), ctypes.c_void_p(tp.ctypes.data),
                                            ctypes.c_void_p(ns.ctypes.data), cnt, PRECISIONS[precision],
                                            refine_iters, ctypes.c_void_p(h.data_ptr()), info, _stream_ptr(stream))
        if rc not in (0, 6):
            _lib.check("dpd_estimate_batched", rc)
        return h, list(info)

    def set_adj_launch(self, gh_blocks, tap_group):
        _lib.check("dpd_set_adj_launch", self._lib.dpd_set_adj_launch(self._h, gh_blocks, tap_group))

    def apply_stream(self, x, out=None, stream=None):
        """Filter the next block of a continuous stream (history carried across calls)."""
        import torch
        _check_samples(x, "x")
        if out is None:
            out = torch.empty_like(x)
        else:
            _check_samples(out, "out")
            if out.numel() != x.numel():
                raise ValueError("out must have as many elements as x")
        _lib.check("dpd_apply_stream", self._lib.dpd_apply_stream(
            self._h, ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(out.data_ptr()), x.numel(),
            _stream_ptr(stream)))
        return out

    def sq_error(self, y, x, gain=1.0, scale=1.0, loss=None, gy=None, stream=None):
        """loss = scale * sum |y - gain x|^2 (one-element float32 CUDA tensor) and, when gy
        is given, gy = 2 scale (y - gain x); one pass on the device (dpd_sq_error)."""
        import torch
        _check_samples(y, "y")
        _check_samples(x, "x")
        if y.numel() != x.numel():
            raise ValueError("y and x must have the same length")
        if loss is None:
            loss = torch.empty(1, dtype=torch.float32, device=y.device)
        if gy is not None:
            _check_samples(gy, "gy")
        g = complex(gain)
        _lib.check("dpd_sq_error", self._lib.dpd_sq_error(
            self._h, ctypes.c_void_p(y.data_ptr()), ctypes.c_void_p(x.data_ptr()), y.numel(), g.real, g.imag,
            float(scale), ctypes.c_void_p(loss.data_ptr()), ctypes.c_void_p(gy.data_ptr() if gy is not None else None),
            _stream_ptr(stream)))
        return loss

    def reset_stream(self, stream=None):
        _lib.check("dpd_reset_stream", self._lib.dpd_reset_stream(self._h, _stream_ptr(stream)))

    def apply_host(self, x, out=None, stream=None, zero_copy=False):
        """y = DPD(x) for complex64 tensors in (pinned) host memory: chunked copy / compute
        pipeline, or zero copy (the kernel reads and writes the host buffers in place).
        Asynchronous: synchronise the stream before reading out."""
        import torch
        if not isinstance(x, torch.Tensor) or x.dtype != torch.complex64 or x.is_cuda or not x.is_contiguous():
            raise ValueError("x must be a contiguous complex64 host tensor")
        if out is None:
            out = torch.empty_like(x, pin_memory=x.is_pinned())
        elif out.dtype != torch.complex64 or out.is_cuda or not out.is_contiguous() or out.numel() != x.numel():
            raise ValueError("out must be a contiguous complex64 host tensor like x")
        _lib.check("dpd_apply_host", self._lib.dpd_apply_host(
            self._h, ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(out.data_ptr()), x.numel(),
            _lib.DPD_HOST_ZERO_COPY if zero_copy else _lib.DPD_HOST_PIPELINED, _stream_ptr(stream)))
        return out

    def set_fwd_launch(self, V=4, warps=8, stages=4, ctas_per_sm=0, use_tma=1, mode=0, group=0):
        _lib.check("dpd_set_fwd_launch", self._lib.dpd_set_fwd_launch(
            self._h, mode, V, warps, stages, ctas_per_sm, use_tma, group))
        self.fwd_launch = dict(mode=mode, V=V, warps=warps, stages=stages, ctas_per_sm=ctas_per_sm,
                               use_tma=use_tma, group=group)

    def sync_status(self, stream=None):
        """Synchronise the stream and raise if a kernel recorded an error."""
        _lib.check("dpd_sync_status", self._lib.dpd_sync_status(self._h, _stream_ptr(stream)))


class BatchedPlan:
    """Many independent streams filtered by one persistent launch.

    ``streams`` is a list of dicts with keys x, y (complex64 CUDA tensors), P, Q,
    M and h (K complex64 coefficients: numpy array, CPU or CUDA tensor; all on
    the same side).  The plan records the buffers; ``execute`` launches one
    kernel on the current (or given) stream and can be captured in a CUDA graph."""

    def __init__(self, streams):
        import numpy as np
        import torch
        self._lib = lib()
        n = len(streams)
        descs = (_lib.StreamDesc * max(n, 1))()
        keep = []
        where = None
        for i, st in enumerate(streams):
            x, y = st["x"], st["y"]
            _check_samples(x, "x")
            _check_samples(y, "y")
            if y.numel() != x.numel():
                raise ValueError("x and y of a stream must have the same length")
            h = st["h"]
            if isinstance(h, np.ndarray):
                h = torch.from_numpy(np.ascontiguousarray(h.astype(np.complex64)))
            if h.dtype != torch.complex64 or h.numel() != num_coeffs(st["P"], st["Q"], st["M"]):
                raise ValueError(f"stream {i}: coefficients must be K complex64 values")
            h = h.contiguous()
            w = DPD_DEVICE if h.is_cuda else DPD_HOST
            if where is None:
                where = w
            elif w != where:
                raise ValueError("all coefficient vectors must be on the same side (host or device)")
            keep.append(h)
            descs[i] = _lib.StreamDesc(x.data_ptr(), y.data_ptr(), x.numel(), st["P"], st["Q"], st["M"],
                                       h.data_ptr())
        p = ctypes.c_void_p()
        _lib.check("dpd_plan_batched", self._lib.dpd_plan_batched(
            ctypes.cast(descs, ctypes.c_void_p), n, DPD_HOST if where is None else where, ctypes.byref(p)))
        self._p = p
        self._streams = streams   # keep the recorded buffers alive

    def execute(self, stream=None):
        _lib.check("dpd_exec_batched", self._lib.dpd_exec_batched(self._p, _stream_ptr(stream)))

    def set_launch(self, V=8, warps=8, stages=4, ctas_per_sm=0, group=0):
        _lib.check("dpd_plan_set_launch", self._lib.dpd_plan_set_launch(self._p, V, warps, stages, ctas_per_sm, group))

    def sync_status(self, stream=None):
        _lib.check("dpd_plan_sync_status", self._lib.dpd_plan_sync_status(self._p, _stream_ptr(stream)))

    def close(self):
        if getattr(self, "_p", None):
            self._lib.dpd_plan_destroy(self._p)
            self._p = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
