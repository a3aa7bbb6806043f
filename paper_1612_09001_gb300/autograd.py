"""torch.autograd.Function around dpd_apply / dpd_grad.

The backward pass calls the library's hand-written adjoint kernels, which
recompute the polynomial basis from the saved input instead of storing it.
Gradients follow PyTorch's complex convention (dL/dRe + j dL/dIm for a real
loss L), which is also the convention of dpd_grad.
"""
from __future__ import annotations

import torch

from . import DPD, _check_samples


class DPDFunction(torch.autograd.Function):
    """y = DPD_h(x).  Usage: ``DPDFunction.apply(x, h, filt)`` with ``filt`` a
    ``DPD`` handle of the right (P, Q, M); x and h complex64 CUDA tensors."""

    @staticmethod
    def _install(filt: DPD, h):
        """set_coeffs unless h (same tensor, unchanged since) is already installed:
        fixed stages (a transmitter model) then cost no table rebuild per call.
        A tensor modified in place bumps its version and is installed again."""
        key = (id(h), h.data_ptr(), h._version)
        if getattr(filt, "_installed", None) != key:
            filt.set_coeffs(h)
            filt._installed = key

    @staticmethod
    def forward(ctx, x, h, filt: DPD):
        _check_samples(x, "x")
        _check_samples(h, "h")
        DPDFunction._install(filt, h)
        y = filt.apply(x)
        ctx.save_for_backward(x, h)
        ctx.filt = filt
        return y

    @staticmethod
    def backward(ctx, gy):
        x, h = ctx.saved_tensors
        filt = ctx.filt
        need_x, need_h = ctx.needs_input_grad[0], ctx.needs_input_grad[1]
        gy = gy.contiguous()
        gx = torch.empty_like(x) if need_x else None
        gh = torch.empty_like(h) if need_h else None
        if need_x:
            DPDFunction._install(filt, h)
        if need_x or need_h:
            filt.grad(x, gy, gh=gh, gx=gx)
        return gx, gh, None


def dpd(x, h, filt: DPD):
    """Differentiable predistortion y = DPD_h(x)."""
    return DPDFunction.apply(x, h, filt)
