"""Direct-learning predistortion through a transmitter model, and the indirect
learning architecture of Sec. 2.2 for comparison.

Direct learning: the predistorter coefficients h are trained by gradient
descent (Adam) on
    L(h) = ||TX(DPD_h(x)) - G x||^2 / ||x||^2,
where TX is a fixed transmitter model made of APH filters (an I/Q modulator
stage followed by a PA stage with memory).  Every stage is a DPDFunction, so
the gradients flow through the library's adjoint kernels: the PA and I/Q stages
contribute input gradients, the predistorter its coefficient gradient.  The
polynomial basis is recomputed from the saved stage inputs in the backward
pass (nothing else is kept).  One training step (forward through three
filters, loss, adjoint back through three filters, Adam) can be captured in a
CUDA graph and replayed.

Indirect learning (Sec. 2.2): iterate z = DPD_h(x), s = TX(z) / G,
h = argmin ||Psi(s) h - z|| (dpd_estimate), 1-3 times.
"""
from __future__ import annotations

import math
import time

import torch

from . import DPD
from .autograd import DPDFunction


class SqErrorLoss(torch.autograd.Function):
    """L = scale * ||y - gain x||^2 with its gradient produced in the same device
    pass (dpd_sq_error); backward scales the saved gradient by dL."""

    @staticmethod
    def forward(ctx, y, x, filt, gain, scale):
        gy = torch.empty_like(y)
        loss = filt.sq_error(y, x, gain=gain, scale=scale, gy=gy)
        ctx.save_for_backward(gy)
        return loss[0]

    @staticmethod
    def backward(ctx, gl):
        (gy,) = ctx.saved_tensors
        return gy * gl, None, None, None, None


class Transmitter:
    """A chain of fixed APH filter stages, each given as dict(P, Q, M, h)."""

    def __init__(self, stages, device="cuda"):
        self.stages = []
        for st in stages:
            f = DPD(st["P"], st["Q"], st["M"])
            h = torch.as_tensor(st["h"]).to(device=device, dtype=torch.complex64).contiguous()
            self.stages.append((f, h))

    def __call__(self, v):
        for f, h in self.stages:
            v = DPDFunction.apply(v, h, f)
        return v

    def apply(self, v):
        with torch.no_grad():
            return self(v)


def nmse_db(y, ref):
    """10 log10(||y - ref||^2 / ||ref||^2): both sums of squares on the device,
    read back together (one synchronisation)."""
    d = torch.view_as_real((y - ref).reshape(-1))
    r = torch.view_as_real(ref.reshape(-1).contiguous())
    e, s = torch.stack([d.square().sum(), r.square().sum()]).tolist()
    return 10.0 * math.log10(e / s)


class DirectLearner:
    """Adam on the predistorter coefficients through the transmitter model."""

    def __init__(self, x, tx, P, Q, M, gain=1.0, lr=1e-3, h0=None, eps=1e-8):
        self.x = x
        self.tx = tx
        self.filt = DPD(P, Q, M)
        if h0 is None:
            h0 = torch.zeros(self.filt.K, dtype=torch.complex64, device=x.device)
            h0[0] = 1.0   # start from the identity predistorter
        # The parameter is the real view (K x 2) of h: Adam treats complex
        # parameters as their real views anyway, and real ones can use the
        # single-kernel (fused) implementation.
        self.param = torch.nn.Parameter(torch.view_as_real(h0.clone().contiguous()).clone())
        self.gain = gain
        self.scale = 1.0 / float(x.abs().pow(2).sum())
        # The learning rate lives in device memory, so a captured step reads
        # the current value and a schedule can change it between replays.
        self.opt = torch.optim.Adam([self.param], lr=torch.tensor(float(lr), dtype=torch.float32, device=x.device),
                                    eps=eps, capturable=True, fused=True)
        self.graph = None
        self.static_loss = None

    @property
    def h(self):
        """The predistorter coefficients (complex view of the parameter)."""
        return torch.view_as_complex(self.param)

    def h_grad(self):
        """Gradient of the last loss with respect to h (complex, dL/dRe + j dL/dIm)."""
        return torch.view_as_complex(self.param.grad)

    def loss(self):
        y = self.tx(DPDFunction.apply(self.x, self.h, self.filt))
        return SqErrorLoss.apply(y, self.x, self.filt, self.gain, self.scale)

    def _step(self):
        self.opt.zero_grad(set_to_none=False)
        loss = self.loss()
        loss.backward()
        self.opt.step()
        return loss

    def capture(self, warmup=3):
        """Capture one training step in a CUDA graph (after a few eager steps)."""
        s = torch.cuda.Stream()
        s.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(s):
            for _ in range(warmup):
                self._step()
        torch.cuda.current_stream().wait_stream(s)
        self.graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(self.graph):
            self.static_loss = self._step()
        return self

    def step(self):
        if self.graph is not None:
            self.graph.replay()
            return self.static_loss
        return self._step()

    @property
    def lr(self):
        return float(self.opt.param_groups[0]["lr"])

    def set_lr(self, lr):
        """Set the learning rate in place (a captured step follows it)."""
        for g in self.opt.param_groups:
            g["lr"].fill_(float(lr))

    def train(self, steps, final_lr=None, decay_start=0.0):
        """Run `steps` training steps (graph replays once captured).  With
        final_lr the learning rate stays at its current value for the first
        decay_start fraction of the steps, then decays geometrically to
        final_lr at the last step.  Returns (step, loss) samples."""
        hist = []
        lr0 = self.lr
        i0 = int(decay_start * steps)
        for i in range(steps):
            if final_lr is not None and i >= i0 and steps - 1 > i0:
                self.set_lr(lr0 * (final_lr / lr0) ** ((i - i0) / (steps - 1 - i0)))
            loss = self.step()
            if i % max(1, steps // 20) == 0 or i == steps - 1:
                hist.append((i, float(loss.detach())))
        return hist

    def time_step(self, reps=50):
        """Milliseconds per graph-replayed training step."""
        if self.graph is None:
            self.capture()
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(reps):
            self.graph.replay()
        e1.record()
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / reps


def indirect_learning(x, tx, P, Q, M, gain=1.0, iterations=3, precision="tf32x3", refine_iters=2):
    """ILA (Sec. 2.2): returns the coefficient vector after `iterations` LS fits."""
    return ila_train(x, tx, P, Q, M, gain, iterations, precision, refine_iters)[0]


def ila_train(x, tx, P, Q, M, gain=1.0, iterations=3, precision="tf32x3", refine_iters=2, basis="monomial"):
    """The indirect-learning loop of Sec. 2.2 / Fig. 1(b), every step on the GPU.
    Iteration i: z = DPD^(i-1)(x) (x itself first), s = TX(z) / G, and the
    post-distorter fit h^(i) = argmin ||Psi(s) h - z|| (dpd_estimate), which
    becomes the predistorter.  Returns (h, history) with, per iteration, the
    NMSE of TX(DPD(x)) / G against x before the fit and the condition estimate
    and relative residual of the fit."""
    est = DPD(P, Q, M)
    est.set_estimate_basis(basis)
    h = None
    history = []
    for i in range(iterations):
        z = x if h is None else est.apply(x)
        s = tx.apply(z) / gain
        rec = {"iteration": i + 1, "nmse_db_before": nmse_db(s, x)}
        h, st = est.estimate(s.contiguous(), z.contiguous(), precision=precision, refine_iters=refine_iters)
        est.set_coeffs(h)
        rec.update(st)
        history.append(rec)
    history.append({"iteration": iterations + 1, "nmse_db_before": nmse_db(tx.apply(est.apply(x)) / gain, x)})
    est.close()
    return h, history


def warp_pa_transmitter(device="cuda"):
    """The memoryless 5th-order WARP PA of Eq. 3 as a one-stage transmitter
    (an APH filter with P = 5, Q = 0, M = 0 and coefficients alpha_1, alpha_3,
    alpha_5); its small-signal gain is alpha_1."""
    alpha = [0.9490 - 0.0197j, 0.4885 + 0.1071j, -1.0156 - 0.0474j]   # Eq. 3
    st = dict(P=5, Q=0, M=0, h=alpha + [0.0])
    return Transmitter([st], device=device), alpha[0]
