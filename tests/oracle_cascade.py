"""FP64 reference of the direct-learning loss and its coefficient gradient
through a chain of APH stages (predistorter, then fixed transmitter stages),
composed from the oracle's per-stage forward and gradient by the chain rule.
Test infrastructure."""
import numpy as np

import oracle


def cascade_forward(x, h, model, stages):
    P, Q, M = model
    vals = [np.asarray(x).astype(np.complex128)]
    vals.append(oracle.apply(vals[0], h, P, Q, M))
    for st in stages:
        vals.append(oracle.apply(vals[-1], st["h"], st["P"], st["Q"], st["M"]))
    return vals


def cascade_loss_grad(x, h, model, stages, gain=1.0):
    """L = ||TX(DPD_h(x)) - G x||^2 / ||x||^2 and dL/dh (dL/dRe + j dL/dIm)."""
    P, Q, M = model
    vals = cascade_forward(x, h, model, stages)
    x64 = vals[0]
    scale = 1.0 / np.sum(np.abs(x64) ** 2)
    e = vals[-1] - gain * x64
    loss = float(np.sum(np.abs(e) ** 2) * scale)
    g = 2.0 * scale * e
    for st, inp in zip(reversed(stages), reversed(vals[1:-1])):
        _, g = oracle.grad(inp, st["h"], g, st["P"], st["Q"], st["M"], want_h=False)
    gh, _ = oracle.grad(x64, h, g, P, Q, M, want_x=False)
    return loss, gh
