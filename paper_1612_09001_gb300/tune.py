"""Autotuner for the library's launch shapes.

Each tuner times candidate shapes of one kernel on the caller's data with CUDA
events (after warm-up, median of several repetitions), installs the fastest
and returns the measurements.  Results are cached per GPU name and model in a
JSON file (default ``~/.cache/dpd_tune.json``, overridable with the
``DPD_TUNE_CACHE`` environment variable) so later handles can reuse them with
``apply_cached``.

* forward filter (``dpd_set_fwd_launch``): compute mode, samples per thread V,
  consumer warps (tile = warps * 32 * V samples), ring stages, CTAs per SM;
* batched plan (``dpd_plan_set_launch``): V, warps (the tile of every work
  item), stages, CTAs per SM;
* adjoint (``dpd_set_adj_launch``): CTAs per tap group and the tap-group size
  (how the taps of the coefficient gradient are split across the grid).
"""
from __future__ import annotations

import json
import os
import statistics

import torch

CACHE = os.environ.get("DPD_TUNE_CACHE", os.path.join(os.path.expanduser("~"), ".cache", "dpd_tune.json"))

# Forward shapes: one group of all warps (as many CTAs per SM as fit), and the
# grouped rings (warps per group dividing the warp count) at 12 and 16 warps.
FWD_CANDIDATES = ([dict(mode=m, V=V, warps=w, stages=s, ctas_per_sm=0, use_tma=1, group=0)
                   for m in (3, 2) for V in (8, 4) for w in (4, 8, 12) for s in (3, 4)] +
                  [dict(mode=m, V=V, warps=w, stages=s, ctas_per_sm=0, use_tma=1, group=g)
                   for m in (3, 2) for V in (8, 4) for (w, g) in ((12, 1), (12, 2), (12, 3), (12, 4), (12, 6),
                                                                 (16, 1), (16, 2), (16, 4), (16, 8))
                   for s in (3, 4)] +

                  [dict(mode=3, V=6, warps=w, stages=s, ctas_per_sm=0, use_tma=1, group=g)
                   for (w, g) in ((8, 0), (12, 0), (12, 2), (12, 3), (12, 4), (16, 2), (16, 4), (16, 8))
                   for s in (3, 4)])
BATCH_CANDIDATES = ([(V, w, s, 0, 0) for V in (8, 6, 4) for w in (4, 8, 12) for s in (2, 3, 4)] +
                    [(V, w, s, 0, g) for V in (8, 6, 4) for (w, g) in ((8, 1), (8, 2), (8, 4), (12, 2), (12, 3), (12, 4),
                                                                  (16, 2), (16, 4), (16, 8))
                     for s in (2, 3, 4)])


def _time(fn, reps=5, inner=5):
    for _ in range(2):
        fn()
    torch.cuda.synchronize()
    ts = []
    for _ in range(reps):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(inner):
            fn()
        e1.record()
        torch.cuda.synchronize()
        ts.append(e0.elapsed_time(e1) / inner)
    return statistics.median(ts)


def _key(kind, P, Q, M):
    return f"{torch.cuda.get_device_name()}|{kind}|P{P}Q{Q}M{M}"


def _load():
    try:
        with open(CACHE) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def _store(key, value):
    d = _load()
    d[key] = value
    try:
        os.makedirs(os.path.dirname(CACHE), exist_ok=True)
        with open(CACHE, "w") as f:
            json.dump(d, f, indent=1)
    except OSError:
        pass


def tune_forward(filt, x, y=None, candidates=None):
    """Time forward launch shapes of `filt` on x; install and return the best."""
    from . import DPDError
    y = torch.empty_like(x) if y is None else y
    results = []
    for cand in candidates or FWD_CANDIDATES:
        try:
            filt.set_fwd_launch(**cand)
            ms = _time(lambda: filt.apply(x, out=y))
        except DPDError:
            continue
        results.append((ms, cand))
    results.sort(key=lambda r: r[0])
    best = results[0][1]
    filt.set_fwd_launch(**best)
    _store(_key("fwd", filt.P, filt.Q, filt.M), best)
    return best, results


def tune_batched(plan, candidates=None):
    """Time tile / stage / grid shapes of a batched plan; install and return the best."""
    from . import DPDError
    results = []
    for cand in candidates or BATCH_CANDIDATES:
        try:
            plan.set_launch(*cand)
            ms = _time(lambda: plan.execute())
        except DPDError:
            continue
        results.append((ms, cand))
    results.sort(key=lambda r: r[0])
    best = results[0][1]
    plan.set_launch(*best)
    return best, results


def tune_adjoint(filt, x, gy, candidates=None):
    """Time the coefficient-gradient tap schedule (CTAs per tap group, taps per group)."""
    from . import DPDError
    sms = torch.cuda.get_device_properties(x.device).multi_processor_count
    gh = torch.empty(filt.K, dtype=torch.complex64, device=x.device)
    gx = torch.empty_like(x)
    results = []
    for cand in candidates or [(b * sms, tg) for b in (1, 2, 4) for tg in (1, 2, 3, 4, 5)]:
        try:
            filt.set_adj_launch(*cand)
            ms = _time(lambda: filt.grad(x, gy, gh=gh, gx=gx))
        except DPDError:
            continue
        results.append((ms, cand))
    results.sort(key=lambda r: r[0])
    best = results[0][1]
    filt.set_adj_launch(*best)
    _store(_key("adj", filt.P, filt.Q, filt.M), list(best))
    return best, results


def apply_cached(filt):
    """Install cached forward / adjoint shapes for this GPU and model, if any."""
    d = _load()
    fwd = d.get(_key("fwd", filt.P, filt.Q, filt.M))
    if fwd:
        filt.set_fwd_launch(**fwd)
    adj = d.get(_key("adj", filt.P, filt.Q, filt.M))
    if adj:
        filt.set_adj_launch(*adj)
    return bool(fwd or adj)
