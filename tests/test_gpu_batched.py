"""GPU parity of the batched plan (many independent streams, one persistent
launch) against the FP64 oracle, stream by stream."""
import ctypes

import numpy as np
import pytest

import dpd_synth as synth
import oracle
from util import assert_parity

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_1612_09001_gb300 as dpd  # noqa: E402
from paper_1612_09001_gb300 import _lib  # noqa: E402


def _prepare(specs, device_coeffs=False):
    streams = []
    for sp in specs:
        x = torch.from_numpy(sp["x"]).cuda()
        y = torch.full_like(x, complex(7, -7))
        h = torch.from_numpy(sp["h"]).cuda() if device_coeffs else sp["h"]
        streams.append(dict(x=x, y=y, P=sp["P"], Q=sp["Q"], M=sp["M"], h=h))
    return streams


def _check(specs, streams):
    for i, (sp, st) in enumerate(zip(specs, streams)):
        ref = oracle.apply(sp["x"], sp["h"], sp["P"], sp["Q"], sp["M"])
        assert_parity(st["y"].cpu().numpy(), ref, what=f"stream {i} n={len(sp['x'])} P={sp['P']} M={sp['M']}")


def test_config2_sixty_four_streams_persistent_and_graph():
    specs = synth.batch_streams(64, seed=0)
    streams = _prepare(specs)
    plan = dpd.BatchedPlan(streams)
    plan.execute()
    plan.sync_status()
    _check(specs, streams)
    # the same launch replayed from a CUDA graph
    for st in streams:
        st["y"].fill_(0)
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    g = torch.cuda.CUDAGraph()
    with torch.cuda.stream(s):
        with torch.cuda.graph(g, stream=s):
            plan.execute(stream=s)
    g.replay()
    torch.cuda.synchronize()
    plan.sync_status()
    _check(specs, streams)
    plan.close()


def _edge_specs():
    rng = np.random.default_rng([40, 0])
    specs = []
    sizes = [0, 1, 2, 3, 7, 8, 9, 1023, 1024, 1025, 2047, 2048, 2049, 4097, 50001]
    models = [(P, Q, M) for P in (0, 1, 3, 5, 7, 9, 11) for Q in (0, 1, 5, 11) for M in (0, 2, 4, 7) if P + Q > 0]
    for i, (P, Q, M) in enumerate(models):
        n = sizes[i % len(sizes)] if i < 2 * len(sizes) else int(rng.integers(1, 30000))
        x = synth.clipped_gaussian(n, 0.5, key=(40, i, 0))
        h = synth.coeffs(P, Q, M, key=(40, i, 1), f_std=0.3, g_std=0.3)
        specs.append(dict(x=x, h=h, P=P, Q=Q, M=M))
    return specs


@pytest.mark.parametrize("launch", [None, (4, 8, 4, 0), (8, 4, 2, 1), (4, 1, 2, 0), (8, 16, 4, 0), (4, 16, 8, 0), (4, 2, 3, 2),
                                    (8, 8, 3, 0, 2), (8, 12, 3, 0, 4), (4, 16, 4, 0, 1), (8, 16, 2, 0, 8), (8, 8, 4, 0, 1),
                                    (6, 8, 3, 0, 0), (6, 16, 4, 0, 4), (6, 12, 3, 0, 2), (6, 16, 2, 0, 4)])
def test_every_model_and_edge_sizes(launch):
    """Every model against the oracle on empty, tiny and ragged streams, for
    launch shapes whose items carry 1, 2 or 4 sub-blocks per thread (the largest
    count whose ring fits in shared memory)."""
    specs = _edge_specs()
    streams = _prepare(specs)
    plan = dpd.BatchedPlan(streams)
    if launch:
        plan.set_launch(*launch)
    plan.execute()
    plan.sync_status()
    _check(specs, streams)
    plan.close()


def test_small_models_use_device_coefficients():
    specs = [dict(x=synth.ofdm2(20000 + 37 * i, key=(41, i)), P=P, Q=P, M=M,
                  h=synth.coeffs(P, P, M, key=(41, i, 1)))
             for i, (P, M) in enumerate([(5, 2), (7, 3), (9, 4), (5, 6), (9, 6), (7, 2)])]
    streams = _prepare(specs, device_coeffs=True)
    plan = dpd.BatchedPlan(streams)
    plan.execute()
    plan.sync_status()
    _check(specs, streams)
    plan.close()


def test_plan_argument_errors():
    lib = _lib.load()
    x = torch.zeros(1001, dtype=torch.complex64, device="cuda")
    y = torch.zeros(1001, dtype=torch.complex64, device="cuda")
    h = torch.from_numpy(synth.coeffs(5, 5, 2))

    def plan(descs):
        arr = (_lib.StreamDesc * len(descs))(*descs)
        p = ctypes.c_void_p()
        rc = lib.dpd_plan_batched(ctypes.cast(arr, ctypes.c_void_p), len(descs), 0, ctypes.byref(p))
        if rc == 0:
            lib.dpd_plan_destroy(p)
        return rc

    ok = _lib.StreamDesc(x.data_ptr(), y.data_ptr(), 1000, 5, 5, 2, h.data_ptr())
    assert plan([ok]) == 0
    assert plan([_lib.StreamDesc(x.data_ptr() + 8, y.data_ptr(), 1000, 5, 5, 2, h.data_ptr())]) == 1   # x not 16 B
    assert plan([_lib.StreamDesc(x.data_ptr(), x.data_ptr(), 1000, 5, 5, 2, h.data_ptr())]) == 1       # in place
    assert plan([ok, _lib.StreamDesc(y.data_ptr(), y.data_ptr() + 16, 10, 5, 5, 2, h.data_ptr())]) == 1  # y overlaps
    assert plan([_lib.StreamDesc(x.data_ptr(), y.data_ptr(), 1000, 4, 5, 2, h.data_ptr())]) == 2       # even order
    assert plan([_lib.StreamDesc(x.data_ptr(), y.data_ptr(), 1000, 5, 5, 8, h.data_ptr())]) == 2       # 9 taps
    assert plan([_lib.StreamDesc(x.data_ptr(), y.data_ptr(), 1000, 0, 0, 2, h.data_ptr())]) == 1       # no branch
    assert lib.dpd_exec_batched(None, None) == 1
    assert lib.dpd_plan_destroy(None) == 0
    with pytest.raises(ValueError):
        dpd.BatchedPlan([dict(x=x, y=y, P=5, Q=5, M=2, h=h),
                         dict(x=x[:0], y=y[:0], P=5, Q=5, M=2, h=h.cuda())])
