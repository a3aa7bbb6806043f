"""The autotuner picks shapes that are correct: after tuning, every kernel still
matches the FP64 oracle."""
import numpy as np
import pytest

import dpd_synth as synth
import oracle
from util import assert_parity

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_1612_09001_gb300 as dpd  # noqa: E402
from paper_1612_09001_gb300 import tune  # noqa: E402


def test_tuned_shapes_stay_correct(tmp_path, monkeypatch):
    monkeypatch.setattr(tune, "CACHE", str(tmp_path / "tune.json"))
    P, Q, M, n = 9, 9, 4, 1 << 20
    x = synth.ofdm2(n, key=(90, 0))
    h = synth.coeffs(P, Q, M, key=(90, 1))
    f = dpd.DPD(P, Q, M)
    f.set_coeffs(h)
    xd = torch.from_numpy(x).cuda()
    best, res = tune.tune_forward(f, xd)
    assert res and best == res[0][1]
    assert_parity(f.apply(xd).cpu().numpy(), oracle.apply(x, h, P, Q, M), what=f"tuned {best}")
    g = np.random.default_rng(91)
    gy = torch.from_numpy((g.standard_normal(n) + 1j * g.standard_normal(n)).astype(np.complex64)).cuda()
    best_a, _ = tune.tune_adjoint(f, xd, gy)
    gh = torch.empty(f.K, dtype=torch.complex64, device="cuda")
    f.grad(xd, gy, gh=gh)
    ref, _ = oracle.grad(x, h, gy.cpu().numpy(), P, Q, M, want_x=False)
    assert np.linalg.norm(gh.cpu().numpy() - ref) / np.linalg.norm(ref) < 1e-5
    f2 = dpd.DPD(P, Q, M)
    assert tune.apply_cached(f2) and f2.fwd_launch == best
    specs = synth.batch_streams(8, seed=3)
    streams = []
    for sp in specs:
        xs = torch.from_numpy(sp["x"]).cuda()
        streams.append(dict(x=xs, y=torch.empty_like(xs), P=sp["P"], Q=sp["Q"], M=sp["M"], h=sp["h"]))
    plan = dpd.BatchedPlan(streams)
    best_b, _ = tune.tune_batched(plan)
    plan.execute()
    plan.sync_status()
    for sp, st in zip(specs, streams):
        assert_parity(st["y"].cpu().numpy(), oracle.apply(sp["x"], sp["h"], sp["P"], sp["Q"], sp["M"]))
