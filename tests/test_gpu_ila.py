"""Indirect learning on the GPU (Sec. 2.2, Fig. 1(b)) around the WARP PA model
of Eq. 3, and the out-of-band suppression it buys on LTE-like signals (the
paper's Fig. 8 experiment, measured on samples)."""
import numpy as np
import pytest

import dpd_synth as synth
import oracle

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_1612_09001_gb300 as dpd  # noqa: E402
from paper_1612_09001_gb300 import direct, spectrum  # noqa: E402


@pytest.mark.parametrize("signal", ["single", "two"])
@pytest.mark.parametrize("P,Q,M", [(7, 0, 0), (9, 3, 1)])
def test_ila_suppresses_spectral_regrowth(signal, P, Q, M):
    gen = synth.lte_single if signal == "single" else synth.lte_two
    x, band = gen(1 << 18, key=(80, P), rms=0.2)
    xd = torch.from_numpy(x).cuda()
    tx, G = direct.warp_pa_transmitter()
    y_plain = (tx.apply(xd) / G).cpu().numpy()
    h, hist = direct.ila_train(xd, tx, P, Q, M, gain=G, iterations=3, precision="tf32x3", basis="orthogonal")
    f = dpd.DPD(P, Q, M)
    f.set_coeffs(h)
    y_dpd = (tx.apply(f.apply(xd)) / G).cpu().numpy()
    f.close()
    rep = spectrum.suppression_report(x, y_plain, y_dpd, band)
    # the paper reports > 10 dB on its hardware; the noise-free memoryless model allows far more
    assert rep["suppression_total_db"] > 25 and rep["suppression_peak_db"] > 25, rep
    nm = [r["nmse_db_before"] for r in hist]
    assert nm[0] > -35 and nm[-1] < -65 and nm[1] < nm[0] - 30, nm


def test_ila_step_matches_oracle_least_squares():
    """One ILA fit: the post-distorter estimated on the GPU from s = PA(x) / G
    equals the FP64 oracle's least-squares solution on the same samples."""
    P, Q, M = 7, 3, 1
    x, _ = synth.lte_two(1 << 16, key=(81, 0), rms=0.2)
    xd = torch.from_numpy(x).cuda()
    tx, G = direct.warp_pa_transmitter()
    s = (tx.apply(xd) / G).contiguous()
    f = dpd.DPD(P, Q, M)
    for basis, tol in (("orthogonal", 1e-5), ("monomial", 1e-4)):
        h, _ = f.estimate(s, xd, precision="tf32x3", refine_iters=3, basis=basis)
        ref = oracle.ls(s.cpu().numpy(), x, P, Q, M)
        err = np.linalg.norm(h.cpu().numpy() - ref) / np.linalg.norm(ref)
        assert err < tol, (basis, err)
    f.close()
