"""The spectral-report helpers against closed forms (host numpy, no GPU)."""
import numpy as np
import pytest

import dpd_synth as synth
from paper_1612_09001_gb300 import spectrum


def test_parseval_single_segment():
    rng = np.random.default_rng(90)
    x = rng.standard_normal(4096) + 1j * rng.standard_normal(4096)
    w = np.hanning(4097)[:4096]
    psd = spectrum.welch_psd(x, nfft=4096)
    assert abs(psd.mean() - np.sum(np.abs(w * x) ** 2) / np.sum(w * w)) < 1e-12 * psd.mean()


def test_tone_lands_in_its_bin():
    n, k = 1 << 15, 700
    x = 0.5 * np.exp(2j * np.pi * k * np.arange(n) / 4096)
    psd = spectrum.welch_psd(x, nfft=4096)
    assert int(np.argmax(psd)) == k
    # Hann: the whole tone power lies in bins k-1 .. k+1 (mean-power normalisation)
    assert abs(psd[k - 1:k + 2].sum() / 4096 - 0.25) < 1e-9
    far = np.ones(4096, bool)
    far[k - 2:k + 3] = False
    assert psd[far].max() < 1e-20 * psd[k]


def test_white_noise_is_flat():
    rng = np.random.default_rng(91)
    x = (rng.standard_normal(1 << 20) + 1j * rng.standard_normal(1 << 20)) / np.sqrt(2)
    psd = spectrum.welch_psd(x, nfft=1024)
    assert abs(psd.mean() - 1.0) < 0.01
    assert psd.std() / psd.mean() < 0.05   # about 511 averaged segments


def test_band_levels_of_a_known_leak():
    """Carrier plus a tone 50 dB below the in-band PSD, far out of band."""
    x, band = synth.lte_single(1 << 18, key=(92, 0))
    x = x.astype(np.complex128)
    lv0 = spectrum.band_levels(spectrum.welch_psd(x), band)
    inband = lv0["inband_psd"]
    amp = np.sqrt(inband * 1e-5)          # tone power = 1e-5 x in-band PSD (per-bin mean-power units)
    tone = amp * np.exp(2j * np.pi * 1500 * np.arange(x.shape[0]) / 4096)
    lv = spectrum.band_levels(spectrum.welch_psd(x + tone), band, smooth=1)
    # periodic Hann: the tone's FFT amplitudes are 1/4, 1/2, 1/4 of N A in three bins, and
    # sum(w^2) = 3N/8, so the peak bin holds (N A / 2)^2 / (3N/8) = (2/3) N A^2
    assert lv["oob_peak_dbc"] == pytest.approx(10 * np.log10(2.0 / 3.0 * 4096 * 1e-5), abs=0.05)
    assert lv["oob_total_dbc"] > lv0["oob_total_dbc"]


def test_suppression_report_signs():
    x, band = synth.lte_single(1 << 17, key=(93, 0))
    x = x.astype(np.complex128)
    distorted = x + 0.05 * np.abs(x) ** 2 * x
    rep = spectrum.suppression_report(x, distorted, x + 0.001 * np.abs(x) ** 2 * x, band)
    assert rep["suppression_total_db"] > 20 and rep["suppression_peak_db"] > 20
    assert rep["input"]["oob_total_dbc"] < rep["dpd"]["oob_total_dbc"] < rep["no_dpd"]["oob_total_dbc"]
