"""Spectral view of predistortion (the paper's Sec. 5.2 / Fig. 8 measurement,
made on samples instead of a spectrum analyzer): Welch power spectral density
and the out-of-band power of a PA output with and without predistortion.

Analysis on the host (numpy), outside the filter path.  Spectra are two-sided
baseband spectra in FFT bin order, normalised so that their mean over the bins
equals the mean power of the windowed samples (Parseval)."""
from __future__ import annotations

import numpy as np


def welch_psd(x, nfft: int = 4096, overlap: float = 0.5) -> np.ndarray:
    """Average of Hann-windowed periodograms of nfft-sample segments with the
    given overlap: |FFT(w s)|^2 / sum(w^2) per segment."""
    x = np.asarray(x).astype(np.complex128)
    if x.shape[0] < nfft:
        raise ValueError("need at least nfft samples")
    w = np.hanning(nfft + 1)[:nfft]   # periodic Hann
    step = max(1, int(round(nfft * (1.0 - overlap))))
    starts = range(0, x.shape[0] - nfft + 1, step)
    acc = np.zeros(nfft)
    for s0 in starts:
        acc += np.abs(np.fft.fft(w * x[s0:s0 + nfft])) ** 2
    return acc / (len(starts) * np.sum(w * w))


def _oob_mask(band: np.ndarray, guard: int) -> np.ndarray:
    """Bins farther than `guard` bins (circularly) from every in-band bin."""
    near = band.copy()
    for d in range(1, guard + 1):
        near |= np.roll(band, d) | np.roll(band, -d)
    return ~near


def band_levels(psd: np.ndarray, band: np.ndarray, guard: int = 16, smooth: int = 32) -> dict:
    """In-band power and out-of-band levels of a spectrum, in dB relative to
    the mean in-band PSD: total out-of-band power (dBc) and the peak of the
    out-of-band PSD after a `smooth`-bin moving average (dBc per bin)."""
    band = np.asarray(band, bool)
    oob = _oob_mask(band, guard)
    inband = psd[band].mean()
    # moving average over out-of-band bins only (in-band power never leaks in)
    kernel = np.ones(smooth)
    wrap = lambda v: np.concatenate([v[-smooth:], v, v[:smooth]])   # noqa: E731
    num = np.convolve(wrap(np.where(oob, psd, 0.0)), kernel, mode="same")[smooth:-smooth]
    cnt = np.convolve(wrap(oob.astype(float)), kernel, mode="same")[smooth:-smooth]
    sm = np.where(oob, num / np.maximum(cnt, 1.0), 0.0)
    return {"inband_psd": float(inband),
            "oob_total_dbc": float(10 * np.log10(psd[oob].sum() / psd[band].sum())),
            "oob_peak_dbc": float(10 * np.log10(sm[oob].max() / inband))}


def suppression_report(x, pa_out_plain, pa_out_dpd, band, nfft: int = 4096, guard: int = 16) -> dict:
    """Out-of-band levels of the PA output without and with predistortion and
    their difference (the suppression in dB, > 0 when predistortion helps);
    the input's own levels give the floor a perfect linearisation would reach."""
    lv = {k: band_levels(welch_psd(v, nfft), band, guard)
          for k, v in (("input", x), ("no_dpd", pa_out_plain), ("dpd", pa_out_dpd))}
    lv["suppression_total_db"] = lv["no_dpd"]["oob_total_dbc"] - lv["dpd"]["oob_total_dbc"]
    lv["suppression_peak_db"] = lv["no_dpd"]["oob_peak_dbc"] - lv["dpd"]["oob_peak_dbc"]
    return lv
