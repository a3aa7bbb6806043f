"""Seeded synthetic inputs for the augmented-parallel-Hammerstein (APH) DPD filter.

This module is shared by the FP64 oracle's tests and the CUDA path's tests and
benchmarks.  It draws random numbers and shapes them into signals and coefficient
vectors; it performs none of the predistorter's arithmetic (no basis terms, no
filtering, no least squares).

The paper's own workloads (a 10 MHz LTE uplink carrier and a 2x3 MHz
non-contiguous carrier-aggregation signal measured on a WARP v3 radio, Sec. 5.2)
are not available, so these generators stand in for them:

* ``clipped_gaussian``: i.i.d. circular complex Gaussian samples, hard-clipped at
  |x| = 1 with the phase kept.
* ``ofdm2``: two LTE-like OFDM carriers (1024-point IFFT, 600 active QPSK
  subcarriers, 72-sample cyclic prefix) shifted to +-0.3 of Nyquist and summed.
* ``coeffs``: a coefficient vector in the order the paper stacks it (Sec. 2.2):
  ``[h_1, h_3, ..., h_P, hbar_1, ..., hbar_Q, c]``, each ``h_p`` holding the
  ``L = M + 1`` taps ``h_{p,0..M}``.

Every array is returned as ``complex64``; tests upcast the same values exactly
to ``complex128`` for the oracle.
"""
from __future__ import annotations

import math

import numpy as np

__all__ = [
    "num_coeffs",
    "clipped_gaussian",
    "ofdm2",
    "coeffs",
    "batch_streams",
    "synthetic_pa",
    "warp_pa_eq3",
    "ls_problem",
]


def num_coeffs(P: int, Q: int, M: int) -> int:
    """Length of the stacked coefficient vector: one FIR of M+1 taps per odd
    order in {1..P} and {1..Q}, plus the LO-leakage constant (Sec. 2.2)."""
    bp = (P + 1) // 2 if P > 0 else 0
    bq = (Q + 1) // 2 if Q > 0 else 0
    return (bp + bq) * (M + 1) + 1


def _rng(key) -> np.random.Generator:
    return np.random.default_rng(list(key))


def clipped_gaussian(n: int, rms: float = 0.3, key=(0, 0)) -> np.ndarray:
    """``n`` complex samples ``rms*(a+jb)/sqrt(2)``, a, b ~ N(0,1) i.i.d., with
    any sample of magnitude above 1 scaled back onto the unit circle."""
    g = _rng(key)
    z = (g.standard_normal(n) + 1j * g.standard_normal(n)) * (rms / math.sqrt(2.0))
    mag = np.abs(z)
    over = mag > 1.0
    z[over] = z[over] / mag[over]
    return z.astype(np.complex64)


def _ofdm_carrier(g: np.random.Generator, nsym: int, nfft=1024, nact=600, ncp=72):
    half = nact // 2
    bins = np.concatenate([np.arange(1, half + 1), np.arange(nfft - half, nfft)])
    qpsk = ((2 * g.integers(0, 2, (nsym, nact)) - 1)
            + 1j * (2 * g.integers(0, 2, (nsym, nact)) - 1)) / math.sqrt(2.0)
    spec = np.zeros((nsym, nfft), dtype=np.complex128)
    spec[:, bins] = qpsk
    sym = np.fft.ifft(spec, axis=1)
    return np.concatenate([sym[:, nfft - ncp:], sym], axis=1).reshape(-1)


def ofdm2(n: int, key=(0, 0), rms: float = 0.25, shift: float = 0.3) -> np.ndarray:
    """Two OFDM carriers, each 1024-point IFFT with 600 active QPSK subcarriers
    (DC null) and a 72-sample cyclic prefix, mixed to +shift and -shift of
    Nyquist, summed and scaled to the given RMS.  No clipping."""
    g = _rng(key)
    sym_len = 1024 + 72
    nsym = max(1, -(-n // sym_len))
    a = _ofdm_carrier(g, nsym)[:n]
    b = _ofdm_carrier(g, nsym)[:n]
    t = np.arange(n, dtype=np.float64)
    z = a * np.exp(1j * math.pi * shift * t) + b * np.exp(-1j * math.pi * shift * t)
    z *= rms / math.sqrt(np.mean(np.abs(z) ** 2))
    return z.astype(np.complex64)


# LTE-like uplink test signals for the spectral-suppression experiment (the
# paper's 10 MHz carrier and two non-contiguous 3 MHz carriers 10 MHz apart).
# The spectrum is built for the whole sequence at once (QPSK on the occupied
# subcarriers of one long FFT, 15 kHz spacing at a 61.44 MHz sample rate, i.e.
# four times oversampled) so the input itself has no out-of-band power and the
# PA's spectral regrowth stays inside the band.  Each generator returns the
# samples (complex64, scaled to the RMS) and the in-band bins of a 4096-point
# spectrum.
LTE_NFFT = 4096


def _banded(g: np.random.Generator, n: int, centres, half: int, rms: float):
    N = -(-n // LTE_NFFT) * LTE_NFFT
    scale = N // LTE_NFFT
    spec = np.zeros(N, dtype=np.complex128)
    band = np.zeros(LTE_NFFT, bool)
    for c in centres:
        k = c * scale + np.arange(-half * scale, half * scale + 1)
        spec[k % N] = ((2 * g.integers(0, 2, k.size) - 1) + 1j * (2 * g.integers(0, 2, k.size) - 1)) / math.sqrt(2.0)
        band[(c + np.arange(-half, half + 1)) % LTE_NFFT] = True
    z = np.fft.ifft(spec)[:n]
    z *= rms / math.sqrt(np.mean(np.abs(z) ** 2))
    return z.astype(np.complex64), band


def lte_single(n: int, key=(0, 0), rms: float = 0.2):
    """One 10 MHz carrier: 600 subcarriers around DC."""
    return _banded(_rng(key), n, (0,), 300, rms)


def lte_two(n: int, key=(0, 0), rms: float = 0.2):
    """Two 3 MHz carriers (180 subcarriers each) centred 10 MHz apart
    (+-5 MHz = +-333 subcarriers)."""
    return _banded(_rng(key), n, (333, -333), 90, rms)


def coeffs(P: int, Q: int, M: int, key=(0, 1), f_std=1e-2, g_std=1e-3,
           c=1e-3 * (1 + 1j)) -> np.ndarray:
    """Coefficient vector in the paper's stacking order.

    ``h_{1,0} = 1`` exactly; every other main-branch tap of order p is complex
    Gaussian with standard deviation ``f_std/p`` (real and imaginary parts each
    with variance sigma^2/2), conjugate-branch taps use ``g_std/q``.  Draw order:
    main taps by increasing order then tap, then conjugate taps likewise."""
    T = M + 1
    orders_p = list(range(1, P + 1, 2)) if P > 0 else []
    orders_q = list(range(1, Q + 1, 2)) if Q > 0 else []
    g = _rng(key)
    K = num_coeffs(P, Q, M)
    h = np.zeros(K, dtype=np.complex128)
    i = 0
    for p in orders_p:
        for _ in range(T):
            s = f_std / p
            h[i] = (g.standard_normal() + 1j * g.standard_normal()) * s / math.sqrt(2.0)
            i += 1
    for q in orders_q:
        for _ in range(T):
            s = g_std / q
            h[i] = (g.standard_normal() + 1j * g.standard_normal()) * s / math.sqrt(2.0)
            i += 1
    if orders_p:
        h[0] = 1.0
    h[K - 1] = c
    return h.astype(np.complex64)


def batch_streams(count: int = 64, seed: int = 0, nmin=1 << 12, nmax=1 << 20,
                  orders=(5, 7, 9), mmin=2, mmax=6):
    """Independent antenna streams of uneven length and model order.

    Stream s draws its length, order P (= Q) and memory M from
    ``default_rng([seed, 2, s])``; its samples from ``[seed, 2, s, 0]`` (clipped
    Gaussian, RMS 0.3) and its coefficients from ``[seed, 2, s, 1]``.
    Returns a list of dicts with keys n, P, Q, M, x, h."""
    out = []
    for s in range(count):
        g = _rng((seed, 2, s))
        n = int(g.integers(nmin, nmax + 1))
        P = int(g.choice(np.asarray(orders)))
        M = int(g.integers(mmin, mmax + 1))
        x = clipped_gaussian(n, 0.3, key=(seed, 2, s, 0))
        h = coeffs(P, P, M, key=(seed, 2, s, 1))
        out.append(dict(n=n, P=P, Q=P, M=M, x=x, h=h))
    return out


def synthetic_pa(seed: int = 1, gain_imb=1.02, phase_deg=2.0, lo=0.005):
    """Transmitter model for direct-learning experiments: an I/Q modulator
    followed by a power amplifier with memory.  Both stages are expressed in
    the APH filter's own parameterisation:

    * I/Q stage (P=1, Q=1, M=0): ``u = K1 v + K2 conj(v) + c_LO`` with
      ``K1 = (1 + g e^{-j phi})/2`` and ``K2 = (1 - g e^{j phi})/2``.
    * PA stage (P=7, Q=0, M=3): main branch only, ``a_{1,0} = 1``,
      ``a_{3,0} = -0.1``, ``a_{5,0} = 0.02``, every other tap complex Gaussian
      with standard deviation ``1e-2/p`` from ``default_rng([seed, 1])``.
    """
    phi = math.radians(phase_deg)
    k1 = (1 + gain_imb * complex(math.cos(-phi), math.sin(-phi))) / 2
    k2 = (1 - gain_imb * complex(math.cos(phi), math.sin(phi))) / 2
    iq = np.array([k1, k2, lo], dtype=np.complex64)
    P, M = 7, 3
    T = M + 1
    g = _rng((seed, 1))
    pa = np.zeros(num_coeffs(P, 0, M), dtype=np.complex128)
    for b, p in enumerate(range(1, P + 1, 2)):
        for k in range(T):
            s = 1e-2 / p
            pa[b * T + k] = (g.standard_normal() + 1j * g.standard_normal()) * s / math.sqrt(2.0)
    pa[0 * T + 0] = 1.0
    pa[1 * T + 0] = -0.1
    pa[2 * T + 0] = 0.02
    return dict(iq=dict(P=1, Q=1, M=0, h=iq), pa=dict(P=P, Q=0, M=M, h=pa.astype(np.complex64)))


def warp_pa_eq3():
    """The memoryless 5th-order WARP v3 PA model of Eq. 3, written as an APH
    filter with P=5, Q=0, M=0: coefficients ``[alpha_1, alpha_3, alpha_5, 0]``."""
    a1 = 0.9490 - 0.0197j
    a3 = 0.4885 + 0.1071j
    a5 = -1.0156 - 0.0474j
    return dict(P=5, Q=0, M=0, h=np.array([a1, a3, a5, 0.0], dtype=np.complex128))


def ls_problem(n: int, P=11, Q=11, M=7, seed=0):
    """Least-squares estimation input: clipped-Gaussian basis input ``u``
    (RMS 0.3, ``default_rng([seed, 0])``) and true coefficients drawn like
    ``coeffs`` from ``[seed, 1]``.  The target ``t = Phi(u) theta_true`` is
    formed by the caller with the filter under test or with the oracle."""
    u = clipped_gaussian(n, 0.3, key=(seed, 0))
    theta = coeffs(P, Q, M, key=(seed, 1))
    return u, theta
