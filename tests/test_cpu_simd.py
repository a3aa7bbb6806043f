"""The portable SIMD + OpenMP CPU filter (include/dpd_cpu.h) against the FP64
oracle: element-wise parity at the GPU's tolerance, ragged blocks and thread
counts, identity coefficients, and argument checks.  Runs on the host, no GPU."""
import numpy as np
import pytest

import dpd_synth as synth
import oracle
from util import assert_parity

from paper_1612_09001_gb300 import build, cpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    build.build_cpu()


@pytest.mark.parametrize("P,Q,M", [(9, 9, 4), (5, 3, 4), (11, 11, 7), (1, 0, 0), (7, 0, 3), (3, 11, 2)])
@pytest.mark.parametrize("n", [1, 7, 8, 9, 4095, 4096, 4097, 70001])
def test_parity(P, Q, M, n):
    x = synth.ofdm2(n, key=(95, P, n % 13))
    h = synth.coeffs(P, Q, M, key=(95, M))
    assert_parity(cpu.apply(x, h, P, Q, M), oracle.apply(x, h, P, Q, M), what=f"cpu P={P} Q={Q} M={M} n={n}")


@pytest.mark.parametrize("threads", [1, 2, 3, 0])
def test_thread_counts_agree_bitwise(threads):
    x = synth.clipped_gaussian(50001, 0.3, key=(96, 0))
    h = synth.coeffs(9, 9, 4, key=(96, 1))
    y1 = cpu.apply(x, h, 9, 9, 4, threads=1)
    assert np.array_equal(cpu.apply(x, h, 9, 9, 4, threads=threads), y1)


def test_identity_is_exact():
    x = synth.ofdm2(10007, key=(97, 0))
    h = np.zeros(synth.num_coeffs(5, 5, 2), np.complex64)
    h[0] = 1.0
    assert np.array_equal(cpu.apply(x, h, 5, 5, 2), x)


def test_empty_and_invalid():
    h = synth.coeffs(5, 5, 2)
    assert cpu.apply(np.zeros(0, np.complex64), h, 5, 5, 2).shape == (0,)
    x = np.ones(16, np.complex64)
    for P, Q, M in ((4, 3, 2), (5, 2, 2), (5, 5, 8), (13, 5, 2)):
        with pytest.raises(ValueError):
            cpu.apply(x, h, P, Q, M)
