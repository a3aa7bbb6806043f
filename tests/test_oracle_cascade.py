"""The chain-rule gradient of the direct-learning loss through the FP64 oracle
stages equals central finite differences of the loss."""
import numpy as np

import dpd_synth as synth
from oracle_cascade import cascade_loss_grad


def test_cascade_gradient_matches_finite_differences():
    tx = synth.synthetic_pa(seed=1)
    stages = [tx["iq"], tx["pa"]]
    P, Q, M = 5, 5, 2
    x = synth.ofdm2(600, key=(80, 0)).astype(np.complex128)
    h = synth.coeffs(P, Q, M, key=(80, 1), f_std=0.2, g_std=0.1).astype(np.complex128)
    loss, gh = cascade_loss_grad(x, h, (P, Q, M), stages)
    eps = 1e-6
    for j in range(len(h)):
        for unit in (1.0, 1j):
            hp, hm = h.copy(), h.copy()
            hp[j] += eps * unit
            hm[j] -= eps * unit
            fd = (cascade_loss_grad(x, hp, (P, Q, M), stages)[0] - cascade_loss_grad(x, hm, (P, Q, M), stages)[0]) / (2 * eps)
            an = gh[j].real if unit == 1.0 else gh[j].imag
            assert abs(fd - an) <= 1e-6 * max(1.0, abs(an)), (j, unit, fd, an)
