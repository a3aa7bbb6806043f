"""Pins for the FP64 oracle: each check ties it to something other than itself.

* closed forms and special cases (identity, linear-only == numpy convolution,
  hand-evaluated Eq. 3 PA values from the printed coefficients),
* a second formulation (the basis matrix of Eq. 2 built with numpy),
* brute force with Python complex scalars on tiny inputs,
* invariants (linearity in the coefficients, shift equivariance),
* calculus (central finite differences for the gradient),
* a library least-squares solver and recovery of known coefficients.

``test_planted_mistakes_are_caught`` compiles copies of the oracle with one
plausible mistake each and checks that at least one pin fails for every copy.
"""
import math
import os
import shutil
import subprocess
import tempfile

import numpy as np
import pytest

import dpd_synth as synth
import oracle
from oracle import basis

HERE = os.path.dirname(os.path.abspath(__file__))


def _orders(top):
    return list(range(1, top + 1, 2)) if top > 0 else []


def brute_force(x, h, P, Q, M):
    """Eq. 1 with Python complex scalars and |x| from abs() (a square root)."""
    L = M + 1
    bp = len(_orders(P))
    out = []
    for n in range(len(x)):
        z = 0j
        for b, p in enumerate(_orders(P)):
            for k in range(L):
                if n - k >= 0:
                    v = complex(x[n - k])
                    z += complex(h[b * L + k]) * abs(v) ** (p - 1) * v
        for b, q in enumerate(_orders(Q)):
            for k in range(L):
                if n - k >= 0:
                    v = complex(x[n - k])
                    z += complex(h[(bp + b) * L + k]) * abs(v) ** (q - 1) * v.conjugate()
        out.append(z + complex(h[-1]))
    return np.array(out)


MODELS = [(1, 1, 0), (1, 0, 3), (3, 1, 2), (5, 3, 4), (5, 5, 2), (7, 0, 3), (9, 9, 4), (11, 11, 7), (3, 7, 1)]


# ----------------------------------------------------------------- pin bodies
# Each takes the oracle library handle so the planted-mistake test can rerun them.

def pin_identity(lib):
    x = synth.clipped_gaussian(777, key=(3, 0))
    h = np.zeros(synth.num_coeffs(5, 5, 3), np.complex128)
    h[0] = 1.0
    y = oracle.apply(x, h, 5, 5, 3, lib=lib)
    assert np.array_equal(y, x.astype(np.complex128))


def pin_linear_only_is_convolution(lib):
    x = synth.ofdm2(1500, key=(4, 0))
    M = 5
    h = synth.coeffs(1, 1, M, key=(4, 1), g_std=0.3)
    f, g, c = h[: M + 1], h[M + 1: 2 * M + 2], h[-1]
    x64 = x.astype(np.complex128)
    ref = (np.convolve(x64, f.astype(np.complex128))[: len(x)]
           + np.convolve(np.conj(x64), g.astype(np.complex128))[: len(x)] + complex(c))
    y = oracle.apply(x, h, 1, 1, M, lib=lib)
    np.testing.assert_allclose(y, ref, rtol=0, atol=1e-14)


def pin_eq1_equals_eq2(lib):
    for P, Q, M in MODELS:
        x = synth.clipped_gaussian(301, rms=0.5, key=(P, Q, M))
        h = synth.coeffs(P, Q, M, key=(P, Q, M, 1), f_std=0.5, g_std=0.5)
        y = oracle.apply(x, h, P, Q, M, lib=lib)
        ref = basis.apply(x, h, P, Q, M)
        err = np.linalg.norm(y - ref) / np.linalg.norm(ref)
        assert err < 1e-14, (P, Q, M, err)


def pin_brute_force(lib):
    for P, Q, M in [(5, 3, 4), (3, 3, 2), (1, 5, 1), (7, 0, 3)]:
        x = synth.clipped_gaussian(13, rms=0.7, key=(9, P, Q, M))
        h = synth.coeffs(P, Q, M, key=(9, P, Q, M, 1), f_std=0.5, g_std=0.5)
        y = oracle.apply(x, h, P, Q, M, lib=lib)
        np.testing.assert_allclose(y, brute_force(x, h, P, Q, M), rtol=1e-13, atol=1e-15)


def pin_golden_warp_pa(lib):
    rows = np.loadtxt(os.path.join(HERE, "golden", "warp_pa_eq3.txt"))
    x = rows[:, 0] + 1j * rows[:, 1]
    want = rows[:, 2] + 1j * rows[:, 3]
    pa = synth.warp_pa_eq3()
    y = oracle.apply(x, pa["h"], pa["P"], pa["Q"], pa["M"], lib=lib)
    np.testing.assert_allclose(y, want, rtol=0, atol=1e-12)


def pin_linearity(lib):
    P, Q, M = 7, 5, 3
    x = synth.clipped_gaussian(400, key=(5, 0))
    h1 = synth.coeffs(P, Q, M, key=(5, 1)).astype(np.complex128)
    h2 = synth.coeffs(P, Q, M, key=(5, 2), f_std=0.3, g_std=0.2).astype(np.complex128)
    a, b = 0.7 - 0.2j, -1.3 + 0.4j
    lhs = oracle.apply(x, a * h1 + b * h2, P, Q, M, lib=lib)
    rhs = a * oracle.apply(x, h1, P, Q, M, lib=lib) + b * oracle.apply(x, h2, P, Q, M, lib=lib)
    np.testing.assert_allclose(lhs, rhs, rtol=0, atol=1e-13)


def pin_shift(lib):
    P, Q, M, d = 5, 3, 4, 9
    x = synth.clipped_gaussian(250, key=(6, 0))
    h = synth.coeffs(P, Q, M, key=(6, 1))
    y = oracle.apply(x, h, P, Q, M, lib=lib)
    xs = np.concatenate([np.zeros(d, np.complex64), x])
    ys = oracle.apply(xs, h, P, Q, M, lib=lib)
    np.testing.assert_allclose(ys[:d], np.full(d, complex(h[-1])), rtol=0, atol=0)
    np.testing.assert_allclose(ys[d:], y, rtol=0, atol=1e-15)


def _loss(x, h, w, P, Q, M, lib):
    y = oracle.apply(x, h, P, Q, M, lib=lib)
    return float(np.sum(w.real * y.real + w.imag * y.imag))


def pin_grad_finite_differences(lib):
    for P, Q, M in [(5, 3, 2), (7, 7, 3), (3, 0, 1)]:
        n = 48
        x = synth.clipped_gaussian(n, rms=0.6, key=(7, P, 0)).astype(np.complex128)
        h = synth.coeffs(P, Q, M, key=(7, P, 1), f_std=0.4, g_std=0.3).astype(np.complex128)
        g = np.random.default_rng([7, P, 2])
        w = g.standard_normal(n) + 1j * g.standard_normal(n)
        gh, gx = oracle.grad(x, h, w, P, Q, M, lib=lib)
        eps = 1e-6
        for j in range(len(h)):
            for unit in (1.0, 1j):
                hp, hm = h.copy(), h.copy()
                hp[j] += eps * unit
                hm[j] -= eps * unit
                fd = (_loss(x, hp, w, P, Q, M, lib) - _loss(x, hm, w, P, Q, M, lib)) / (2 * eps)
                an = gh[j].real if unit == 1.0 else gh[j].imag
                assert abs(fd - an) <= 1e-6 * max(1.0, abs(an)), ("h", P, j, unit, fd, an)
        for i in range(0, n, 5):
            for unit in (1.0, 1j):
                xp, xm = x.copy(), x.copy()
                xp[i] += eps * unit
                xm[i] -= eps * unit
                fd = (_loss(xp, h, w, P, Q, M, lib) - _loss(xm, h, w, P, Q, M, lib)) / (2 * eps)
                an = gx[i].real if unit == 1.0 else gx[i].imag
                assert abs(fd - an) <= 1e-6 * max(1.0, abs(an)), ("x", P, i, unit, fd, an)


def pin_grad_h_is_psi_h_gy(lib):
    P, Q, M = 9, 9, 4
    x = synth.clipped_gaussian(500, key=(8, 0))
    h = synth.coeffs(P, Q, M, key=(8, 1))
    g = np.random.default_rng([8, 2])
    gy = g.standard_normal(500) + 1j * g.standard_normal(500)
    gh, _ = oracle.grad(x, h, gy, P, Q, M, want_x=False, lib=lib)
    ref = basis.basis_matrix(x, P, Q, M).conj().T @ gy
    np.testing.assert_allclose(gh, ref, rtol=1e-13, atol=1e-13)


def pin_gram_is_psi_h_psi(lib):
    for P, Q, M in [(5, 3, 4), (11, 11, 7), (3, 0, 2)]:
        u = synth.clipped_gaussian(700, key=(10, P))
        t = synth.ofdm2(700, key=(10, P, 1))
        G, b = oracle.gram(u, t, P, Q, M, lib=lib)
        Psi = basis.basis_matrix(u, P, Q, M)
        scale = np.abs(Psi.conj().T @ Psi).max()
        np.testing.assert_allclose(G, Psi.conj().T @ Psi, rtol=0, atol=1e-13 * scale)
        np.testing.assert_allclose(b, Psi.conj().T @ t.astype(np.complex128), rtol=0, atol=1e-12)


def pin_ls_recovers_coefficients(lib):
    P, Q, M = 5, 3, 4
    u, theta = synth.ls_problem(4000, P, Q, M, seed=3)
    t = basis.apply(u, theta, P, Q, M)       # noise-free target from the model itself
    h = oracle.ls(u, t, P, Q, M, lib=lib)
    np.testing.assert_allclose(h, theta.astype(np.complex128), rtol=0, atol=1e-8)
    np.testing.assert_allclose(h, basis.lstsq(u, t, P, Q, M), rtol=0, atol=1e-8)


def pin_chol_solve(lib):
    g = np.random.default_rng(11)
    K = 23
    A = g.standard_normal((60, K)) + 1j * g.standard_normal((60, K))
    G = A.conj().T @ A
    b = g.standard_normal(K) + 1j * g.standard_normal(K)
    h = oracle.chol_solve(G, b, lib=lib)
    np.testing.assert_allclose(h, np.linalg.solve(G, b), rtol=1e-10, atol=1e-12)


PINS = [pin_identity, pin_linear_only_is_convolution, pin_eq1_equals_eq2, pin_brute_force,
        pin_golden_warp_pa, pin_linearity, pin_shift, pin_grad_finite_differences,
        pin_grad_h_is_psi_h_gy, pin_gram_is_psi_h_psi, pin_ls_recovers_coefficients, pin_chol_solve]


@pytest.mark.parametrize("pin", PINS, ids=[p.__name__ for p in PINS])
def test_pin(pin, oracle_lib):
    pin(oracle_lib)


def test_table2_coefficient_count(oracle_lib):
    rows = np.loadtxt(os.path.join(HERE, "golden", "table2_config.txt"), ndmin=2)
    for P, Q, M, fm, fc, K in rows.astype(int):
        assert len(_orders(P)) == fm and len(_orders(Q)) == fc
        assert oracle.num_coeffs(P, Q, M) == K == synth.num_coeffs(P, Q, M)


def test_chol_rejects_indefinite(oracle_lib):
    G = np.diag([1.0, -1.0, 2.0]).astype(np.complex128)
    with pytest.raises(np.linalg.LinAlgError):
        oracle.chol_solve(G, np.ones(3), lib=oracle_lib)


def test_zero_history_and_empty(oracle_lib):
    h = synth.coeffs(3, 3, 2)
    assert oracle.apply(np.zeros(0, np.complex64), h, 3, 3, 2).shape == (0,)
    y = oracle.apply(np.array([0.5 + 0.25j], np.complex64), h, 3, 3, 2)
    assert y.shape == (1,)
    np.testing.assert_allclose(y, brute_force(np.array([0.5 + 0.25j]), h, 3, 3, 2), rtol=1e-14)


def test_ila_with_eq3_pa_reduces_error(oracle_lib):
    """Indirect learning (Sec. 2.2, 1-3 iterations) around the Eq. 3 PA.

    The paper prints no NMSE, so this is an improvement check only: after the
    first iteration the normalised error of PA(DPD(x))/G against x must be at
    least 10 dB below that of PA(x)/G, and later iterations must not undo it."""
    pa = synth.warp_pa_eq3()
    G = pa["h"][0]
    x = synth.clipped_gaussian(20000, rms=0.15, key=(12, 0)).astype(np.complex128)
    P, Q, M = 7, 1, 0

    def run_pa(v):
        return oracle.apply(v, pa["h"], pa["P"], pa["Q"], pa["M"])

    def nmse_db(v):
        e = run_pa(v) / G - x
        return 10 * math.log10(np.sum(np.abs(e) ** 2) / np.sum(np.abs(x) ** 2))

    base = nmse_db(x)
    h = None
    hist = []
    for _ in range(3):
        z = x if h is None else oracle.apply(x, h, P, Q, M)
        s = run_pa(z) / G
        h = oracle.ls(s, z, P, Q, M)
        hist.append(nmse_db(oracle.apply(x, h, P, Q, M)))
    assert hist[0] < base - 10.0, (base, hist)
    assert max(hist[1:]) < hist[0] + 1.0, (base, hist)


# ------------------------------------------------------- planted mistakes
MUTANTS = {
    "conjugate_branch_uses_x": ("return mag_pow(x, q) * conj(x);", "return mag_pow(x, q) * x;"),
    "tap_index_off_by_one": ("f += h[b * L + k] * psi(sample(x, n, i - k), p);",
                             "f += h[b * L + k] * psi(sample(x, n, i - k - 1), p);"),
    "lo_leakage_dropped": ("y[i] = z + c;", "y[i] = z;"),
    "order_power_wrong": ("for (int o = 1; o < p; o += 2) w *= r;", "for (int o = 1; o <= p; o += 2) w *= r;"),
    "circular_history": ("return (j >= 0 && j < n) ? x[j] : 0.0;", "return x[(j + n) % n];"),
    "conj_taps_reversed": ("f += h[(Bp + b) * L + k] * psibar", "f += h[(Bp + b) * L + (L - 1 - k)] * psibar"),
    "grad_missing_conj": ("g += conj(dx) * gy[i + k]", "g += dx * gy[i + k]"),
    "grad_h_no_conj": ("acc[j] += conj(row[j]) * gy[i];", "acc[j] += row[j] * gy[i];"),
    "gram_transposed": ("accG[(size_t)a * K + c2] += ca * row[c2];", "accG[(size_t)c2 * K + a] += ca * row[c2];"),
    "chol_missing_conj": ("s -= Lm[(size_t)i * K + k] * conj(Lm[(size_t)j * K + k]);",
                          "s -= Lm[(size_t)i * K + k] * Lm[(size_t)j * K + k];"),
    "grad_derivative_factor": ("dx += hk * (m + 1) * rm;", "dx += hk * m * rm;"),
}


@pytest.mark.skipif(shutil.which(os.environ.get("CC", "gcc")) is None, reason="no C compiler")
def test_planted_mistakes_are_caught():
    src = open(os.path.join(os.path.dirname(oracle.__file__), "dpd_oracle.c")).read()
    tmp = tempfile.mkdtemp(prefix="oracle_mutants_")
    try:
        for name, (old, new) in MUTANTS.items():
            assert src.count(old) == 1, name
            path = os.path.join(tmp, name + ".c")
            with open(path, "w") as f:
                f.write(src.replace(old, new))
            so = oracle.build.build(src=path, out=os.path.join(tmp, name + ".so"))
            lib = oracle.load(so)
            caught = []
            for pin in PINS:
                try:
                    pin(lib)
                except (AssertionError, RuntimeError, np.linalg.LinAlgError, ValueError):
                    caught.append(pin.__name__)
            assert caught, f"planted mistake '{name}' passed every pin"
    finally:
        shutil.rmtree(tmp, ignore_errors=True)
