"""Pins of the oracle's orthogonal-polynomial basis (the u_{m,p} of Sec. 2.1):
orthonormality by construction, closed forms for one order and for a known
magnitude distribution, and equivalence of the least-squares estimate with the
monomial one (the basis change is an invertible reparametrisation)."""
import inspect
import textwrap

import numpy as np
import pytest

import dpd_synth as synth
from oracle import basis


def _tap0_columns(P, Q, M, conj=False):
    L = M + 1
    Bp, Bq = (P + 1) // 2, (Q + 1) // 2
    if conj:
        return [Bp * L + b * L for b in range(Bq)]
    return [b * L for b in range(Bp)]


def pin_orthonormal_tap0(mod=basis):
    P, Q, M = 11, 7, 3
    u = synth.clipped_gaussian(20000, 0.3, key=(70, 0))
    U = mod.orthonormal_coefficients(u, 6)
    Po = mod.basis_matrix(u, P, Q, M) @ mod.transform_matrix(U, P, Q, M)
    for conj in (False, True):
        idx = _tap0_columns(P, Q, M, conj)
        G = Po[:, idx].conj().T @ Po[:, idx] / len(u)
        assert np.abs(G - np.eye(len(idx))).max() < 1e-10, conj
    assert np.allclose(np.tril(U, -1), 0.0)   # psi_p mixes only orders up to p


def pin_single_order_closed_form(mod=basis):
    u = synth.clipped_gaussian(4096, 0.5, key=(70, 1))
    U = mod.orthonormal_coefficients(u, 1)
    ref = 1.0 / np.sqrt(np.mean(np.abs(u.astype(np.complex128)) ** 2))
    assert abs(U[0, 0] - ref) < 1e-12 * ref


def pin_uniform_power_closed_form(mod=basis):
    # |x|^2 uniform on (0, 1): E r^k = 1 / (k + 1), so by hand
    #   psi_1 = sqrt(2) x,  psi_3 = (6 r - 4) x
    # (r - E r^2 / E r = r - 2/3, normalised by E[(r - 2/3)^2 r] = 1/36).
    rng = np.random.default_rng([70, 2])
    n = 1 << 21
    r = (np.arange(n) + 0.5) / n          # midpoint rule: moments within 1e-12
    x = np.sqrt(r) * np.exp(2j * np.pi * rng.random(n))
    U = mod.orthonormal_coefficients(x, 2)
    assert np.allclose(U, [[np.sqrt(2.0), -4.0], [0.0, 6.0]], rtol=1e-8, atol=1e-8), U


def pin_lstsq_equals_monomial(mod=basis):
    P, Q, M, n = 9, 5, 3, 6000
    u = synth.clipped_gaussian(n, 0.3, key=(70, 3))
    t = synth.ofdm2(n, key=(70, 4))
    h_mono = basis.lstsq(u, t, P, Q, M)
    h, h_o, U = mod.lstsq_orthogonal(u, t, P, Q, M)
    assert np.linalg.norm(h - h_mono) <= 1e-9 * np.linalg.norm(h_mono)
    # the orthogonal system is much better conditioned
    Psi = basis.basis_matrix(u, P, Q, M)
    W = mod.transform_matrix(U, P, Q, M)
    assert np.linalg.cond(Psi @ W) < 1e-2 * np.linalg.cond(Psi)


PINS = [pin_orthonormal_tap0, pin_single_order_closed_form, pin_uniform_power_closed_form,
        pin_lstsq_equals_monomial]


@pytest.mark.parametrize("pin", PINS, ids=[p.__name__ for p in PINS])
def test_pin(pin):
    pin()


MUTANTS = {
    "w_transposed": ("W[base + a * L + k, base + b * L + k] = U[a, b]", "W[base + b * L + k, base + a * L + k] = U[a, b]"),
    "not_normalised": ("coef = coef / nrm", "coef = coef / 1.0"),
    "projection_sign": ("v = v - proj * phi", "v = v + proj * phi"),
    "conj_branch_skipped": ("for base, nb in ((0, Bp), (Bp * L, Bq)):", "for base, nb in ((0, Bp),):"),
}


def _mutated_module(old, new):
    ns = {"np": np, "_orders": basis._orders, "basis_matrix": basis.basis_matrix}
    for fn in (basis.orthonormal_coefficients, basis.transform_matrix, basis.lstsq_orthogonal):
        src = textwrap.dedent(inspect.getsource(fn))
        exec(compile(src.replace(old, new), "<mutant>", "exec"), ns)

    class M:
        pass
    m = M()
    for name in ("orthonormal_coefficients", "transform_matrix", "lstsq_orthogonal", "basis_matrix"):
        setattr(m, name, ns[name])
    return m


def test_planted_mistakes_are_caught():
    src = "".join(inspect.getsource(f) for f in (basis.orthonormal_coefficients, basis.transform_matrix))
    for name, (old, new) in MUTANTS.items():
        assert src.count(old) == 1, name
        mod = _mutated_module(old, new)
        caught = []
        for pin in PINS:
            try:
                pin(mod)
            except (AssertionError, np.linalg.LinAlgError, ValueError, FloatingPointError):
                caught.append(pin.__name__)
        assert caught, f"planted mistake '{name}' passed every pin"
