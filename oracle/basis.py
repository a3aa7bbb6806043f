"""Second, independent formulation of the APH DPD filter: the basis matrix Psi.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

Eq. 2 defines, for every odd order p, a Toeplitz block Psi_p whose row n holds
``psi_p(x_n), psi_p(x_{n-1}), ..., psi_p(x_{n-L+1})`` with zeros above the first
sample.  Sec. 2.2 stacks the blocks side by side, ``[Psi_1 .. Psi_P, Psibar_1 ..
Psibar_Q, 1]``, so that the filter output is the matrix-vector product
``z = Psi h`` and the least-squares estimate is ``(Psi^H Psi)^{-1} Psi^H z``.

The full-convolution tail rows of Eq. 2 (past the last input sample) are
dropped: the filter produces one output per input sample.
"""
from __future__ import annotations

import numpy as np


def _orders(top: int):
    return list(range(1, top + 1, 2)) if top > 0 else []


def basis_matrix(x, P: int, Q: int, M: int) -> np.ndarray:
    """N x K complex128 basis matrix, columns in the paper's stacking order."""
    x = np.asarray(x).astype(np.complex128)
    n = x.shape[0]
    L = M + 1
    cols = []
    mag = np.abs(x)
    for p in _orders(P):
        col0 = mag ** (p - 1) * x                  # psi_p(x_n) = |x_n|^{p-1} x_n
        for k in range(L):                         # Toeplitz shift by k, zero history
            c = np.zeros(n, dtype=np.complex128)
            c[k:] = col0[: n - k] if k < n else 0
            cols.append(c)
    for q in _orders(Q):
        col0 = mag ** (q - 1) * np.conj(x)         # psibar_q(x_n) = |x_n|^{q-1} x_n^*
        for k in range(L):
            c = np.zeros(n, dtype=np.complex128)
            c[k:] = col0[: n - k] if k < n else 0
            cols.append(c)
    cols.append(np.ones(n, dtype=np.complex128))   # multiplies the LO-leakage constant c
    return np.stack(cols, axis=1)


def apply(x, h, P: int, Q: int, M: int) -> np.ndarray:
    """z = Psi h."""
    return basis_matrix(x, P, Q, M) @ np.asarray(h).astype(np.complex128)


def lstsq(u, t, P: int, Q: int, M: int) -> np.ndarray:
    """argmin_h ||Psi(u) h - t||_2 by numpy's SVD-based solver."""
    Psi = basis_matrix(u, P, Q, M)
    return np.linalg.lstsq(Psi, np.asarray(t).astype(np.complex128), rcond=None)[0]


def orthonormal_coefficients(u, B: int) -> np.ndarray:
    """The u_{m,p} of Sec. 2.1 ("statistically orthogonal polynomials") for the
    odd orders 1, 3, .., 2B-1, taken with respect to the samples u themselves:
    the upper-triangular B x B real matrix U such that

        psi_{2b+1}(x) = sum_{a <= b} U[a, b] |x|^{2a} x

    are orthonormal under <f, g> = (1/N) sum_n conj(f(u_n)) g(u_n).  Built by
    modified Gram-Schmidt on the monomials |x|^{2a} x in order of increasing
    degree, so psi_p mixes only orders up to p, as in Sec. 2.1.  (The products
    <psi_j, |x|^{2b} x> are real: both factors are real multiples of x.)"""
    x = np.asarray(u).astype(np.complex128)
    n = x.shape[0]
    r = np.abs(x) ** 2
    U = np.zeros((B, B))
    done = []   # (psi_j values, column j of U)
    for b in range(B):
        v = r ** b * x
        coef = np.zeros(B)
        coef[b] = 1.0
        for phi, cj in done:
            proj = (np.vdot(phi, v) / n).real
            v = v - proj * phi
            coef = coef - proj * cj
        nrm = np.sqrt((np.vdot(v, v) / n).real)
        v = v / nrm
        coef = coef / nrm
        done.append((v, coef))
        U[:, b] = coef
    return U


def transform_matrix(U, P: int, Q: int, M: int) -> np.ndarray:
    """K x K real matrix W with Psi(orthogonal basis) = Psi(monomials) W: per
    branch and tap, column (b, k) holds U[a, b] at row (a, k); the constant
    column maps to itself.  Coefficients convert as h_monomial = W h_orthogonal."""
    L = M + 1
    Bp, Bq = len(_orders(P)), len(_orders(Q))
    K = (Bp + Bq) * L + 1
    W = np.zeros((K, K))
    for base, nb in ((0, Bp), (Bp * L, Bq)):
        for a in range(nb):
            for b in range(nb):
                for k in range(L):
                    W[base + a * L + k, base + b * L + k] = U[a, b]
    W[K - 1, K - 1] = 1.0
    return W


def lstsq_orthogonal(u, t, P: int, Q: int, M: int):
    """Least squares in the orthogonal-polynomial basis of the samples u:
    returns (h, h_orth, U) with h = W h_orth in the monomial stacking order."""
    B = max(len(_orders(P)), len(_orders(Q)))
    U = orthonormal_coefficients(u, B)
    W = transform_matrix(U, P, Q, M)
    Psi_o = basis_matrix(u, P, Q, M) @ W
    h_o = np.linalg.lstsq(Psi_o, np.asarray(t).astype(np.complex128), rcond=None)[0]
    return W @ h_o, h_o, U
