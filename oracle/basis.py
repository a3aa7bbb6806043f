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
