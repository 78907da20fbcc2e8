"""Gradient of the smooth-plus-l2,1 objective built from the measurement model
(Sec. 2.1, Eq. "inverse") and the joint average sparsity prior (Sec. 2.3):

    f(X) = 0.5 ||Phi(X) - y||_2^2 + ||Psi^dagger X||_{2,1},

    grad f(X) = Phi^dagger (Phi(X) - y) + Psi D(Psi^dagger X),

where D(A) scales every row a_n (one coefficient across the L channels) to
a_n / ||a_n|| and maps a zero row to 0 (the minimum-norm subgradient of the
row norm). Phi^dagger keeps the real part (X is real, Sec. 2.1), so the first
term is the gradient for the real inner product.

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).
"""

from __future__ import annotations

import numpy as np

from . import prox, wavelets


def row_directions(A: np.ndarray, w_rows=1.0) -> np.ndarray:
    """D(A): w_n a_n / ||a_n|| row by row (0 for zero rows); A is (9, L, ny, nx)."""
    nrm = prox.row_norms(A)
    w = np.broadcast_to(np.asarray(w_rows, dtype=np.float64), nrm.shape)
    with np.errstate(divide="ignore", invalid="ignore"):
        f = np.where(nrm > 0, w / nrm, 0.0)
    return A * f[:, None]


def objective(op, X: np.ndarray, y: np.ndarray, levels: int, w_rows=1.0) -> float:
    r = op.forward(X) - y
    A = wavelets.psi_adjoint_cube(X, levels)
    w = np.broadcast_to(np.asarray(w_rows, dtype=np.float64), prox.row_norms(A).shape)
    return float(0.5 * np.sum(np.abs(r) ** 2) + np.sum(w * prox.row_norms(A)))


def gradient(op, X: np.ndarray, y: np.ndarray, levels: int, w_rows=1.0) -> np.ndarray:
    g = op.adjoint(op.forward(X) - y)
    A = wavelets.psi_adjoint_cube(X, levels)
    return g + wavelets.psi_cube(row_directions(A, w_rows), levels)
