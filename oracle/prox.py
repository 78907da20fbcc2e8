"""Proximity operators of the HyperSARA problem and their Moreau duals (Sec. 3.3).

All operators act on channel-major cubes: an image cube X (L, ny, nx) is the
paper's N x L matrix with column l = X[l].ravel(); a coefficient cube A
(9, L, ny, nx) is the R x L matrix (R = 9N) whose row n collects one
coefficient across all L channels.

Dual forms follow the Moreau decomposition (Eq. "md") with U = I:
  (I - prox_{g})(z)  is the prox of the conjugate, used in Algorithm 2 steps
  5, 7 and 11.
Zero-norm ties: a zero row / zero residual is returned unchanged by the dual
forms (the primal prox returns 0 there); a zero singular value has dual factor 1.
"""

from __future__ import annotations

import numpy as np


def proj_positive(X: np.ndarray) -> np.ndarray:
    """Eq. "proj-plus": Re(x) where Re(x) > 0, else 0."""
    return np.maximum(np.real(X), 0.0)


def _as_matrix(X: np.ndarray) -> np.ndarray:
    """(L, ny, nx) cube -> N x L matrix (columns are channels)."""
    return X.reshape(X.shape[0], -1).T


def _from_matrix(M: np.ndarray, shape) -> np.ndarray:
    return M.T.reshape(shape)


def prox_nuclear(X: np.ndarray, w, thr: float = 1.0) -> np.ndarray:
    """Eq. "prox-L*": singular values soft-thresholded by thr * w_j (w: scalar or
    (L,) weights ordered like the singular values, descending)."""
    Mx = _as_matrix(X)
    U, s, Vt = np.linalg.svd(Mx, full_matrices=False)
    wv = np.broadcast_to(np.asarray(w, dtype=np.float64), s.shape)
    s2 = np.maximum(s - thr * wv, 0.0)
    return _from_matrix((U * s2) @ Vt, X.shape)


def nuclear_dual(Z: np.ndarray, w, thr: float = 1.0):
    """(I - S*_w)(Z) = U diag(min(s, thr w)) V^T (Algorithm 2 step 5).

    Returns (out, singular values of Z)."""
    Mz = _as_matrix(Z)
    U, s, Vt = np.linalg.svd(Mz, full_matrices=False)
    wv = np.broadcast_to(np.asarray(w, dtype=np.float64), s.shape)
    s2 = np.minimum(s, thr * wv)
    return _from_matrix((U * s2) @ Vt, Z.shape), s


def row_norms(A: np.ndarray) -> np.ndarray:
    """l2 norm of every row n (across channels): A (D, L, ...) -> (D, ...)."""
    return np.sqrt(np.sum(A * A, axis=1))


def prox_l21(A: np.ndarray, w_rows, thr: float) -> np.ndarray:
    """Eq. "prox-L21": row n -> max(||a_n|| - thr w_n, 0) a_n / ||a_n||.

    A is (D, L, ny, nx); w_rows is a scalar or (D, ny, nx)."""
    nrm = row_norms(A)
    lam = thr * np.broadcast_to(np.asarray(w_rows, dtype=np.float64), nrm.shape)
    with np.errstate(divide="ignore", invalid="ignore"):
        f = np.where(nrm > 0, np.maximum(nrm - lam, 0.0) / nrm, 0.0)
    return A * f[:, None]


def l21_dual(Q: np.ndarray, w_rows, thr: float) -> np.ndarray:
    """(I - S^{l21}_{thr w})(Q): row n scaled by min(1, thr w_n / ||q_n||)
    (Algorithm 2 step 7)."""
    nrm = row_norms(Q)
    lam = thr * np.broadcast_to(np.asarray(w_rows, dtype=np.float64), nrm.shape)
    with np.errstate(divide="ignore", invalid="ignore"):
        f = np.where(nrm > lam, lam / nrm, 1.0)
    return Q * f[:, None]


def prox_l1(A: np.ndarray, w, thr: float) -> np.ndarray:
    """Weighted l1 prox (soft thresholding) of every coefficient: sign(a) max(|a| - thr w, 0).
    The SARA prior of the single-channel benchmark (Sec. 4.2): the sparsity
    term of each channel on its own, no coupling across channels."""
    lam = thr * np.broadcast_to(np.asarray(w, dtype=np.float64), A.shape)
    return np.sign(A) * np.maximum(np.abs(A) - lam, 0.0)


def l1_dual(Q: np.ndarray, w, thr: float) -> np.ndarray:
    """(I - S^{l1}_{thr w})(Q): every coefficient clipped to [-thr w, thr w]
    (the step-7 dual update with the l1 prior in place of l2,1)."""
    lam = thr * np.broadcast_to(np.asarray(w, dtype=np.float64), Q.shape)
    return np.clip(Q, -lam, lam)


def proj_l2ball(z: np.ndarray, y: np.ndarray, eps: float) -> np.ndarray:
    """Projection onto B(y, eps) = {z : ||z - y||_2 <= eps} (Sec. 3.2, functions g_l)."""
    d = z - y
    nrm = np.sqrt(np.sum(np.abs(d) ** 2))
    if nrm <= eps:
        return np.array(z, copy=True)
    return y + d * (eps / nrm)


def l2ball_dual(vbar: np.ndarray, y: np.ndarray, eps: float, U=None) -> np.ndarray:
    """Algorithm 2 step 11 with diagonal U:
    v = U^{1/2} (z - P_B(y, eps)(z)), z = U^{-1/2} vbar.

    The ellipsoid projection is read as the Euclidean ball projection of the
    U^{-1/2}-scaled variable (Sec. 3.3); U = I gives (I - P_B)(vbar)."""
    if U is None:
        return vbar - proj_l2ball(vbar, y, eps)
    s = np.sqrt(np.asarray(U, dtype=np.float64))
    z = vbar / s
    return s * (z - proj_l2ball(z, y, eps))
