"""Data synthesis and solver parameters for a synthetic problem (Secs. 2.3, 3.4, 4.1).

Readings:
  * one noise level for all visibilities, set from the input SNR on the whole
    cube: sigma = ||Phi(X_true)|| / sqrt(sum M) * 10^(-InSNR / 20), noise
    sigma * (N(0,1) + i N(0,1)) / sqrt(2) (Sec. 4.1);
  * l2 bound from the chi-square statistics of the noise norm (Sec. 4.1):
    ||w_l||^2 has mean sigma^2 M_l and standard deviation sigma^2 sqrt(M_l), so
    epsilon_l = sigma sqrt(M_l + 2 sqrt(M_l)) (mean plus two deviations);
  * dirty cube X_dirty,l = eta_l Phi_l^dagger y_l with eta_l = 1 / max(Phi_l^dagger
    Phi_l delta), delta the unit image at the phase centre (Sec. 4.3 footnote);
  * mu = ||X_dirty||_* / ||Psi^dagger X_dirty||_{2,1} (Sec. 2.3);
  * kappa_3 = 1 / max_l ||U_l^{1/2} Phi_l||^2 by power iteration on
    Phi_l^dagger U_l Phi_l (Sec. 3.4).
"""

from __future__ import annotations

from dataclasses import dataclass

import numpy as np

from . import nufft, wavelets, prox


@dataclass
class Problem:
    op: nufft.WidebandOperator
    truth: np.ndarray
    y: np.ndarray
    sigma: float
    eps: np.ndarray


def build_operator(inp, weights=None, uv=None) -> nufft.WidebandOperator:
    uv = inp.uv if uv is None else uv
    return nufft.WidebandOperator(inp.nx, inp.ny, uv, inp.offsets, weights)


def noise_sigma(y_clean: np.ndarray, insnr_db: float) -> float:
    return float(np.linalg.norm(y_clean) / np.sqrt(y_clean.size) * 10.0 ** (-insnr_db / 20.0))


def l2_bounds(sigma: float, M: np.ndarray) -> np.ndarray:
    M = np.asarray(M, dtype=np.float64)
    return sigma * np.sqrt(M + 2.0 * np.sqrt(M))


def make_problem(inp, weights=None, truth=None, uv=None) -> Problem:
    """y = Phi(X_true) + sigma * noise with the generator's draws."""
    op = build_operator(inp, weights, uv)
    X = inp.truth if truth is None else truth
    y_clean = op.forward(X)
    sigma = noise_sigma(y_clean, inp.insnr)
    y = y_clean + sigma * inp.noise
    eps = l2_bounds(sigma, np.diff(inp.offsets))
    return Problem(op=op, truth=X, y=y, sigma=sigma, eps=eps)


def psf_peak_norm(op: nufft.WidebandOperator) -> np.ndarray:
    """eta_l = 1 / max_n (Phi_l^dagger Phi_l delta)_n."""
    delta = np.zeros((op.ny, op.nx))
    delta[op.ny // 2, op.nx // 2] = 1.0
    return np.array([1.0 / np.max(ch.adjoint(ch.forward(delta))) for ch in op.ch])


def dirty_cube(op: nufft.WidebandOperator, y: np.ndarray) -> np.ndarray:
    eta = psf_peak_norm(op)
    return eta[:, None, None] * op.adjoint(y)


def nuclear_norm(X: np.ndarray) -> float:
    return float(np.sum(np.linalg.svd(X.reshape(X.shape[0], -1).T, compute_uv=False)))


def l21_norm(A: np.ndarray) -> float:
    return float(np.sum(prox.row_norms(A)))


def mu_from_cube(X: np.ndarray, levels: int = 4) -> float:
    """||X||_* / ||Psi^dagger X||_{2,1} of a cube (the ratio of Sec. 2.3)."""
    return nuclear_norm(X) / l21_norm(wavelets.psi_adjoint_cube(X, levels))


def estimate_mu(op, y, levels: int = 4) -> float:
    """mu = ||X_dirty||_* / ||Psi^dagger X_dirty||_{2,1} (Sec. 2.3)."""
    return mu_from_cube(dirty_cube(op, y), levels)


def op_norm2(op: nufft.WidebandOperator, U=None, iters: int = 500, tol: float = 1e-10,
             seed: int = 0) -> float:
    """max_l ||U_l^{1/2} Phi_l||_S^2 by power iteration on Phi_l^dagger U_l Phi_l."""
    rng = np.random.Generator(np.random.PCG64(seed))
    best = 0.0
    for l, ch in enumerate(op.ch):
        if ch.M == 0:
            continue
        Ul = None if U is None else U[op.offsets[l]:op.offsets[l + 1]]
        x = rng.standard_normal((op.ny, op.nx))
        x /= np.linalg.norm(x)
        lam = 0.0
        for _ in range(iters):
            yv = ch.forward(x)
            if Ul is not None:
                yv = Ul * yv
            z = ch.adjoint(yv)
            lam_new = float(np.linalg.norm(z))
            x = z / lam_new
            if abs(lam_new - lam) <= tol * lam_new:
                lam = lam_new
                break
            lam = lam_new
        best = max(best, lam)
    return best
