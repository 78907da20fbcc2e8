"""Reconstruction quality metrics (Sec. 4.3)."""

from __future__ import annotations

import numpy as np


def snr(x_true: np.ndarray, x_hat: np.ndarray) -> float:
    """SNR_l = 20 log10(||x_true|| / ||x_true - x_hat||)."""
    num = np.sqrt(np.sum(np.asarray(x_true, dtype=np.float64) ** 2))
    den = np.sqrt(np.sum((np.asarray(x_true, dtype=np.float64) - x_hat) ** 2))
    return float(20.0 * np.log10(num / den))


def asnr(X_true: np.ndarray, X_hat: np.ndarray) -> float:
    """aSNR = mean over channels of SNR_l; cubes are (L, ny, nx)."""
    return float(np.mean([snr(X_true[l], X_hat[l]) for l in range(X_true.shape[0])]))
