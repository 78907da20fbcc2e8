"""Kaiser-Bessel interpolation kernel for the de-gridding matrix G (Sec. 2.1).

The paper only says that G carries "a convolution kernel on its rows"; the
reading used here is the separable Kaiser-Bessel kernel with support J cells,

    phi(x) = I0(beta * sqrt(1 - (2x/J)^2))   for |x| <= J/2, else 0,

with beta from the published rule of Beatty, Nishimura & Pauly (2005) for
oversampling o:  beta = pi * sqrt((J/o)^2 (o - 1/2)^2 - 0.8).

Its continuous Fourier transform (Jackson et al. 1991) is

    phihat(f) = J * sinh(sqrt(beta^2 - (pi J f)^2)) / sqrt(beta^2 - (pi J f)^2),

continued with sin/sqrt when the radicand is negative. Z scales pixel n
(centred coordinate) by 1 / phihat(n / K) on each axis, which undoes the
kernel's apodisation ("corrects for imperfections in the interpolation").
"""

from __future__ import annotations

import numpy as np


def kb_beta(J: int, o: float) -> float:
    """Beatty et al. shape parameter for support J and oversampling o."""
    return float(np.pi * np.sqrt((J / o) ** 2 * (o - 0.5) ** 2 - 0.8))


def kb(x, J: int, beta: float) -> np.ndarray:
    """phi(x): Kaiser-Bessel window of support [-J/2, J/2]."""
    x = np.asarray(x, dtype=np.float64)
    out = np.zeros_like(x)
    inside = np.abs(x) <= J / 2.0
    r = 1.0 - (2.0 * x[inside] / J) ** 2
    out[inside] = np.i0(beta * np.sqrt(np.maximum(r, 0.0)))
    return out


def kb_ft(f, J: int, beta: float) -> np.ndarray:
    """Closed-form continuous Fourier transform of kb at frequency f (cycles/cell)."""
    f = np.asarray(f, dtype=np.float64)
    a = beta ** 2 - (np.pi * J * f) ** 2
    out = np.empty_like(f)
    pos = a > 0
    neg = a < 0
    zero = ~(pos | neg)
    s = np.sqrt(a[pos])
    out[pos] = J * np.sinh(s) / s
    s = np.sqrt(-a[neg])
    out[neg] = J * np.sin(s) / s
    out[zero] = J
    return out


def scaling(n_pix: int, K: int, J: int, beta: float) -> np.ndarray:
    """Z's per-axis scale c(n) = 1 / phihat(n / K) for centred n = i - n_pix/2."""
    n = np.arange(n_pix) - n_pix // 2
    return 1.0 / kb_ft(n / K, J, beta)
