"""SARA dictionary: Dirac basis plus Daubechies 1-8 wavelet bases (Sec. 2.3).

Psi^dagger = (Psi_1, ..., Psi_D)^dagger with D = 9 is the analysis operator
image -> coefficients. Readings (the paper gives the bases only by name):
  * each Daubechies basis is the 2-D separable orthonormal DWT with periodic
    extension, 4 levels by default, Mallat layout in an ny x nx array;
  * the frame is normalised by 1/sqrt(9) = 1/3 so that Psi Psi^dagger = I and
    ||Psi^dagger||_S = 1;
  * db_p low-pass filters are the minimum-phase ones, obtained by spectral
    factorisation of the Daubechies polynomial (Daubechies, Ten Lectures, 6.1),
    ordered so that db2 = [(1+sqrt3), (3+sqrt3), (3-sqrt3), (1-sqrt3)] / (4 sqrt2);
    high-pass g[j] = (-1)^j h[F-1-j];
  * one level on a length-m signal (m even):
        a[k] = sum_j h[j] x[(2k + j) mod m],  d[k] = sum_j g[j] x[(2k + j) mod m],
    written as an explicit m x m matrix W = [H; G] so that the synthesis is W^T.
"""

from __future__ import annotations

from functools import lru_cache

import mpmath
import numpy as np

N_WAVELETS = 8
N_BASES = N_WAVELETS + 1
FRAME_SCALE = 1.0 / 3.0


@lru_cache(maxsize=None)
def daubechies_lowpass(p: int) -> np.ndarray:
    """db_p low-pass filter (length 2p) by spectral factorisation, computed in
    50-digit arithmetic and rounded to FP64.

    |m0(w)|^2 = cos^2p(w/2) P(sin^2(w/2)), P(y) = sum_{k<p} C(p-1+k, k) y^k.
    Each root y_r of P maps to the pair z, 1/z of z^2 + (4 y_r - 2) z + 1 = 0;
    keeping the roots inside the unit circle gives the minimum-phase factor."""
    with mpmath.workdps(50):
        if p == 1:
            q = [mpmath.mpf(1)]
        else:
            coeffs = [mpmath.binomial(p - 1 + k, k) for k in range(p)]       # ascending
            yroots = mpmath.polyroots(list(reversed(coeffs)), maxsteps=200, extraprec=200)
            zroots = []
            for yr in yroots:
                b = 1 - 2 * yr
                disc = mpmath.sqrt(b * b - 1)
                z1, z2 = b + disc, b - disc
                zroots.append(z1 if abs(z1) < 1 else z2)
            # ascending coefficients of prod (z - z_r)
            q = [mpmath.mpc(1)]
            for zr in zroots:
                nq = [mpmath.mpc(0)] * (len(q) + 1)
                for i, c in enumerate(q):
                    nq[i + 1] += c
                    nq[i] -= zr * c
                q = nq
        # multiply by (1 + z)^p
        for _ in range(p):
            nq = [mpmath.mpc(0)] * (len(q) + 1)
            for i, c in enumerate(q):
                nq[i] += c
                nq[i + 1] += c
            q = nq
        re = [mpmath.re(c) for c in q]
        s = mpmath.fsum(re)
        h = [c * mpmath.sqrt(2) / s for c in reversed(re)]
        return np.array([float(c) for c in h])


def highpass(h: np.ndarray) -> np.ndarray:
    F = len(h)
    return np.array([(-1) ** j * h[F - 1 - j] for j in range(F)])


@lru_cache(maxsize=None)
def _analysis_matrix_cached(m: int, p: int) -> np.ndarray:
    h = daubechies_lowpass(p)
    g = highpass(h)
    W = np.zeros((m, m))
    half = m // 2
    for k in range(half):
        for j in range(len(h)):
            W[k, (2 * k + j) % m] += h[j]
            W[half + k, (2 * k + j) % m] += g[j]
    W.setflags(write=False)
    return W


def analysis_matrix(m: int, p: int) -> np.ndarray:
    """One periodic DWT level on length m as the matrix [H; G] (rows: low then high)."""
    if m % 2:
        raise ValueError("DWT level needs an even length")
    return _analysis_matrix_cached(m, p)


def dwt2(x: np.ndarray, p: int, levels: int) -> np.ndarray:
    """2-D periodic orthonormal DWT with db_p, Mallat layout."""
    c = np.array(x, dtype=np.float64, copy=True)
    my, mx = c.shape
    for _ in range(levels):
        Wy = analysis_matrix(my, p)
        Wx = analysis_matrix(mx, p)
        c[:my, :mx] = Wy @ c[:my, :mx] @ Wx.T
        my //= 2
        mx //= 2
    return c


def idwt2(c: np.ndarray, p: int, levels: int) -> np.ndarray:
    """Inverse (= adjoint) of dwt2."""
    x = np.array(c, dtype=np.float64, copy=True)
    ny, nx = x.shape
    sizes = [(ny >> lev, nx >> lev) for lev in range(levels)]
    for my, mx in reversed(sizes):
        Wy = analysis_matrix(my, p)
        Wx = analysis_matrix(mx, p)
        x[:my, :mx] = Wy.T @ x[:my, :mx] @ Wx
    return x


def check_levels(ny: int, nx: int, levels: int) -> None:
    if ny % (1 << levels) or nx % (1 << levels):
        raise ValueError("image sides must be divisible by 2^levels")


def psi_adjoint(x: np.ndarray, levels: int = 4) -> np.ndarray:
    """Psi^dagger x for one image: (9, ny, nx) = [x, W_1 x, ..., W_8 x] / 3."""
    check_levels(*x.shape, levels)
    out = np.empty((N_BASES,) + x.shape)
    out[0] = x
    for p in range(1, N_WAVELETS + 1):
        out[p] = dwt2(x, p, levels)
    return FRAME_SCALE * out


def psi(a: np.ndarray, levels: int = 4) -> np.ndarray:
    """Psi a for one image's coefficients (9, ny, nx): (a_0 + sum_p W_p^T a_p) / 3."""
    x = np.array(a[0], dtype=np.float64, copy=True)
    for p in range(1, N_WAVELETS + 1):
        x += idwt2(a[p], p, levels)
    return FRAME_SCALE * x


def psi_adjoint_cube(X: np.ndarray, levels: int = 4) -> np.ndarray:
    """Psi^dagger applied to every channel: (L, ny, nx) -> (9, L, ny, nx)."""
    out = np.empty((N_BASES,) + X.shape)
    for l in range(X.shape[0]):
        out[:, l] = psi_adjoint(X[l], levels)
    return out


def psi_cube(A: np.ndarray, levels: int = 4) -> np.ndarray:
    """Psi applied to every channel: (9, L, ny, nx) -> (L, ny, nx)."""
    out = np.empty(A.shape[1:])
    for l in range(A.shape[1]):
        out[l] = psi(A[:, l], levels)
    return out
