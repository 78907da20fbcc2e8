"""Measurement operator Phi_l = Theta_l G_l F Z and its adjoint (Sec. 2.1, Eq. "inverse").

Conventions (the paper fixes none of them; these are the readings used):
  * image x_l is real, stored (ny, nx); pixel (iy, ix) has centred coordinates
    (n1, n2) = (ix - nx/2, iy - ny/2); u pairs with n1 (x axis), v with n2;
  * Z: place c_y(iy) c_x(ix) x[iy, ix] at grid cell (n2 mod Ky, n1 mod Kx) of the
    o-times oversampled grid Ky x Kx = (o ny) x (o nx), zero elsewhere;
  * F: unnormalised 2-D DFT with a negative exponent, matching the sign of
    Eq. "RIdata1" (numpy's fft2);
  * G_l: row m interpolates the spectrum at grid coordinate t = u_m K / (2 pi)
    from the J cells k = floor(t) - (J/2 - 1) ... floor(t) + J/2 (mod K) with
    weight phi(t - k), separably in both axes;
  * Theta_l: real diagonal weights (1 when not given).
  * adjoint: Phi_l^dagger y = Re(Z^T F^H G_l^H Theta_l y). X is real (Sec. 2.1),
    so the adjoint for the real inner product <a, b> = Re(a^H b) keeps the real
    part; F^H is the unnormalised inverse DFT (K * numpy ifft2).

With these choices Phi_l x approximates the direct NUDFT
    sum_n x_n exp(-i (u n1 + v n2))
(Eq. "RIdata1" with w = 0 and the sky already multiplied by the beam).
"""

from __future__ import annotations

import numpy as np

from .kaiser_bessel import kb, kb_beta, scaling


class ChannelOperator:
    """Phi_l for one channel, explicit and unfused."""

    def __init__(self, nx: int, ny: int, uv: np.ndarray, weights=None, o: int = 2, J: int = 8,
                 beta: float | None = None):
        self.nx, self.ny, self.o, self.J = nx, ny, o, J
        self.Kx, self.Ky = o * nx, o * ny
        self.beta = kb_beta(J, o) if beta is None else float(beta)
        uv = np.asarray(uv, dtype=np.float64)
        self.M = uv.shape[0]
        self.w = np.ones(self.M) if weights is None else np.asarray(weights, dtype=np.float64)
        # grid coordinates and interpolation windows
        tu = uv[:, 0] * self.Kx / (2.0 * np.pi)
        tv = uv[:, 1] * self.Ky / (2.0 * np.pi)
        taps = np.arange(J) - (J // 2 - 1)
        ku = np.floor(tu)[:, None] + taps[None, :]
        kv = np.floor(tv)[:, None] + taps[None, :]
        self.phi_u = kb(tu[:, None] - ku, J, self.beta)       # (M, J)
        self.phi_v = kb(tv[:, None] - kv, J, self.beta)       # (M, J)
        self.ix = np.mod(ku, self.Kx).astype(np.int64)        # (M, J)
        self.iy = np.mod(kv, self.Ky).astype(np.int64)        # (M, J)
        self.cx = scaling(nx, self.Kx, J, self.beta)
        self.cy = scaling(ny, self.Ky, J, self.beta)
        self.rows = np.mod(np.arange(ny) - ny // 2, self.Ky)
        self.cols = np.mod(np.arange(nx) - nx // 2, self.Kx)

    # ---- Z and its transpose ------------------------------------------------
    def Z(self, x: np.ndarray) -> np.ndarray:
        g = np.zeros((self.Ky, self.Kx), dtype=np.complex128)
        g[np.ix_(self.rows, self.cols)] = self.cy[:, None] * self.cx[None, :] * x
        return g

    def Zt(self, g: np.ndarray) -> np.ndarray:
        return self.cy[:, None] * self.cx[None, :] * g[np.ix_(self.rows, self.cols)]

    # ---- G and its adjoint --------------------------------------------------
    def G(self, ghat: np.ndarray) -> np.ndarray:
        win = ghat[self.iy[:, :, None], self.ix[:, None, :]]   # (M, J, J) rows v, cols u
        return np.einsum("ma,mb,mab->m", self.phi_v, self.phi_u, win)

    def GH(self, z: np.ndarray) -> np.ndarray:
        contrib = z[:, None, None] * self.phi_v[:, :, None] * self.phi_u[:, None, :]
        flat = (self.iy[:, :, None] * self.Kx + self.ix[:, None, :]).ravel()
        c = contrib.ravel()
        n = self.Ky * self.Kx
        re = np.bincount(flat, weights=c.real, minlength=n)
        im = np.bincount(flat, weights=c.imag, minlength=n)
        return (re + 1j * im).reshape(self.Ky, self.Kx)

    # ---- Phi and Phi^dagger -------------------------------------------------
    def forward(self, x: np.ndarray) -> np.ndarray:
        """Phi_l x = Theta G F Z x."""
        return self.w * self.G(np.fft.fft2(self.Z(x)))

    def adjoint(self, y: np.ndarray) -> np.ndarray:
        """Phi_l^dagger y = Re(Z^T F^H G^H Theta y)."""
        g = self.GH(self.w * np.asarray(y, dtype=np.complex128))
        gt = np.fft.ifft2(g) * (self.Ky * self.Kx)
        return self.Zt(gt).real

    def adjoint_pixels(self, y: np.ndarray, pix: np.ndarray) -> np.ndarray:
        """Selected entries of Phi_l^dagger y, each summed directly without the FFT:
        (Phi^dagger y)[iy, ix] = c_y c_x Re(sum_m w_m y_m sum_window phi phi
        exp(+2 pi i (k_v n2 / Ky + k_u n1 / Kx))). pix is (P, 2) of (iy, ix)."""
        z = self.w * np.asarray(y, dtype=np.complex128)
        out = np.empty(len(pix))
        for p, (iy, ix) in enumerate(pix):
            n1 = ix - self.nx // 2
            n2 = iy - self.ny // 2
            eu = np.exp(2j * np.pi * self.ix * n1 / self.Kx) * self.phi_u   # (M, J)
            ev = np.exp(2j * np.pi * self.iy * n2 / self.Ky) * self.phi_v   # (M, J)
            s = np.sum(z * eu.sum(axis=1) * ev.sum(axis=1))
            out[p] = self.cy[iy] * self.cx[ix] * s.real
        return out


class WidebandOperator:
    """Phi(X) = [Phi_l x_l]_l over channel-concatenated visibilities (Sec. 2.1)."""

    def __init__(self, nx: int, ny: int, uv: np.ndarray, offsets: np.ndarray, weights=None,
                 o: int = 2, J: int = 8):
        self.nx, self.ny = nx, ny
        self.offsets = np.asarray(offsets, dtype=np.int64)
        self.L = len(self.offsets) - 1
        self.ch = []
        for l in range(self.L):
            a, b = self.offsets[l], self.offsets[l + 1]
            w = None if weights is None else weights[a:b]
            self.ch.append(ChannelOperator(nx, ny, uv[a:b], w, o=o, J=J))

    def forward(self, X: np.ndarray) -> np.ndarray:
        out = np.empty(int(self.offsets[-1]), dtype=np.complex128)
        for l, op in enumerate(self.ch):
            out[self.offsets[l]:self.offsets[l + 1]] = op.forward(X[l])
        return out

    def adjoint(self, Y: np.ndarray) -> np.ndarray:
        out = np.empty((self.L, self.ny, self.nx))
        for l, op in enumerate(self.ch):
            out[l] = op.adjoint(Y[self.offsets[l]:self.offsets[l + 1]])
        return out

    def split(self, Y: np.ndarray):
        return [Y[self.offsets[l]:self.offsets[l + 1]] for l in range(self.L)]


def nudft(x: np.ndarray, uv: np.ndarray) -> np.ndarray:
    """Direct sum y_m = sum_n x_n exp(-i (u_m n1 + v_m n2)), centred pixel
    coordinates (coplanar limit of Eq. "RIdata1")."""
    ny, nx = x.shape
    n1 = np.arange(nx) - nx // 2
    n2 = np.arange(ny) - ny // 2
    eu = np.exp(-1j * np.outer(uv[:, 0], n1))     # (M, nx)
    ev = np.exp(-1j * np.outer(uv[:, 1], n2))     # (M, ny)
    return np.einsum("my,yx,mx->m", ev, x, eu)
