"""Pins for the oracle's interpolation kernel and measurement operator.

Each check compares the oracle with something other than itself: the I0 power
series, numerical quadrature of the kernel, a direct NUDFT of the coplanar
measurement equation (Eq. "RIdata1" with w = 0), dense DFT matrices, and the
adjoint definition (Sec. 3.2)."""

import math

import numpy as np
import pytest
from scipy import integrate

from oracle import kaiser_bessel as kbm
from oracle import nufft


def i0_series(z: float) -> float:
    """I0(z) = sum_k (z/2)^(2k) / (k!)^2."""
    s, term, k = 1.0, 1.0, 0
    while term > 1e-18 * s:
        k += 1
        term *= (z / 2.0) ** 2 / (k * k)
        s += term
    return s


def test_beta_rule():
    # Beatty et al.: pi sqrt((J/o)^2 (o - 1/2)^2 - 0.8) for J = 8, o = 2 is pi sqrt(35.2)
    assert kbm.kb_beta(8, 2) == pytest.approx(math.pi * math.sqrt(35.2), rel=1e-15)


def test_kernel_matches_power_series():
    beta = kbm.kb_beta(8, 2)
    xs = np.linspace(-4.0, 4.0, 81)
    got = kbm.kb(xs, 8, beta)
    ref = np.array([i0_series(beta * math.sqrt(max(0.0, 1 - (x / 4.0) ** 2))) for x in xs])
    np.testing.assert_allclose(got, ref, rtol=1e-13)
    assert kbm.kb(np.array([4.0001, -4.5, 7.0]), 8, beta).tolist() == [0.0, 0.0, 0.0]


@pytest.mark.parametrize("f", [0.0, 0.05, 0.125, 0.2, 0.25, 0.4, 0.75])
def test_fourier_transform_closed_form_vs_quadrature(f):
    beta = kbm.kb_beta(8, 2)
    val, err = integrate.quad(lambda x: i0_series(beta * math.sqrt(max(0.0, 1 - (x / 4) ** 2)))
                              * math.cos(2 * math.pi * f * x), -4.0, 4.0, limit=400,
                              epsabs=0, epsrel=1e-13)
    got = float(kbm.kb_ft(np.array([f]), 8, beta)[0])
    assert got == pytest.approx(val, rel=1e-11, abs=1e-9 * abs(kbm.kb_ft(np.array([0.0]), 8, beta)[0]))


def _rand_uv(rng, M):
    return rng.uniform(-np.pi, np.pi, size=(M, 2))


@pytest.mark.parametrize("nx,ny,M", [(16, 16, 200), (32, 32, 500), (32, 16, 300)])
def test_nufft_matches_direct_nudft(nx, ny, M):
    rng = np.random.default_rng(11 + nx + ny)
    uv = _rand_uv(rng, M)
    x = rng.standard_normal((ny, nx))
    op = nufft.ChannelOperator(nx, ny, uv)
    a = op.forward(x)
    # direct sum written out from the measurement equation, independent of the oracle
    n1 = np.arange(nx) - nx // 2
    n2 = np.arange(ny) - ny // 2
    b = np.zeros(M, dtype=complex)
    for m in range(M):
        ph = np.exp(-1j * (uv[m, 0] * n1[None, :] + uv[m, 1] * n2[:, None]))
        b[m] = np.sum(x * ph)
    rel = np.linalg.norm(a - b) / np.linalg.norm(b)
    # measured ~7e-8 for J = 8, o = 2; the bound is the one the method states
    assert rel <= 1e-5
    assert rel <= 5e-7


def test_point_source_at_phase_centre_gives_constant_visibilities():
    rng = np.random.default_rng(5)
    uv = _rand_uv(rng, 400)
    op = nufft.ChannelOperator(32, 32, uv)
    d = np.zeros((32, 32))
    d[16, 16] = 1.0
    np.testing.assert_allclose(op.forward(d), np.ones(400), atol=1e-6)


def test_weights_scale_visibilities():
    rng = np.random.default_rng(6)
    uv = _rand_uv(rng, 50)
    w = rng.uniform(0.5, 2.0, 50)
    x = rng.standard_normal((16, 16))
    a = nufft.ChannelOperator(16, 16, uv, weights=w).forward(x)
    b = nufft.ChannelOperator(16, 16, uv).forward(x)
    np.testing.assert_allclose(a, w * b, rtol=1e-14, atol=1e-14)


@pytest.mark.parametrize("nx,ny", [(16, 16), (32, 16)])
def test_adjoint_identity(nx, ny):
    rng = np.random.default_rng(7)
    M = 333
    uv = _rand_uv(rng, M)
    w = rng.uniform(0.5, 1.5, M)
    op = nufft.ChannelOperator(nx, ny, uv, weights=w)
    x = rng.standard_normal((ny, nx))
    y = rng.standard_normal(M) + 1j * rng.standard_normal(M)
    lhs = np.real(np.vdot(op.forward(x), y))
    rhs = np.sum(x * op.adjoint(y))
    assert abs(lhs - rhs) <= 1e-13 * abs(lhs)


def test_operator_equals_dense_matrix_product():
    """G F Z as dense matrices (explicit DFT matrix, explicit interpolation rows)."""
    rng = np.random.default_rng(8)
    nx, ny, M = 8, 4, 20
    Kx, Ky = 16, 8
    uv = _rand_uv(rng, M)
    op = nufft.ChannelOperator(nx, ny, uv)
    beta = kbm.kb_beta(8, 2)
    Z = np.zeros((Ky * Kx, ny * nx))
    cx = 1.0 / kbm.kb_ft((np.arange(nx) - nx // 2) / Kx, 8, beta)
    cy = 1.0 / kbm.kb_ft((np.arange(ny) - ny // 2) / Ky, 8, beta)
    for iy in range(ny):
        for ix in range(nx):
            k = ((iy - ny // 2) % Ky) * Kx + (ix - nx // 2) % Kx
            Z[k, iy * nx + ix] = cy[iy] * cx[ix]
    Fx = np.exp(-2j * np.pi * np.outer(np.arange(Kx), np.arange(Kx)) / Kx)
    Fy = np.exp(-2j * np.pi * np.outer(np.arange(Ky), np.arange(Ky)) / Ky)
    F = np.kron(Fy, Fx)
    G = np.zeros((M, Ky * Kx))
    for m in range(M):
        tu = uv[m, 0] * Kx / (2 * np.pi)
        tv = uv[m, 1] * Ky / (2 * np.pi)
        for a in range(8):
            kv = math.floor(tv) - 3 + a
            for b in range(8):
                ku = math.floor(tu) - 3 + b
                G[m, (kv % Ky) * Kx + ku % Kx] += (kbm.kb(np.array([tv - kv]), 8, beta)[0]
                                                   * kbm.kb(np.array([tu - ku]), 8, beta)[0])
    x = rng.standard_normal((ny, nx))
    dense = G @ F @ Z @ x.ravel()
    np.testing.assert_allclose(op.forward(x), dense, rtol=1e-12, atol=1e-9)
    y = rng.standard_normal(M) + 1j * rng.standard_normal(M)
    adj = np.real(Z.T @ F.conj().T @ G.T @ y).reshape(ny, nx)
    np.testing.assert_allclose(op.adjoint(y), adj, rtol=1e-12, atol=1e-9)


def test_fft_parseval():
    rng = np.random.default_rng(9)
    g = rng.standard_normal((16, 32)) + 1j * rng.standard_normal((16, 32))
    assert np.sum(np.abs(np.fft.fft2(g)) ** 2) == pytest.approx(g.size * np.sum(np.abs(g) ** 2),
                                                               rel=1e-13)


def test_adjoint_pixels_direct_sum_matches_fft_adjoint():
    rng = np.random.default_rng(10)
    uv = _rand_uv(rng, 120)
    op = nufft.ChannelOperator(16, 16, uv)
    y = rng.standard_normal(120) + 1j * rng.standard_normal(120)
    pix = np.array([[0, 0], [15, 15], [8, 8], [3, 11]])
    full = op.adjoint(y)
    np.testing.assert_allclose(op.adjoint_pixels(y, pix), full[pix[:, 0], pix[:, 1]],
                               rtol=1e-12, atol=1e-10)
