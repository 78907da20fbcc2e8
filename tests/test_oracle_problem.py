"""Pins for the oracle's problem set-up quantities (Secs. 2.3, 4.3).

* eta_l (PSF normalisation of the dirty cube): Phi_l delta of the unit image at
  the phase centre is Theta_l times the all-ones vector (every visibility of a
  point source at the origin is 1), so the PSF Phi_l^dagger Phi_l delta peaks
  at the centre with value sum_m w_m^2 (= M_l without weights), to the NUFFT's
  accuracy; eta_l is its reciprocal.
* mu = ||X||_* / ||Psi^dagger X||_{2,1} on a rank-two cube whose two terms
  have closed-form wavelet coefficients: a constant image (only the coarsest
  approximation band of every wavelet is non-zero, 2^J c per coefficient) and
  a checkerboard (only the finest diagonal band, 2 c per coefficient, because
  sum_j h_j (-1)^j = 0 and sum_j g_j (-1)^j = sqrt(2)), with orthogonal unit
  spectra. The nuclear norm n (c1 + c2) differs from the Frobenius norm
  n sqrt(c1^2 + c2^2), and the l2,1 norm counts the 1/3 frame scaling, the
  Dirac rows and the level count."""

import numpy as np
import pytest

import synth
from oracle import nufft, problem


def _op(n=32, L=3, M=(300, 451, 800), seed=91, weights=False):
    inp = synth.make_inputs(1, n=n, L=L, M=M[-1], seed=seed)
    off = np.zeros(L + 1, dtype=np.int64)
    off[1:] = np.cumsum(M)
    uv = np.concatenate([inp.uv[inp.offsets[l]:inp.offsets[l] + M[l]] for l in range(L)])
    w = None
    if weights:
        w = np.random.default_rng(seed).uniform(0.5, 1.5, off[-1])
    return nufft.WidebandOperator(n, n, uv, off, w), w, off


@pytest.mark.parametrize("weights", [False, True])
def test_psf_peak_is_sum_of_squared_weights(weights):
    op, w, off = _op(weights=weights)
    eta = problem.psf_peak_norm(op)
    for l, ch in enumerate(op.ch):
        expect = float(ch.M) if w is None else float(np.sum(w[off[l]:off[l + 1]] ** 2))
        assert 1.0 / eta[l] == pytest.approx(expect, rel=1e-5)
        delta = np.zeros((op.ny, op.nx))
        delta[op.ny // 2, op.nx // 2] = 1.0
        psf = ch.adjoint(ch.forward(delta))
        assert np.unravel_index(np.argmax(psf), psf.shape) == (op.ny // 2, op.nx // 2)


def test_dirty_cube_is_eta_times_adjoint():
    op, _, off = _op()
    y = np.random.default_rng(2).standard_normal(off[-1]) + 0j
    Xd = problem.dirty_cube(op, y)
    for l, ch in enumerate(op.ch):
        np.testing.assert_allclose(Xd[l] * ch.M, ch.adjoint(y[off[l]:off[l + 1]]), rtol=1e-5, atol=1e-9)


@pytest.mark.parametrize("n,levels", [(32, 2), (64, 3), (64, 4)])
def test_mu_closed_form_rank_two_cube(n, levels):
    c1, c2 = 0.7, 0.3
    L = 5
    rng = np.random.default_rng(n + levels)
    Q, _ = np.linalg.qr(rng.standard_normal((L, 2)))
    h1, h2 = Q[:, 0], Q[:, 1]
    iy, ix = np.meshgrid(np.arange(n), np.arange(n), indexing="ij")
    chk = (-1.0) ** (iy + ix)
    X = c1 * h1[:, None, None] * np.ones((n, n))[None] + c2 * h2[:, None, None] * chk[None]
    nuc = n * (c1 + c2)
    assert problem.nuclear_norm(X) == pytest.approx(nuc, rel=1e-12)
    l21 = (n * n * np.hypot(c1, c2) + 8 * (n / 2 ** levels) ** 2 * 2 ** levels * c1
           + 8 * (n / 2) ** 2 * 2 * c2) / 3.0
    assert problem.mu_from_cube(X, levels) == pytest.approx(nuc / l21, rel=1e-12)
