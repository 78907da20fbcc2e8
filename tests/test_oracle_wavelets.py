"""Pins for the oracle's SARA dictionary (Sec. 2.3): published closed forms of
db1-db3, the defining properties of Daubechies filters (orthonormality under
double shifts, p vanishing moments), orthogonality of every periodic level
matrix (also when the level is shorter than the filter), the Mallat layout on
a constant image, and the frame identities Psi Psi^dagger = I and Parseval."""

import math

import numpy as np
import pytest

from oracle import wavelets as wv


def test_db1_is_haar():
    np.testing.assert_allclose(wv.daubechies_lowpass(1), [1 / math.sqrt(2)] * 2, rtol=0, atol=2e-16)


def test_db2_closed_form():
    s3 = math.sqrt(3.0)
    ref = np.array([1 + s3, 3 + s3, 3 - s3, 1 - s3]) / (4 * math.sqrt(2))
    np.testing.assert_allclose(wv.daubechies_lowpass(2), ref, rtol=0, atol=1e-15)


def test_db3_closed_form():
    # Daubechies (1988): h = [1 + sqrt10 + a, 5 + sqrt10 + 3a, 10 - 2 sqrt10 + 2a,
    # 10 - 2 sqrt10 - 2a, 5 + sqrt10 - 3a, 1 + sqrt10 - a] / (16 sqrt2), a = sqrt(5 + 2 sqrt10)
    r10 = math.sqrt(10.0)
    a = math.sqrt(5 + 2 * r10)
    ref = np.array([1 + r10 + a, 5 + r10 + 3 * a, 10 - 2 * r10 + 2 * a,
                    10 - 2 * r10 - 2 * a, 5 + r10 - 3 * a, 1 + r10 - a]) / (16 * math.sqrt(2))
    np.testing.assert_allclose(wv.daubechies_lowpass(3), ref, rtol=0, atol=1e-15)


@pytest.mark.parametrize("p", range(1, 9))
def test_filter_properties(p):
    h = wv.daubechies_lowpass(p)
    assert len(h) == 2 * p
    assert h.sum() == pytest.approx(math.sqrt(2), abs=1e-15)
    for s in range(p):
        ref = 1.0 if s == 0 else 0.0
        assert np.dot(h[: len(h) - 2 * s], h[2 * s:]) == pytest.approx(ref, abs=1e-15)
    # p vanishing moments of the wavelet: sum_j (-1)^j j^q h_j = 0 for q < p
    j = np.arange(2 * p, dtype=np.float64)
    for q in range(p):
        mom = np.sum((-1.0) ** j * j ** q * h)
        assert abs(mom) <= 1e-13 * max(1.0, np.sum(np.abs(j ** q * h)))


@pytest.mark.parametrize("p", range(1, 9))
@pytest.mark.parametrize("m", [2, 4, 8, 16, 64])
def test_level_matrix_orthogonal(p, m):
    W = wv.analysis_matrix(m, p)
    np.testing.assert_allclose(W @ W.T, np.eye(m), atol=1e-14)


@pytest.mark.parametrize("p", range(2, 9))
def test_detail_coefficients_vanish_on_polynomials(p):
    """Away from the periodic wrap, a polynomial of degree < p has zero detail."""
    m = 64
    W = wv.analysis_matrix(m, p)
    t = np.arange(m, dtype=np.float64) / m
    for q in range(p):
        d = W[m // 2:] @ (t ** q)
        inner = [k for k in range(m // 2) if 2 * k + 2 * p - 1 < m]
        assert np.max(np.abs(d[inner])) <= 1e-11


@pytest.mark.parametrize("p", [1, 4, 8])
def test_constant_image_mallat_layout(p):
    c = 0.7
    x = np.full((32, 64), c)
    out = wv.dwt2(x, p, 4)
    # each level multiplies a constant by sum(h)^2 = 2; after 4 levels LL = 16 c
    np.testing.assert_allclose(out[:2, :4], 16 * c, rtol=1e-13)
    rest = out.copy()
    rest[:2, :4] = 0
    assert np.max(np.abs(rest)) <= 1e-12


def test_frame_identities():
    rng = np.random.default_rng(3)
    x = rng.standard_normal((32, 32))
    a = wv.psi_adjoint(x, 4)
    assert a.shape == (9, 32, 32)
    np.testing.assert_allclose(wv.psi(a, 4), x, atol=1e-13)
    assert np.sum(a * a) == pytest.approx(np.sum(x * x), rel=1e-13)
    # adjointness: <Psi^dagger x, b> = <x, Psi b>
    b = rng.standard_normal((9, 32, 32))
    assert np.sum(a * b) == pytest.approx(np.sum(x * wv.psi(b, 4)), rel=1e-12)


def test_small_image_with_long_filters():
    """64 x 64 at 4 levels: level 4 works on 8 x 8 with db8 (length 16 > 8)."""
    rng = np.random.default_rng(4)
    x = rng.standard_normal((64, 64))
    for p in (7, 8):
        c = wv.dwt2(x, p, 4)
        np.testing.assert_allclose(wv.idwt2(c, p, 4), x, atol=1e-12)
        assert np.sum(c * c) == pytest.approx(np.sum(x * x), rel=1e-13)


def test_rectangular_and_cube():
    rng = np.random.default_rng(5)
    X = rng.standard_normal((3, 16, 32))
    A = wv.psi_adjoint_cube(X, 3)
    assert A.shape == (9, 3, 16, 32)
    np.testing.assert_allclose(wv.psi_cube(A, 3), X, atol=1e-13)
