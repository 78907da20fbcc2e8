"""Pins for the oracle's proximity operators (Sec. 3.3): closed forms on inputs
where the answer is known, the optimality conditions of each prox, and the
Moreau identity (Eq. "md") checked against the projection onto the dual-norm
ball computed by an independent route (eigendecomposition of the Gram matrix
instead of the SVD, explicit row clipping, explicit ball geometry)."""

import numpy as np
import pytest

from oracle import prox


def test_proj_positive():
    x = np.array([1.5 + 2j, -0.5 + 1j, 0.0 - 3j, 2.0])
    np.testing.assert_array_equal(prox.proj_positive(x), [1.5, 0.0, 0.0, 2.0])


def test_nuclear_on_diagonal_input():
    # cube (L=3, 1, 4): matrix N x L = 4 x 3 with singular values 5, 2, 0.5
    M = np.zeros((4, 3))
    M[0, 0], M[1, 1], M[2, 2] = 5.0, 2.0, 0.5
    X = M.T.reshape(3, 1, 4)
    out = prox.prox_nuclear(X, 1.0).reshape(3, 4).T
    ref = np.zeros((4, 3))
    ref[0, 0], ref[1, 1] = 4.0, 1.0
    np.testing.assert_allclose(out, ref, atol=1e-14)


def test_nuclear_rank_one_closed_form():
    rng = np.random.default_rng(1)
    u = rng.standard_normal(50)
    v = rng.standard_normal(4)
    X = np.outer(u, v).T.reshape(4, 5, 10)
    s = np.linalg.norm(u) * np.linalg.norm(v)
    out = prox.prox_nuclear(X, 0.3)
    np.testing.assert_allclose(out, X * (s - 0.3) / s, rtol=1e-12, atol=1e-13)


def _gram_clip(Z, w):
    """Projection onto {||.||_2 <= w} through eigh of the Gram matrix."""
    Mz = Z.reshape(Z.shape[0], -1).T
    lam, V = np.linalg.eigh(Mz.T @ Mz)
    s = np.sqrt(np.maximum(lam, 0))
    f = np.where(s > w, w / np.where(s > 0, s, 1), 1.0)
    return ((Mz @ V) * f) @ V.T


def test_nuclear_dual_is_spectral_ball_projection():
    rng = np.random.default_rng(2)
    Z = rng.standard_normal((5, 8, 8)) * 3
    out, s = prox.nuclear_dual(Z, 2.0)
    ref = _gram_clip(Z, 2.0)
    np.testing.assert_allclose(out.reshape(5, -1).T, ref, atol=1e-11)
    # Moreau: prox + dual prox = identity
    np.testing.assert_allclose(out + prox.prox_nuclear(Z, 2.0), Z, atol=1e-12)
    assert np.all(np.diff(s) <= 0)


def test_nuclear_optimality_condition():
    rng = np.random.default_rng(3)
    Z = rng.standard_normal((4, 6, 6)) * 4
    X = prox.prox_nuclear(Z, 1.0)
    Mx = X.reshape(4, -1).T
    Mz = Z.reshape(4, -1).T
    U, s, Vt = np.linalg.svd(Mx, full_matrices=False)
    r = int(np.sum(s > 1e-10))
    # Z - X = U_r V_r^T + W with ||W|| <= 1 and W orthogonal to the range of X
    D = Mz - Mx
    Ur, Vr = U[:, :r], Vt[:r].T
    W = D - Ur @ Vr.T
    assert np.linalg.norm(W, 2) <= 1.0 + 1e-10
    np.testing.assert_allclose(Ur.T @ W, 0, atol=1e-10)
    np.testing.assert_allclose(W @ Vr, 0, atol=1e-10)


def test_l21_rows_closed_form():
    A = np.zeros((2, 3, 1, 2))
    A[0, :, 0, 0] = [3.0, 4.0, 0.0]      # norm 5
    A[1, :, 0, 1] = [0.1, 0.0, 0.0]      # norm 0.1
    out = prox.prox_l21(A, 1.0, 2.0)
    np.testing.assert_allclose(out[0, :, 0, 0], [3.0 * 3 / 5, 4.0 * 3 / 5, 0.0])
    np.testing.assert_array_equal(out[1], 0.0)
    dual = prox.l21_dual(A, 1.0, 2.0)
    np.testing.assert_allclose(dual[0, :, 0, 0], [3.0 * 2 / 5, 4.0 * 2 / 5, 0.0])
    np.testing.assert_allclose(dual[1], A[1])
    # zero rows stay zero in both forms
    np.testing.assert_array_equal(out[0, :, 0, 1], 0.0)
    np.testing.assert_array_equal(dual[0, :, 0, 1], 0.0)


def test_l21_weights_and_moreau():
    rng = np.random.default_rng(4)
    Q = rng.standard_normal((9, 5, 4, 4))
    w = rng.uniform(0.0, 2.0, (9, 4, 4))
    thr = 0.8
    lam = thr * w
    dual = prox.l21_dual(Q, w, thr)
    # projection onto {||row_n|| <= lam_n}, row by row
    ref = np.empty_like(Q)
    for d in range(9):
        for i in range(4):
            for j in range(4):
                q = Q[d, :, i, j]
                n = np.linalg.norm(q)
                ref[d, :, i, j] = q if n <= lam[d, i, j] else q * lam[d, i, j] / n
    np.testing.assert_allclose(dual, ref, rtol=1e-14, atol=1e-15)
    np.testing.assert_allclose(dual + prox.prox_l21(Q, w, thr), Q, atol=1e-14)


def test_l2ball_projection_geometry():
    rng = np.random.default_rng(5)
    y = rng.standard_normal(40) + 1j * rng.standard_normal(40)
    z_in = y + 0.01 * (rng.standard_normal(40) + 1j * rng.standard_normal(40))
    z_out = y + 3.0 * (rng.standard_normal(40) + 1j * rng.standard_normal(40))
    eps = 1.0
    np.testing.assert_array_equal(prox.proj_l2ball(z_in, y, eps), z_in)
    p = prox.proj_l2ball(z_out, y, eps)
    assert np.linalg.norm(p - y) == pytest.approx(eps, rel=1e-14)
    # same direction from the centre, and idempotent
    d0 = (z_out - y) / np.linalg.norm(z_out - y)
    np.testing.assert_allclose((p - y) / eps, d0, atol=1e-14)
    np.testing.assert_allclose(prox.proj_l2ball(p, y, eps), p, atol=1e-14)
    # Moreau: dual form + projection = identity
    np.testing.assert_allclose(prox.l2ball_dual(z_out, y, eps) + p, z_out, atol=1e-14)


def test_l2ball_dual_with_preconditioner():
    rng = np.random.default_rng(6)
    M = 30
    y = rng.standard_normal(M) + 1j * rng.standard_normal(M)
    vbar = 4 * (rng.standard_normal(M) + 1j * rng.standard_normal(M))
    U = rng.uniform(0.2, 3.0, M)
    eps = 0.5
    v = prox.l2ball_dual(vbar, y, eps, U)
    z = vbar / np.sqrt(U)
    d = z - y
    ref = np.sqrt(U) * d * max(0.0, 1 - eps / np.linalg.norm(d))
    np.testing.assert_allclose(v, ref, atol=1e-13)


def test_l1_prox_and_dual_closed_forms_and_moreau():
    """Soft thresholding (SARA prior): known values, and prox + dual = identity."""
    q = np.array([[-3.0, -0.5, 0.0, 0.2, 2.5]])
    w = np.array([[1.0, 1.0, 2.0, 0.1, 0.5]])
    np.testing.assert_array_equal(prox.prox_l1(q, w, 1.0), [[-2.0, 0.0, 0.0, 0.1, 2.0]])
    np.testing.assert_array_equal(prox.l1_dual(q, w, 1.0), [[-1.0, -0.5, 0.0, 0.1, 0.5]])
    rng = np.random.default_rng(8)
    Q = rng.standard_normal((9, 3, 8, 8))
    W = rng.uniform(0.1, 2.0, Q.shape)
    np.testing.assert_allclose(prox.prox_l1(Q, W, 0.7) + prox.l1_dual(Q, W, 0.7), Q, rtol=0, atol=1e-15)
    # the l1 prox is the minimiser of 0.5 ||a - q||^2 + thr sum w |a|: check optimality per entry
    A = prox.prox_l1(Q, W, 0.7)
    g = A - Q
    nz = A != 0
    np.testing.assert_allclose(g[nz], -0.7 * W[nz] * np.sign(A[nz]), rtol=0, atol=1e-14)
    assert np.all(np.abs(g[~nz]) <= 0.7 * W[~nz] + 1e-15)
