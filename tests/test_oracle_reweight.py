"""Pins for the oracle's re-weighting loop (Algorithm 1, Eqs. "weights-l21" and
"weights-n") by closed forms and invariants that do not go through the weight
functions' own formulas:

* zero image: every weight is exactly 1;
* rank-one cube X_l = a_l B: one singular value ||a|| ||B||_F, the rest 0;
* a single bright pixel: its Dirac row is ||a|| / 3, and with one level of the
  Haar basis the four subband rows at that position are ||a|| / 6;
* tight frame: the squared row norms recovered from the weights sum to ||X||_F^2;
* one outer iteration is the plain PD solve with unit weights, and the weights
  after the second use the decayed gammas."""

import dataclasses

import numpy as np
import pytest

import synth
from oracle import pd, problem, reweight


def test_zero_image_gives_unit_weights():
    X = np.zeros((3, 16, 16))
    assert np.array_equal(reweight.weights_l21(X, 2, 0.7), np.ones((9, 16, 16)))
    assert np.array_equal(reweight.weights_nuclear(X, 0.3), np.ones(3))


def test_rank_one_cube_nuclear_weights():
    rng = np.random.default_rng(3)
    a = rng.uniform(0.5, 2.0, 4)
    B = rng.standard_normal((16, 16))
    X = a[:, None, None] * B[None]
    g = 0.6
    w = reweight.weights_nuclear(X, g)
    s1 = np.linalg.norm(a) * np.linalg.norm(B)
    assert w[0] == pytest.approx(g / (g + s1), rel=1e-12)
    np.testing.assert_allclose(w[1:], 1.0, atol=1e-12)


def test_single_pixel_dirac_and_haar_rows():
    a = np.array([0.3, 1.2, 0.7])
    X = np.zeros((3, 16, 16))
    X[:, 6, 10] = a                       # even (row, column): the pixel starts a 2 x 2 Haar block
    g = 0.9
    w = reweight.weights_l21(X, 1, g)
    na = np.linalg.norm(a)
    assert w[0, 6, 10] == pytest.approx(g / (g + na / 3), rel=1e-13)
    mask = np.ones((16, 16), bool)
    mask[6, 10] = False
    assert np.all(w[0][mask] == 1.0)
    # Haar (basis 1), one level, Mallat layout: LL at (3, 5), details at (3, 13), (11, 5), (11, 13)
    for (r, c) in [(3, 5), (3, 13), (11, 5), (11, 13)]:
        assert w[1, r, c] == pytest.approx(g / (g + na / 6), rel=1e-12), (r, c)


def test_row_norms_from_weights_obey_the_tight_frame():
    rng = np.random.default_rng(5)
    X = rng.uniform(0.0, 1.0, (4, 32, 32))
    g = 0.45
    w = reweight.weights_l21(X, 3, g)
    rows = g * (1.0 / w - 1.0)
    assert np.sum(rows ** 2) == pytest.approx(np.sum(X ** 2), rel=1e-11)
    assert np.all((w > 0) & (w <= 1))


def test_outer_loop_structure():
    inp = synth.make_inputs(1, n=16, L=3, M=150, seed=41)
    prob = problem.make_problem(inp)
    prm = pd.PDParams(mu=problem.estimate_mu(prob.op, prob.y, 2), levels=2,
                      kappa3=1.0 / problem.op_norm2(prob.op, iters=200, tol=1e-9))
    st1, w21, wn = reweight.reweighted_solve(prob.op, prob.y, prob.eps, prm, outer=1, inner=5)
    ref = pd.pd_solve(prob.op, prob.y, prob.eps, prm, 5)
    assert np.array_equal(st1.X, ref.X)
    np.testing.assert_allclose(wn, reweight.weights_nuclear(ref.X, 1.0), rtol=0, atol=0)
    # second outer iteration: runs with the first weights, then weights with gamma = decay
    st2, w21b, wnb = reweight.reweighted_solve(prob.op, prob.y, prob.eps, prm, outer=2, inner=5, decay=0.5)
    ref2 = pd.pd_solve(prob.op, prob.y, prob.eps, dataclasses.replace(prm, w_l21=w21, w_nuc=wn), 5, state=ref)
    np.testing.assert_allclose(st2.X, ref2.X, rtol=0, atol=1e-15)
    s = np.linalg.svd(ref2.X.reshape(3, -1).T, compute_uv=False)
    np.testing.assert_allclose(wnb, 0.5 / (0.5 + s), rtol=1e-12)


def test_l1_weights_single_pixel():
    """SARA weights are per coefficient: the bright pixel's Dirac coefficient of
    channel l is a_l / 3."""
    a = np.array([0.3, 1.2])
    X = np.zeros((2, 16, 16))
    X[:, 4, 4] = a
    w = reweight.weights_l1(X, 1, 0.5)
    np.testing.assert_allclose(w[0, :, 4, 4], 0.5 / (0.5 + a / 3), rtol=1e-13)
    assert w.shape == (9, 2, 16, 16) and np.all(w[0, :, 0, 0] == 1.0)
