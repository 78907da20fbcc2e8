"""Pins for the oracle's data blocks (M_l^b, Sec. 2.1) and adaptive l2 bounds
(Algorithm 2 steps 13-19, Sec. 3.6).

* One block per channel is the plain iteration.
* From the zero state the first dual update of block b is the closed form
  v_b = -y_b max(0, 1 - eps_b / ||y_b||) (vbar = 0): each block is projected on
  its own ball, with its own bound.
* The residual reported per block is ||y_b - Phi_b X~|| at the image the
  iteration used.
* Adaptive bounds: lambda_1 = 0 (beta never below it) leaves the run identical
  to fixed bounds; when every condition holds the bound moves to
  lambda_3 rho + (1 - lambda_3) eps and vartheta records the iteration; the
  first iteration never adjusts (beta^{(0)} undefined); a block adjusted at t is
  not adjusted again before t + vartheta_bar + 1."""

import dataclasses

import numpy as np
import pytest

import synth
from oracle import pd, problem


def _setup(seed=61, n=16, L=2, M=(260, 300)):
    inp = synth.make_inputs(1, n=n, L=L, M=M, seed=seed)
    prob = problem.make_problem(inp)
    prm = pd.PDParams(mu=problem.estimate_mu(prob.op, prob.y, 2), levels=2,
                      kappa3=1.0 / problem.op_norm2(prob.op, iters=200, tol=1e-9))
    # three blocks in channel 0, two in channel 1 (contiguous caller ranges)
    o = prob.op.offsets
    blocks = np.array([0, 100, 210, o[1], o[1] + 130, o[2]])
    return inp, prob, prm, blocks


def test_one_block_per_channel_is_the_plain_iteration():
    inp, prob, prm, _ = _setup()
    a = pd.pd_solve(prob.op, prob.y, prob.eps, prm, 6)
    b = pd.pd_solve(prob.op, prob.y, prob.eps, prm, 6, blocks=prob.op.offsets)
    assert np.array_equal(a.X, b.X) and np.array_equal(a.v, b.v)


def test_first_dual_update_per_block_closed_form():
    inp, prob, prm, blocks = _setup()
    ynb = np.array([np.linalg.norm(prob.y[blocks[k]:blocks[k + 1]]) for k in range(5)])
    eps = ynb * np.array([0.3, 0.9, 1.5, 0.5, 0.1])     # block 2 contains the origin: v = 0
    st = pd.pd_step(pd.init_state(2, 16, 16, int(prob.op.offsets[-1])), prob.op, prob.y, eps, prm,
                    blocks=blocks)
    for k in range(5):
        a, b = blocks[k], blocks[k + 1]
        want = -prob.y[a:b] * max(0.0, 1.0 - eps[k] / ynb[k])
        np.testing.assert_allclose(st.v[a:b], want, rtol=1e-13, atol=1e-15)
        assert st.resid[k] == pytest.approx(ynb[k], rel=1e-13)   # X~ = 0


def test_adaptive_with_unreachable_lambda1_changes_nothing():
    inp, prob, prm, blocks = _setup()
    eps = np.full(5, 0.01)
    a = pd.pd_solve(prob.op, prob.y, eps, prm, 8, blocks=blocks)
    b = pd.pd_solve(prob.op, prob.y, eps, prm, 8, blocks=blocks,
                    adapt=pd.AdaptParams(lambda1=0.0, min_gap=0))
    assert np.array_equal(a.X, b.X)
    np.testing.assert_array_equal(b.eps, eps)


def test_adaptive_update_rule_and_gap():
    inp, prob, prm, blocks = _setup()
    eps0 = np.full(5, 1e-3)                               # far below the residuals: every block adjusts
    ad = pd.AdaptParams(lambda1=1e9, lambda2=0.01, lambda3=0.618, min_gap=2)
    st = pd.init_state(2, 16, 16, int(prob.op.offsets[-1]))
    st = pd.pd_step(st, prob.op, prob.y, eps0, prm, blocks=blocks, adapt=ad)
    np.testing.assert_array_equal(st.eps, eps0)            # t = 1: beta^{(0)} undefined
    st1 = st
    st = pd.pd_step(st, prob.op, prob.y, eps0, prm, blocks=blocks, adapt=ad)   # t = 2: 2 - 0 > 2 false
    np.testing.assert_array_equal(st.eps, eps0)
    st = pd.pd_step(st, prob.op, prob.y, eps0, prm, blocks=blocks, adapt=ad)   # t = 3: adjusts
    want = 0.618 * st.resid + (1 - 0.618) * eps0
    np.testing.assert_allclose(st.eps, want, rtol=1e-15)
    assert np.all(st.theta == 3)
    e3 = st.eps.copy()
    for t in (4, 5):                                       # within the gap: unchanged
        st = pd.pd_step(st, prob.op, prob.y, eps0, prm, blocks=blocks, adapt=ad)
        np.testing.assert_array_equal(st.eps, e3)
    st = pd.pd_step(st, prob.op, prob.y, eps0, prm, blocks=blocks, adapt=ad)   # t = 6: 6 - 3 > 2
    moved = np.abs(st.resid - e3) / e3 > 0.01
    np.testing.assert_allclose(st.eps[moved], 0.618 * st.resid[moved] + 0.382 * e3[moved], rtol=1e-15)
    assert np.all(st.theta[moved] == 6)
    assert st1.t == 1
