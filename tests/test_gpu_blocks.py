"""GPU parity of intra-channel data blocks (M_l^b, Sec. 2.1) and the adaptive
l2 bounds (Algorithm 2 steps 13-19, Sec. 3.6) against the oracle."""

import numpy as np
import pytest

import synth
from gpu_util import dev, host, rel
from oracle import pd, problem

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built(cuda_device):
    import __graft_entry__ as ge
    ge.build()


def _setup(prec, seed=61, n=32, L=3, M=(500, 700)):
    inp = synth.make_inputs(1, n=n, L=L, M=M, seed=seed)
    if prec == "f32":
        inp.uv = inp.uv.astype(np.float32).astype(np.float64)
        inp.truth = inp.truth.astype(np.float32).astype(np.float64)
    prob = problem.make_problem(inp)
    if prec == "f32":
        prob.y = prob.y.astype(np.complex64).astype(np.complex128)
    prm = pd.PDParams(mu=problem.estimate_mu(prob.op, prob.y, 3), levels=3,
                      kappa3=1.0 / problem.op_norm2(prob.op, iters=300, tol=1e-9))
    o = prob.op.offsets
    # uneven blocks: three in channel 0, one in channel 1, two in channel 2 (one of them empty)
    blocks = np.array([0, 120, 333, o[1], o[2], o[2] + 200, o[3], o[3]])
    return inp, prob, prm, blocks


def _state(inp, prob, prm, prec, blocks, eps):
    import torch
    from paper_1806_04596_gb300 import hypersara as hs
    plan = hs.Plan(inp.nx, inp.ny, inp.offsets, dev(inp.uv, prec), levels=prm.levels, prec=prec, blocks=blocks)
    st = hs.PDState(plan, dev(prob.y, prec, True), torch.tensor(eps, dtype=torch.float64, device="cuda"),
                    tau=prm.tau, kappa3=prm.kappa3, mu=prm.mu)
    return plan, st


def _block_eps(prob, blocks, frac):
    return np.array([frac * np.linalg.norm(prob.y[blocks[k]:blocks[k + 1]]) + 1e-3
                     for k in range(len(blocks) - 1)])


@pytest.mark.parametrize("prec,tol", [("f64", 1e-11), ("f32", 1e-4)])
def test_blocks_track_oracle(prec, tol):
    inp, prob, prm, blocks = _setup(prec)
    eps = _block_eps(prob, blocks, 0.2)
    plan, st = _state(inp, prob, prm, prec, blocks, eps)
    assert plan.info["nblocks"] == len(blocks) - 1
    st.solve(20, graph=True)
    X, beta, rho = st.get()
    ref = pd.pd_solve(prob.op, prob.y, eps, prm, 20, blocks=blocks)
    assert rel(host(X), ref.X) <= tol
    np.testing.assert_allclose(rho, ref.rho, rtol=100 * tol, atol=1e-12)


@pytest.mark.parametrize("prec,tol", [("f64", 1e-11), ("f32", 1e-4)])
def test_adaptive_bounds_track_oracle(prec, tol):
    """Under-estimated bounds that every block adjusts, twice, with a 3-iteration gap."""
    inp, prob, prm, blocks = _setup(prec)
    eps = _block_eps(prob, blocks, 0.01)
    plan, st = _state(inp, prob, prm, prec, blocks, eps)
    st.set_adaptive(True, lambda1=1e9, lambda2=0.01, lambda3=0.618, min_gap=3)
    st.solve(12, graph=True)
    ad = pd.AdaptParams(lambda1=1e9, lambda2=0.01, lambda3=0.618, min_gap=3)
    ref = pd.pd_solve(prob.op, prob.y, eps, prm, 12, blocks=blocks, adapt=ad)
    e, r, t = st.bounds()
    assert rel(host(st.get()[0]), ref.X) <= tol
    np.testing.assert_array_equal(t, ref.theta)
    assert np.any(ref.theta > 0)
    np.testing.assert_allclose(e, ref.eps, rtol=100 * tol)
    np.testing.assert_allclose(r, ref.resid, rtol=100 * tol, atol=1e-12)


def test_adaptive_off_equals_fixed_bounds():
    inp, prob, prm, blocks = _setup("f64")
    eps = _block_eps(prob, blocks, 0.2)
    _, s1 = _state(inp, prob, prm, "f64", blocks, eps)
    _, s2 = _state(inp, prob, prm, "f64", blocks, eps)
    s2.set_adaptive(True, lambda1=0.0)          # beta is never below 0: no update
    s1.solve(8, graph=True)
    s2.solve(8, graph=True)
    assert np.array_equal(host(s1.get()[0]), host(s2.get()[0]))
    np.testing.assert_array_equal(s2.bounds()[0], eps)


def test_block_offsets_are_validated():
    from paper_1806_04596_gb300 import hypersara as hs
    inp, prob, prm, blocks = _setup("f64")
    bad = np.delete(blocks, 3)                   # drops the boundary of channel 1
    with pytest.raises(hs.HSError):
        hs.Plan(inp.nx, inp.ny, inp.offsets, dev(inp.uv, "f64"), levels=3, prec="f64", blocks=bad)
