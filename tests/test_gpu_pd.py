"""GPU parity of the primal-dual iteration (Algorithm 2) against the oracle.

FP64 plans follow the oracle's iterates to ~1e-12 per step; FP32 plans must
reach the oracle's reconstruction quality: aSNR within 0.05 dB after the
configuration's iteration count. Parameters (mu, kappa_3) are computed by the
oracle and passed to both sides so the two runs solve the same problem."""

import numpy as np
import pytest

import synth
from gpu_util import dev, host, rel
from oracle import metrics, pd, problem

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built(cuda_device):
    import __graft_entry__ as ge
    ge.build()


def _setup(inp, prec, levels=4, U=None):
    """Oracle problem on the inputs rounded to `prec`."""
    if prec == "f32":
        inp.uv = inp.uv.astype(np.float32).astype(np.float64)
        inp.truth = inp.truth.astype(np.float32).astype(np.float64)
    prob = problem.make_problem(inp)
    if prec == "f32":
        prob.y = prob.y.astype(np.complex64).astype(np.complex128)
    mu = problem.estimate_mu(prob.op, prob.y, levels)
    k3 = 1.0 / problem.op_norm2(prob.op, U=U, iters=300, tol=1e-9)
    prm = pd.PDParams(mu=mu, tau=0.33, kappa3=k3, levels=levels)
    return prob, prm


def _gpu_state(inp, prob, prm, prec, U=None, use_nuclear=True, use_l21=True, compensated=False):
    import torch
    from paper_1806_04596_gb300 import hypersara as hs
    plan = hs.Plan(inp.nx, inp.ny, inp.offsets, dev(inp.uv, prec),
                   precond=None if U is None else dev(U, prec), levels=prm.levels, prec=prec,
                   compensated=compensated)
    st = hs.PDState(plan, dev(prob.y, prec, True), torch.tensor(prob.eps, dtype=torch.float64,
                                                                device="cuda"),
                    tau=prm.tau, kappa1=prm.kappa1, kappa2=prm.kappa2, kappa3=prm.kappa3, mu=prm.mu,
                    use_nuclear=use_nuclear, use_l21=use_l21)
    return plan, st


def test_pd_fp64_tracks_oracle_c1():
    """Configuration 1 (64 x 64, L = 4, M = 2000, FP64, 200 iterations)."""
    inp = synth.make_inputs(1)
    prob, prm = _setup(inp, "f64")
    plan, st = _gpu_state(inp, prob, prm, "f64")
    ref = pd.init_state(inp.L, inp.ny, inp.nx, int(inp.offsets[-1]))
    done = 0
    for k in (1, 4, 45, 150):
        ref = pd.pd_solve(prob.op, prob.y, prob.eps, prm, k, state=ref)
        st.solve(k, graph=(done > 0))
        done += k
        X, beta, rho = st.get()
        Xg = host(X)
        e = rel(Xg, ref.X)
        assert e <= 1e-12 * max(1.0, done / 10), (done, e)
        assert beta == pytest.approx(ref.beta, rel=1e-9)
        np.testing.assert_allclose(rho, ref.rho, rtol=1e-10)
    assert abs(metrics.asnr(prob.truth, Xg) - metrics.asnr(prob.truth, ref.X)) < 1e-6


def test_pd_fp32_matches_oracle_snr_c1():
    inp = synth.make_inputs(1)
    prob, prm = _setup(inp, "f32")
    ref = pd.pd_solve(prob.op, prob.y, prob.eps, prm, 200)
    plan, st = _gpu_state(inp, prob, prm, "f32")
    st.solve(200, graph=True)
    X, beta, rho = st.get()
    Xg = host(X)
    a_gpu = metrics.asnr(prob.truth, Xg)
    a_ref = metrics.asnr(prob.truth, ref.X)
    assert abs(a_gpu - a_ref) <= 0.05, (a_gpu, a_ref)
    assert rel(Xg, ref.X) <= 1e-3


def test_pd_graph_equals_eager():
    """Every gridding form sums in a fixed order, so the replayed graph
    reproduces the eager launches bitwise, for the compensated tiles and for the
    default register sweep; the two forms agree to FP32 rounding."""
    inp = synth.make_inputs(1, n=64, L=3, M=(800, 1500), seed=77)
    prob, prm = _setup(inp, "f32")
    _, s1 = _gpu_state(inp, prob, prm, "f32", compensated=True)
    _, s2 = _gpu_state(inp, prob, prm, "f32", compensated=True)
    s1.solve(7, graph=True)
    s2.solve(7, graph=False)
    a = host(s1.get()[0])
    b = host(s2.get()[0])
    assert np.array_equal(a, b)
    _, s3 = _gpu_state(inp, prob, prm, "f32")
    _, s4 = _gpu_state(inp, prob, prm, "f32")
    s3.solve(7, graph=True)
    s4.solve(7, graph=False)
    c = host(s3.get()[0])
    assert np.array_equal(c, host(s4.get()[0]))
    assert rel(c, a) <= 1e-5


def test_pd_fp64_with_preconditioner_and_priors_off():
    inp = synth.make_inputs(1, n=32, L=3, M=(300, 700), seed=78)
    U = np.random.default_rng(9).uniform(0.3, 2.0, int(inp.offsets[-1]))
    prob, prm = _setup(inp, "f64", levels=3, U=U)
    plan, st = _gpu_state(inp, prob, prm, "f64", U=U)
    ref = pd.pd_solve(prob.op, prob.y, prob.eps, prm, 12, U=U)
    st.solve(12, graph=False)
    assert rel(host(st.get()[0]), ref.X) <= 1e-11
    for nuc, l21 in ((False, True), (True, False), (False, False)):
        import dataclasses
        prm2 = dataclasses.replace(prm, use_nuclear=nuc, use_l21=l21)
        ref = pd.pd_solve(prob.op, prob.y, prob.eps, prm2, 6, U=U)
        _, st2 = _gpu_state(inp, prob, prm2, "f64", U=U, use_nuclear=nuc, use_l21=l21)
        st2.solve(6, graph=True)
        assert rel(host(st2.get()[0]), ref.X) <= 1e-11, (nuc, l21)


def test_pd_fp32_c2_shape_reduced_channels():
    """Configuration 2's generator (256 x 256, M = 32768 per channel, FP32) on
    4 of its 60 channels, 20 iterations."""
    inp = synth.make_inputs(2, L=4)
    prob, prm = _setup(inp, "f32")
    ref = pd.pd_solve(prob.op, prob.y, prob.eps, prm, 20)
    _, st = _gpu_state(inp, prob, prm, "f32")
    st.solve(20, graph=True)
    Xg = host(st.get()[0])
    assert rel(Xg, ref.X) <= 1e-4
    assert abs(metrics.asnr(prob.truth, Xg) - metrics.asnr(prob.truth, ref.X)) <= 0.05


def test_pd_fp64_holed_coverage():
    """Configuration 1's generator with 20 holes in the uv coverage (Sec. 4.1),
    FP64, 30 iterations."""
    inp = synth.make_inputs(1, holes=20)
    prob, prm = _setup(inp, "f64")
    ref = pd.pd_solve(prob.op, prob.y, prob.eps, prm, 30)
    _, st = _gpu_state(inp, prob, prm, "f64")
    st.solve(30, graph=True)
    assert rel(host(st.get()[0]), ref.X) <= 1e-11
