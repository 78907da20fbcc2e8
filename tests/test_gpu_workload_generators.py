"""Parity on the generators of the other workloads at reduced sizes (the full
sizes are measured by bench.py --config 3 / 5):

* the 2048^2, L = 64, 1-4 GHz, M_l ~ U[5e5, 2e6] generator at 256^2, L = 6,
  M_l ~ U[5e3, 2e4]: FP64 PD iterations and one re-weighting step (Algorithm 1)
  against the oracle, FP32 within the FP32 tolerance of the oracle;
* the 512^2, L = 32, M_l ~ U[1e5, 4e5] generator at 128^2, L = 4,
  M_l ~ U[2e3, 8e3]: the objective gradient against the oracle's;
* mu and eta_l from the library (hs_estimate_mu) against the oracle's."""

import numpy as np
import pytest

import synth
from gpu_util import dev, host, rel
from oracle import grad as ograd
from oracle import pd, problem, reweight

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built(cuda_device):
    import __graft_entry__ as ge
    ge.build()


def _c5_small():
    inp = synth.make_inputs(5, n=256, L=6, M=(5000, 20000))
    prob = problem.make_problem(inp)
    return inp, prob


@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_c5_generator_pd_and_reweight(prec):
    import torch
    from paper_1806_04596_gb300 import hypersara as hs
    inp, prob = _c5_small()
    assert len(set(np.diff(inp.offsets))) > 1 and inp.freqs[-1] == pytest.approx(4.0)
    uv = inp.uv if prec == "f64" else inp.uv.astype(np.float32).astype(np.float64)
    y = prob.y if prec == "f64" else prob.y.astype(np.complex64).astype(np.complex128)
    op = problem.nufft.WidebandOperator(inp.nx, inp.ny, uv, inp.offsets)
    mu = problem.estimate_mu(op, y, 4)
    k3 = 1.0 / problem.op_norm2(op, iters=200, tol=1e-9)
    prm = pd.PDParams(mu=mu, tau=0.33, kappa3=k3, levels=4)
    plan = hs.Plan(inp.nx, inp.ny, inp.offsets, dev(uv, prec), levels=4, prec=prec)
    w21 = torch.ones((9, inp.ny, inp.nx), dtype=plan.rdtype, device="cuda")
    wnu = torch.ones(inp.L, dtype=torch.float64, device="cuda")
    st = hs.PDState(plan, dev(y, prec, True), torch.tensor(prob.eps, dtype=torch.float64, device="cuda"),
                    tau=0.33, kappa3=k3, mu=mu, w_nuc=wnu, w_l21=w21)
    st.solve(8, graph=True)
    ref = pd.pd_solve(op, y, prob.eps, prm, 8)
    X, beta, rho = st.get()
    tol = 1e-10 if prec == "f64" else 1e-4
    assert rel(host(X), ref.X) <= tol
    np.testing.assert_allclose(rho, ref.rho, rtol=tol)
    # one re-weighting step (Algorithm 1) from the same primal, then 4 more iterations
    st.reweight(1.0, 1.0, w21, wnu)
    Xg = host(X)   # the weights of the library's own primal, computed by the oracle
    assert rel(host(w21), reweight.weights_l21(Xg, 4, 1.0)) <= (1e-10 if prec == "f64" else 1e-5)
    assert rel(host(wnu), reweight.weights_nuclear(Xg, 1.0)) <= (1e-10 if prec == "f64" else 1e-5)
    # continue with the weights the library uses (those of its own primal); FP32
    # iterates drift from the FP64 ones by a few 1e-4 after a dozen iterations
    w_rows, w_sv = reweight.weights_l21(Xg, 4, 1.0), reweight.weights_nuclear(Xg, 1.0)
    prm2 = pd.PDParams(mu=mu, tau=0.33, kappa3=k3, levels=4, w_nuc=w_sv, w_l21=w_rows)
    st.solve(4, graph=True)
    ref2 = pd.pd_solve(op, y, prob.eps, prm2, 4, state=ref)
    X2, _, _ = st.get()
    assert rel(host(X2), ref2.X) <= (1e-10 if prec == "f64" else 5e-4)


@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_c3_generator_objective_gradient(prec):
    from paper_1806_04596_gb300 import autograd as ag
    from paper_1806_04596_gb300 import hypersara as hs
    import torch
    inp = synth.make_inputs(3, n=128, L=4, M=(2000, 8000))
    prob = problem.make_problem(inp)
    uv = inp.uv if prec == "f64" else inp.uv.astype(np.float32).astype(np.float64)
    y = prob.y if prec == "f64" else prob.y.astype(np.complex64).astype(np.complex128)
    X = np.random.default_rng(3).uniform(0, 1, inp.truth.shape)
    if prec == "f32":
        X = X.astype(np.float32).astype(np.float64)
    op = problem.nufft.WidebandOperator(inp.nx, inp.ny, uv, inp.offsets)
    plan = hs.Plan(inp.nx, inp.ny, inp.offsets, dev(uv, prec), levels=4, prec=prec)
    Xt = dev(X, prec).requires_grad_(True)
    (g,) = torch.autograd.grad(ag.objective(plan, Xt, dev(y, prec, True)), Xt)
    assert rel(host(g), ograd.gradient(op, X, y, 4)) <= (1e-10 if prec == "f64" else 2e-5)


@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_estimate_mu_matches_oracle(prec):
    from paper_1806_04596_gb300 import hypersara as hs
    inp = synth.make_inputs(1, n=64, L=4, M=(800, 2500))
    prob = problem.make_problem(inp)
    uv = inp.uv if prec == "f64" else inp.uv.astype(np.float32).astype(np.float64)
    y = prob.y if prec == "f64" else prob.y.astype(np.complex64).astype(np.complex128)
    op = problem.nufft.WidebandOperator(inp.nx, inp.ny, uv, inp.offsets)
    plan = hs.Plan(inp.nx, inp.ny, inp.offsets, dev(uv, prec), levels=4, prec=prec)
    mu, eta, Xd = plan.estimate_mu(dev(y, prec, True))
    tol = 1e-10 if prec == "f64" else 1e-5
    assert mu == pytest.approx(problem.estimate_mu(op, y, 4), rel=tol)
    np.testing.assert_allclose(host(eta), problem.psf_peak_norm(op), rtol=tol)
    assert rel(host(Xd), problem.dirty_cube(op, y)) <= tol
