"""GPU parity of the re-weighting outer loop (Algorithm 1): the weights of
hs_pd_reweight against the oracle's from the same primal cube, and the whole
re-weighted solve (FP64) against the oracle's."""

import numpy as np
import pytest

import synth
from gpu_util import dev, host, rel
from oracle import pd, problem, reweight

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built(cuda_device):
    import __graft_entry__ as ge
    ge.build()


def _problem(prec, n=32, L=4, M=(600, 800), seed=91, levels=3):
    inp = synth.make_inputs(1, n=n, L=L, M=M, seed=seed)
    if prec == "f32":
        inp.uv = inp.uv.astype(np.float32).astype(np.float64)
        inp.truth = inp.truth.astype(np.float32).astype(np.float64)
    prob = problem.make_problem(inp)
    if prec == "f32":
        prob.y = prob.y.astype(np.complex64).astype(np.complex128)
    mu = problem.estimate_mu(prob.op, prob.y, levels)
    k3 = 1.0 / problem.op_norm2(prob.op, iters=300, tol=1e-9)
    prm = pd.PDParams(mu=mu, tau=0.33, kappa3=k3, levels=levels)
    return inp, prob, prm


def _state(inp, prob, prm, prec):
    import torch
    from paper_1806_04596_gb300 import hypersara as hs
    plan = hs.Plan(inp.nx, inp.ny, inp.offsets, dev(inp.uv, prec), levels=prm.levels, prec=prec)
    rt = torch.float32 if prec == "f32" else torch.float64
    w_l21 = torch.ones((9, inp.ny, inp.nx), dtype=rt, device="cuda")
    w_nuc = torch.ones(inp.L, dtype=torch.float64, device="cuda")
    st = hs.PDState(plan, dev(prob.y, prec, True), torch.tensor(prob.eps, dtype=torch.float64, device="cuda"),
                    tau=prm.tau, kappa3=prm.kappa3, mu=prm.mu, w_nuc=w_nuc, w_l21=w_l21)
    return plan, st, w_l21, w_nuc


@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_reweight_weights_match_oracle(prec):
    import torch
    inp, prob, prm = _problem(prec)
    plan, st, w_l21, w_nuc = _state(inp, prob, prm, prec)
    st.solve(30, graph=True)
    X = host(st.get()[0])
    sv = torch.empty(inp.L, dtype=torch.float64, device="cuda")
    st.reweight(0.7, 0.6, w_l21, w_nuc, sv)
    ref_l21 = reweight.weights_l21(X, prm.levels, 0.7)
    ref_nuc = reweight.weights_nuclear(X, 0.6)
    ref_sv = np.linalg.svd(X.reshape(inp.L, -1).T, compute_uv=False)
    if prec == "f64":
        assert rel(host(w_l21), ref_l21) <= 1e-12
        np.testing.assert_allclose(host(sv), ref_sv, rtol=1e-10, atol=1e-12 * ref_sv[0])
        np.testing.assert_allclose(host(w_nuc), ref_nuc, rtol=1e-10)
    else:
        assert rel(host(w_l21), ref_l21) <= 2e-6
        np.testing.assert_allclose(host(sv), ref_sv, rtol=1e-5, atol=1e-3 * ref_sv[0])
        np.testing.assert_allclose(host(w_nuc), ref_nuc, rtol=0, atol=1e-4)


def test_reweight_rejects_bad_gamma():
    inp, prob, prm = _problem("f64", n=16, L=2, M=(100, 120))
    plan, st, w_l21, w_nuc = _state(inp, prob, prm, "f64")
    from paper_1806_04596_gb300 import hypersara as hs
    with pytest.raises(hs.HSError):
        st.reweight(0.0, 1.0, w_l21, w_nuc)
    with pytest.raises(hs.HSError):
        st.reweight(1.0, float("nan"), w_l21, w_nuc)


def test_reweighted_solve_tracks_oracle_fp64():
    from paper_1806_04596_gb300 import hypersara as hs
    inp, prob, prm = _problem("f64")
    plan, st, w_l21, w_nuc = _state(inp, prob, prm, "f64")
    hs.reweighted_solve(st, outer=3, inner=10, decay=0.8, graph=True)
    ref, r21, rnuc = reweight.reweighted_solve(prob.op, prob.y, prob.eps, prm, outer=3, inner=10, decay=0.8)
    assert rel(host(st.get()[0]), ref.X) <= 1e-11
    assert rel(host(w_l21), r21) <= 1e-11
    np.testing.assert_allclose(host(w_nuc), rnuc, rtol=1e-9)


def _sara_state(inp, prob, prm, prec, weights=False):
    import torch
    from paper_1806_04596_gb300 import hypersara as hs
    plan = hs.Plan(inp.nx, inp.ny, inp.offsets, dev(inp.uv, prec), levels=prm.levels, prec=prec)
    rt = torch.float32 if prec == "f32" else torch.float64
    w = torch.ones((9, inp.L, inp.ny, inp.nx), dtype=rt, device="cuda") if weights else None
    st = hs.PDState(plan, dev(prob.y, prec, True), torch.tensor(prob.eps, dtype=torch.float64, device="cuda"),
                    tau=prm.tau, kappa3=prm.kappa3, mu=prm.mu, use_nuclear=False, w_l21=w, sparsity="l1")
    return plan, st, w


@pytest.mark.parametrize("prec,tol", [("f64", 1e-11), ("f32", 1e-4)])
def test_sara_variant_tracks_oracle(prec, tol):
    """SARA (Sec. 4.2): per-channel l1 prior, no nuclear term."""
    import dataclasses
    inp, prob, prm = _problem(prec)
    prm = dataclasses.replace(prm, use_nuclear=False, sparsity="l1")
    plan, st, _ = _sara_state(inp, prob, prm, prec)
    st.solve(20, graph=True)
    ref = pd.pd_solve(prob.op, prob.y, prob.eps, prm, 20)
    assert rel(host(st.get()[0]), ref.X) <= tol


def test_sara_reweighted_fp64():
    import dataclasses
    from paper_1806_04596_gb300 import hypersara as hs
    inp, prob, prm = _problem("f64")
    prm = dataclasses.replace(prm, use_nuclear=False, sparsity="l1")
    plan, st, w = _sara_state(inp, prob, prm, "f64", weights=True)
    hs.reweighted_solve(st, outer=2, inner=10, decay=0.7)
    ref, r1, _ = reweight.reweighted_solve(prob.op, prob.y, prob.eps, prm, outer=2, inner=10, decay=0.7)
    assert rel(host(st.get()[0]), ref.X) <= 1e-11
    assert rel(host(w), r1) <= 1e-11
