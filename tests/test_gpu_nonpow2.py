"""Grids whose side is not a power of two (Sec. 5's 1280 x 1280 image; images
r 2^a with r = 3 or 5): the mixed-radix FFT (radix-5 or -3 pass, then 4 and 2),
periodic wraps of the gridding, de-gridding and wavelet kernels without
power-of-two masks, against the FP64 oracle in both precisions.

Cases: 192 x 192 (K = 384 = 3 x 128), 320 x 192 (K = 640 x 384, rectangular),
and 1280 x 1280 (K = 2560 = 5 x 512) with coverage reaching the band edge, so
windows wrap around the grid; Phi, Phi^dagger, Psi^dagger and Psi, and a few
FP64 PD iterations against the oracle's Algorithm 2."""

import numpy as np
import pytest

import synth
from gpu_util import assert_close, dev, host, make_plan, oracle_op, ragged_case, rounded
from oracle import pd, problem, wavelets

pytestmark = pytest.mark.gpu

CASES = {
    "n192": (dict(n=192, L=2, M=(3000, 1700), seed=41, uv_std=1.2), 2),
    "rect320x192": (dict(nx=320, ny=192, L=2, M=(2500, 900), seed=42, uv_std=1.2), 2),
    "n1280": (dict(n=1280, L=1, M=(4000,), seed=43, uv_std=1.4), 4),
}


@pytest.fixture(scope="module", autouse=True)
def _built(cuda_device):
    import __graft_entry__ as ge
    ge.build()


@pytest.mark.parametrize("prec", ["f64", "f32"])
@pytest.mark.parametrize("name", list(CASES))
def test_phi_and_adjoint(prec, name):
    kw, levels = CASES[name]
    c = rounded(ragged_case(**kw), prec)
    plan = make_plan(c, prec, levels=levels)
    op = oracle_op(c)
    assert_close(host(plan.phi_fwd(dev(c["X"], prec))), op.forward(c["X"]), prec)
    assert_close(host(plan.phi_adj(dev(c["Y"], prec, True))), op.adjoint(c["Y"]), prec)


@pytest.mark.parametrize("prec", ["f64", "f32"])
@pytest.mark.parametrize("name", list(CASES))
def test_psi_analysis_and_synthesis(prec, name):
    kw, levels = CASES[name]
    c = rounded(ragged_case(**kw), prec)
    plan = make_plan(c, prec, levels=levels)
    A = host(plan.psi_fwd(dev(c["X"], prec)))
    assert_close(A, wavelets.psi_adjoint_cube(c["X"], levels), prec)
    B = np.random.default_rng(7).standard_normal(A.shape)
    if prec == "f32":
        B = B.astype(np.float32).astype(np.float64)
    assert_close(host(plan.psi_adj(dev(B, prec))), wavelets.psi_cube(B, levels), prec)


def test_pd_fp64_on_non_power_of_two_grid():
    import torch
    from paper_1806_04596_gb300 import hypersara as hs
    inp = synth.make_inputs(1, n=192, L=3, M=1500, seed=44)
    prob = problem.make_problem(inp)
    mu = problem.estimate_mu(prob.op, prob.y, 2)
    k3 = 1.0 / problem.op_norm2(prob.op)
    plan = hs.Plan(inp.nx, inp.ny, inp.offsets, dev(inp.uv, "f64"), levels=2, prec="f64")
    st = hs.PDState(plan, dev(prob.y, "f64", True), torch.tensor(prob.eps, dtype=torch.float64, device="cuda"),
                    tau=0.33, kappa3=k3, mu=mu)
    st.solve(10, graph=True)
    X, beta, rho = st.get()
    ref = pd.pd_solve(prob.op, prob.y, prob.eps, pd.PDParams(mu=mu, tau=0.33, kappa3=k3, levels=2), 10)
    assert_close(host(X), ref.X, "f64")
    np.testing.assert_allclose(rho, ref.rho, rtol=1e-10)


def test_unsupported_sides_are_rejected():
    import torch
    from paper_1806_04596_gb300 import hypersara as hs
    uv = torch.zeros((1, 2), dtype=torch.float64, device="cuda")
    for nx, ny, levels in ((100, 64, 2), (112, 64, 2), (80, 80, 4)):
        with pytest.raises(hs.HSError):   # 25 x 4; 7 x 16; level subbands of 40 x 40
            hs.Plan(nx, ny, np.array([0, 1]), uv, levels=levels, prec="f64")
