"""GPU parity at the full size of the 256 x 256, L = 60, M = 32768 per channel
FP32 workload, in the launch configuration the benchmark times (one plan for
all channels, the PD iteration replayed from its CUDA graph):

* Phi, Phi^dagger, Psi^dagger and Psi of the whole cube, checked on three
  sampled channels against the oracle (the operators are channel-separable);
* two PD iterations of the whole problem against the FP64 oracle (the nuclear
  prior couples all channels, so the oracle runs all of them), with the same
  mu, kappa_3 and tau on both sides.

Tolerances are the FP32 ones of the smaller cases (inputs rounded to FP32)."""

import numpy as np
import pytest

import synth
from gpu_util import TOL, dev, host, rel
from oracle import pd, problem, wavelets

pytestmark = pytest.mark.gpu

CH = (0, 29, 59)   # sampled channels: lowest, middle and highest frequency


@pytest.fixture(scope="module")
def c2(cuda_device):
    import __graft_entry__ as ge
    ge.build()
    from paper_1806_04596_gb300 import hypersara as hs
    inp = synth.make_inputs(2)
    inp.uv = inp.uv.astype(np.float32).astype(np.float64)
    inp.truth = inp.truth.astype(np.float32).astype(np.float64)
    prob = problem.make_problem(inp)
    prob.y = prob.y.astype(np.complex64).astype(np.complex128)
    plan = hs.Plan(inp.nx, inp.ny, inp.offsets, dev(inp.uv, "f32"), levels=4, prec="f32")
    return inp, prob, plan


def _vis(inp, Y, l):
    return Y[inp.offsets[l]:inp.offsets[l + 1]]


def test_c2_operators_on_sampled_channels(c2):
    inp, prob, plan = c2
    rng = np.random.default_rng(5)
    X = rng.uniform(0.0, 1.0, (inp.L, inp.ny, inp.nx)).astype(np.float32).astype(np.float64)
    Y = host(plan.phi_fwd(dev(X, "f32")))
    for l in CH:
        ref = prob.op.ch[l].forward(X[l])
        assert rel(_vis(inp, Y, l), ref) <= TOL["f32"], l
    Yin = prob.y
    Xa = host(plan.phi_adj(dev(Yin, "f32", True)))
    for l in CH:
        ref = prob.op.ch[l].adjoint(_vis(inp, Yin, l))
        assert rel(Xa[l], ref) <= TOL["f32"], l
    A = host(plan.psi_fwd(dev(X, "f32")))
    refA = wavelets.psi_adjoint_cube(X[list(CH)], 4)
    assert rel(A[:, list(CH)], refA) <= TOL["f32"]
    B = rng.standard_normal(A.shape).astype(np.float32).astype(np.float64)
    Xb = host(plan.psi_adj(dev(B, "f32")))
    assert rel(Xb[list(CH)], wavelets.psi_cube(B[:, list(CH)], 4)) <= TOL["f32"]


def test_c2_pd_iterations_whole_problem(c2):
    import torch
    from paper_1806_04596_gb300 import hypersara as hs
    inp, prob, plan = c2
    prm = pd.PDParams(mu=0.0182, tau=0.33, kappa3=1.48e-6, levels=4)
    st = hs.PDState(plan, dev(prob.y, "f32", True), torch.tensor(prob.eps, dtype=torch.float64, device="cuda"),
                    tau=prm.tau, kappa1=prm.kappa1, kappa2=prm.kappa2, kappa3=prm.kappa3, mu=prm.mu)
    st.solve(2, graph=True)
    X, beta, rho = st.get()
    ref = pd.pd_solve(prob.op, prob.y, prob.eps, prm, 2)
    assert rel(host(X), ref.X) <= 1e-4
    np.testing.assert_allclose(rho, ref.rho, rtol=1e-4)
