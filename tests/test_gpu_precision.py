"""Precision of the FP32 forms on the generator of the 1024 x 1024, L = 16,
M = 1e6 workload (50 sources plus a diffuse field, 30 dB), at reduced size
(128 x 128, L = 4, M = 20000): per-operator error of the FP32 and FP32
compensated-gridding plans against the FP64 oracle, and the reconstruction
after 100 PD iterations against the FP64 GPU form (which tracks the oracle to
~1e-12 per iteration): aSNR within 0.05 dB."""

import numpy as np
import pytest

import synth
from gpu_util import dev, host, rel
from oracle import nufft, problem

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def c4small(cuda_device):
    import __graft_entry__ as ge
    ge.build()
    inp = synth.make_inputs(4, n=128, L=4, M=20000)
    inp.uv = inp.uv.astype(np.float32).astype(np.float64)
    prob = problem.make_problem(inp)
    return inp, prob


def test_operator_errors_fp32_and_compensated(c4small):
    import torch
    from paper_1806_04596_gb300 import hypersara as hs
    inp, prob = c4small
    y = prob.y.astype(np.complex64).astype(np.complex128)
    errs = {}
    for comp in (False, True):
        plan = hs.Plan(inp.nx, inp.ny, inp.offsets, dev(inp.uv, "f32"), levels=4, prec="f32", compensated=comp)
        Xa = host(plan.phi_adj(dev(y, "f32", True)))
        ref = prob.op.adjoint(y)
        errs[comp] = rel(Xa, ref)
        X = inp.truth.astype(np.float32).astype(np.float64)
        assert rel(host(plan.phi_fwd(dev(X, "f32"))), prob.op.forward(X)) <= 1e-5
    assert errs[False] <= 1e-5 and errs[True] <= 1e-5
    assert errs[True] <= errs[False] * 1.5   # compensation never worse beyond noise


def test_cube_snr_fp32_matches_fp64(c4small):
    import torch
    from paper_1806_04596_gb300 import hypersara as hs
    inp, prob = c4small
    mu = problem.estimate_mu(prob.op, prob.y, 4)
    k3 = 1.0 / problem.op_norm2(prob.op, iters=100, tol=1e-8)
    eps = torch.tensor(prob.eps, dtype=torch.float64, device="cuda")
    out = {}
    for prec, comp in (("f64", False), ("f32", False), ("f32", True)):
        plan = hs.Plan(inp.nx, inp.ny, inp.offsets, dev(inp.uv, prec), levels=4, prec=prec, compensated=comp)
        st = hs.PDState(plan, dev(prob.y, prec, True), eps, tau=0.33, kappa3=k3, mu=mu)
        st.solve(100, graph=True)
        X, _, _ = st.get()
        Xh = host(X)
        out[(prec, comp)] = (np.mean([20 * np.log10(np.linalg.norm(inp.truth[l]) /
                                                    np.linalg.norm(inp.truth[l] - Xh[l])) for l in range(inp.L)]), Xh)
    s64 = out[("f64", False)][0]
    for key in (("f32", False), ("f32", True)):
        assert abs(out[key][0] - s64) <= 0.05, (key, out[key][0], s64)
        assert rel(out[key][1], out[("f64", False)][1]) <= 1e-3
