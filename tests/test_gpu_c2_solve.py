"""The benchmarked workload solved to its stated iteration count: 256 x 256,
L = 60, M = 32768 per channel, 500 PD iterations replayed from the CUDA graph,
against the FP64 oracle's solve of the same problem (tests/golden/c2_pd500.json,
written by tests/golden/make_c2_golden.py from oracle/ only: same seeded inputs
rounded to FP32, the oracle's mu and kappa_3 passed to both sides).

FP32 form: aSNR within 0.05 dB of the oracle's (the workload's criterion), the
per-channel SNR within 0.1 dB, the per-channel norms and a 16 x 16 block-sum
checksum of the cube within 1e-3. FP64 form: the same quantities within 1e-8
(it follows the oracle's iterates to rounding)."""

import json
import os

import numpy as np
import pytest

import synth
from gpu_util import dev, host
from oracle import metrics, problem

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "c2_pd500.json")


@pytest.fixture(scope="module")
def c2_golden(cuda_device):
    import __graft_entry__ as ge
    ge.build()
    g = json.load(open(GOLDEN))
    inp = synth.make_inputs(2)
    inp.uv = inp.uv.astype(np.float32).astype(np.float64)
    inp.truth = inp.truth.astype(np.float32).astype(np.float64)
    prob = problem.make_problem(inp)
    prob.y = prob.y.astype(np.complex64).astype(np.complex128)
    return g, inp, prob


def _solve(g, inp, prob, prec):
    import torch
    from paper_1806_04596_gb300 import hypersara as hs
    plan = hs.Plan(inp.nx, inp.ny, inp.offsets, dev(inp.uv, prec), levels=4, prec=prec)
    st = hs.PDState(plan, dev(prob.y, prec, True), torch.tensor(prob.eps, dtype=torch.float64, device="cuda"),
                    tau=g["tau"], kappa1=g["kappa1"], kappa2=g["kappa2"], kappa3=g["kappa3"], mu=g["mu"])
    st.solve(g["iterations"], graph=True)
    X, beta, rho = st.get()
    plan.check()
    return host(X), beta, rho


def _summary(X, truth):
    L, ny, nx = X.shape
    return dict(asnr=metrics.asnr(truth, X), snr=np.array([metrics.snr(truth[l], X[l]) for l in range(L)]),
                x_norm=np.linalg.norm(X.reshape(L, -1), axis=1),
                blocks=X.sum(axis=0).reshape(16, ny // 16, 16, nx // 16).sum(axis=(1, 3)).ravel())


def test_fp32_solve_matches_oracle_snr(c2_golden):
    g, inp, prob = c2_golden
    X, beta, rho = _solve(g, inp, prob, "f32")
    s = _summary(X, prob.truth)
    assert abs(s["asnr"] - g["asnr"]) <= 0.05, (s["asnr"], g["asnr"])
    assert np.max(np.abs(s["snr"] - np.array(g["snr"]))) <= 0.1
    np.testing.assert_allclose(s["x_norm"], g["x_norm"], rtol=1e-3)
    gb = np.array(g["block_sums_16x16"])
    assert np.max(np.abs(s["blocks"] - gb)) <= 1e-3 * np.max(np.abs(gb))
    np.testing.assert_allclose(rho, g["rho"], rtol=1e-3)


def test_fp64_solve_follows_oracle(c2_golden):
    g, inp, prob = c2_golden
    X, beta, rho = _solve(g, inp, prob, "f64")
    s = _summary(X, prob.truth)
    assert abs(s["asnr"] - g["asnr"]) <= 1e-6
    np.testing.assert_allclose(s["x_norm"], g["x_norm"], rtol=1e-8)
    gb = np.array(g["block_sums_16x16"])
    assert np.max(np.abs(s["blocks"] - gb)) <= 1e-8 * np.max(np.abs(gb))
    np.testing.assert_allclose(rho, g["rho"], rtol=1e-8)
    assert beta == pytest.approx(g["beta"], rel=1e-5)
