"""Differentiable operators (paper_1806_04596_gb300.autograd) through the C ABI:
Phi, Phi^dagger, Psi^dagger, Psi and the l2,1 norm as torch.autograd
Functions whose backward passes are the adjoint kernels.

* torch.autograd.gradcheck (central differences) of every Function on an FP64
  plan with uneven and empty channels;
* the gradient of f(X) = 0.5 ||Phi X - y||^2 + ||Psi^dagger X||_{2,1} against
  the oracle's (oracle/grad.py) in FP64 and FP32, and against central
  differences with step 1e-3 (FP64 and FP32 objectives);
* the unrolled primal-dual solve against the oracle's Algorithm 2 (JAS and
  LRJAS), its gradient with respect to the data against central differences,
  and checkpointed (every 5 iterations) against stored gradients and peak
  memory."""

import numpy as np
import pytest

import synth
from gpu_util import dev, host, rel
from oracle import grad as ograd
from oracle import pd, problem

pytestmark = pytest.mark.gpu


def _setup(prec, n=32, L=3, M=(300, 0, 420), seed=31, levels=2):
    import __graft_entry__ as ge
    ge.build()
    from paper_1806_04596_gb300 import hypersara as hs
    inp = synth.make_inputs(1, n=n, L=L, M=max(M), seed=seed)
    off = np.zeros(L + 1, dtype=np.int64)
    off[1:] = np.cumsum(M)
    uv = np.concatenate([inp.uv[inp.offsets[l]:inp.offsets[l] + M[l]] for l in range(L)])
    if prec == "f32":
        uv = uv.astype(np.float32).astype(np.float64)
    op = problem.nufft.WidebandOperator(n, n, uv, off)
    plan = hs.Plan(n, n, off, dev(uv, prec), levels=levels, prec=prec)
    return plan, op, off


def test_gradcheck_operators(cuda_device):
    import torch
    from paper_1806_04596_gb300 import autograd as ag
    plan, _, off = _setup("f64", n=16, L=2, M=(40, 25), levels=1)
    X = torch.rand((2, 16, 16), dtype=torch.float64, device="cuda", requires_grad=True)
    Y = torch.randn(int(off[-1]), dtype=torch.complex128, device="cuda", requires_grad=True)
    A = torch.randn((9, 2, 16, 16), dtype=torch.float64, device="cuda", requires_grad=True)
    kw = dict(eps=1e-6, atol=1e-6, rtol=1e-5)
    assert torch.autograd.gradcheck(lambda x: ag.phi(plan, x), (X,), **kw)
    assert torch.autograd.gradcheck(lambda y: ag.phi_adj(plan, y), (Y,), **kw)
    assert torch.autograd.gradcheck(lambda x: ag.psi_analysis(plan, x), (X,), **kw)
    assert torch.autograd.gradcheck(lambda a: ag.psi_synthesis(plan, a), (A,), **kw)
    assert torch.autograd.gradcheck(lambda a: ag.l21_norm(plan, a), (A,), **kw)


@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_objective_gradient_vs_oracle_and_differences(cuda_device, prec):
    import torch
    from paper_1806_04596_gb300 import autograd as ag
    plan, op, off = _setup(prec)
    rng = np.random.default_rng(2)
    X = rng.uniform(0.0, 1.0, (3, 32, 32))
    y = rng.standard_normal(int(off[-1])) + 1j * rng.standard_normal(int(off[-1]))
    if prec == "f32":
        X = X.astype(np.float32).astype(np.float64)
        y = y.astype(np.complex64).astype(np.complex128)
    Xt = dev(X, prec).requires_grad_(True)
    Yt = dev(y, prec, True)
    f = ag.objective(plan, Xt, Yt)
    (g,) = torch.autograd.grad(f, Xt)
    g = host(g)
    ref = ograd.gradient(op, X, y, 2)
    assert rel(g, ref) <= (1e-10 if prec == "f64" else 2e-5)
    assert float(f.detach()) == pytest.approx(ograd.objective(op, X, y, 2), rel=1e-10 if prec == "f64" else 1e-5)
    # central differences with step 1e-3 along random directions
    for k in range(3):
        D = rng.standard_normal(X.shape)
        h = 1e-3
        with torch.no_grad():
            fp = float(ag.objective(plan, dev(X + h * D, prec), Yt).double())
            fm = float(ag.objective(plan, dev(X - h * D, prec), Yt).double())
        fd = (fp - fm) / (2 * h)
        assert np.sum(g * D) == pytest.approx(fd, rel=1e-6 if prec == "f64" else 2e-2)


def _pd_problem(n=32, L=3, M=400, seed=8, levels=2):
    inp = synth.make_inputs(1, n=n, L=L, M=M, seed=seed)
    prob = problem.make_problem(inp)
    mu = problem.estimate_mu(prob.op, prob.y, levels)
    k3 = 1.0 / problem.op_norm2(prob.op)
    return inp, prob, mu, k3


@pytest.mark.parametrize("nuclear", [False, True])
def test_unrolled_pd_matches_oracle(cuda_device, nuclear):
    import torch
    from paper_1806_04596_gb300 import autograd as ag
    from paper_1806_04596_gb300 import hypersara as hs
    inp, prob, mu, k3 = _pd_problem()
    plan = hs.Plan(inp.nx, inp.ny, inp.offsets, dev(inp.uv, "f64"), levels=2, prec="f64")
    eps = torch.tensor(prob.eps, dtype=torch.float64, device="cuda")
    X = ag.unrolled_pd(plan, dev(prob.y, "f64", True), eps, iters=15, mu=mu, kappa3=k3, use_nuclear=nuclear)
    prm = pd.PDParams(mu=mu, tau=0.33, kappa3=k3, levels=2, use_nuclear=nuclear)
    ref = pd.pd_solve(prob.op, prob.y, prob.eps, prm, 15)
    assert rel(host(X), ref.X) <= 1e-10


def test_unrolled_pd_gradient_and_checkpointing(cuda_device):
    import torch
    from paper_1806_04596_gb300 import autograd as ag
    from paper_1806_04596_gb300 import hypersara as hs
    inp, prob, mu, k3 = _pd_problem()
    plan = hs.Plan(inp.nx, inp.ny, inp.offsets, dev(inp.uv, "f64"), levels=2, prec="f64")
    eps = torch.tensor(prob.eps, dtype=torch.float64, device="cuda")
    truth = dev(prob.truth, "f64")
    y0 = dev(prob.y, "f64", True)

    def loss(Y, ck):
        X = ag.unrolled_pd(plan, Y, eps, iters=20, mu=mu, kappa3=k3, checkpoint_every=ck)
        return 0.5 * torch.sum((X - truth) ** 2)

    grads = {}
    for ck in (0, 5):
        Y = y0.clone().requires_grad_(True)
        (grads[ck],) = torch.autograd.grad(loss(Y, ck), Y)
    assert rel(host(grads[5]), host(grads[0])) <= 1e-12
    rng = np.random.default_rng(4)
    g = host(grads[0])
    for _ in range(2):
        D = rng.standard_normal(g.shape) + 1j * rng.standard_normal(g.shape)
        h = 1e-6 * np.linalg.norm(prob.y) / np.linalg.norm(D)
        with torch.no_grad():
            fd = (float(loss(y0 + h * dev(D, "f64", True), 0)) - float(loss(y0 - h * dev(D, "f64", True), 0))) / (2 * h)
        assert np.real(np.vdot(g, D)) == pytest.approx(fd, rel=1e-4)


def test_checkpointing_lowers_peak_memory(cuda_device):
    import torch
    from paper_1806_04596_gb300 import autograd as ag
    from paper_1806_04596_gb300 import hypersara as hs
    inp = synth.make_inputs(1, n=128, L=8, M=20000, seed=9)
    prob = problem.make_problem(inp)
    plan = hs.Plan(inp.nx, inp.ny, inp.offsets, dev(inp.uv, "f32"), levels=4, prec="f32")
    eps = torch.tensor(prob.eps, dtype=torch.float64, device="cuda")
    peaks = {}
    for ck in (0, 5):
        Y = dev(prob.y, "f32", True).requires_grad_(True)
        torch.cuda.synchronize()
        torch.cuda.reset_peak_memory_stats()
        base = torch.cuda.memory_allocated()
        X = ag.unrolled_pd(plan, Y, eps, iters=20, mu=0.01, kappa3=1.0 / plan.op_norm2(iters=50, tol=1e-4),
                           checkpoint_every=ck)
        torch.sum(X).backward()
        torch.cuda.synchronize()
        peaks[ck] = torch.cuda.max_memory_allocated() - base
        del X, Y
    assert peaks[5] < 0.5 * peaks[0], peaks
