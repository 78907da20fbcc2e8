"""Host-buffer entry points of the PD state (hs_pd_set_data_host,
hs_pd_get_host): the same iterates as the device-buffer calls, bit for bit,
from numpy arrays and from pinned torch tensors."""

import numpy as np
import pytest

import synth
from gpu_util import dev, host
from oracle import problem

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("prec", ["f32", "f64"])
def test_host_buffers_match_device_buffers(cuda_device, prec):
    import torch
    import __graft_entry__ as ge
    ge.build()
    from paper_1806_04596_gb300 import hypersara as hs
    inp = synth.make_inputs(1, n=32, L=3, M=500, seed=17)
    prob = problem.make_problem(inp)
    plan = hs.Plan(inp.nx, inp.ny, inp.offsets, dev(inp.uv, prec), levels=2, prec=prec)
    eps = torch.tensor(prob.eps, dtype=torch.float64, device="cuda")
    kw = dict(tau=0.33, kappa3=1.0 / problem.op_norm2(prob.op), mu=0.02)
    a = hs.PDState(plan, dev(prob.y, prec, True), eps, **kw)
    a.solve(4, graph=False)
    Xa, beta_a, rho_a = a.get()
    # same problem, data given from host memory; zero data first so set_data_host matters
    b = hs.PDState(plan, torch.zeros_like(dev(prob.y, prec, True)), eps, **kw)
    ynp = prob.y.astype(np.complex64 if prec == "f32" else np.complex128)
    b.set_data_host(ynp, prob.eps.astype(np.float64))
    b.solve(4, graph=False)
    Xh = np.empty((3, 32, 32), dtype=np.float32 if prec == "f32" else np.float64)
    beta_b, rho_b = b.get_host(Xh)
    assert np.array_equal(Xh, host(Xa).astype(Xh.dtype))
    assert beta_b == beta_a and np.array_equal(rho_b, rho_a)
    # pinned torch tensors
    c = hs.PDState(plan, torch.zeros_like(dev(prob.y, prec, True)), eps, **kw)
    yp = torch.tensor(ynp).pin_memory()
    c.set_data_host(yp, prob.eps.astype(np.float64))
    c.solve(4, graph=True)
    Xp = torch.empty((3, 32, 32), dtype=plan.rdtype).pin_memory()
    c.get_host(Xp)
    assert np.array_equal(Xp.numpy(), Xh)
    with pytest.raises(ValueError):
        c.set_data_host(ynp[:-1], prob.eps.astype(np.float64))
