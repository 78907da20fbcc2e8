"""The allocation-free l2-ball projection (hs_proj_l2ball_static) against the
plan-based hs_proj_l2ball on the same inputs: two calls in a row, both
precisions, both modes; device memory unchanged by the calls after the first.
Collected last so that it also runs after every other GPU test."""

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def hs(cuda_device):
    import __graft_entry__ as ge
    ge.build()
    from paper_1806_04596_gb300 import hypersara
    return hypersara


@pytest.mark.parametrize("prec,tol", [("f32", 1e-6), ("f64", 1e-13)])
def test_static_matches_plan_projection(hs, prec, tol):
    import torch
    rng = np.random.default_rng(31)
    M = np.array([700, 0, 1500, 33, 4097])     # ragged, with an empty channel
    off = np.concatenate([[0], np.cumsum(M)]).astype(np.int64)
    total = int(off[-1])
    rt = torch.float32 if prec == "f32" else torch.float64
    uv = torch.tensor(rng.uniform(-np.pi, np.pi, (total, 2)), dtype=rt, device="cuda")
    plan = hs.Plan(64, 64, off, uv, prec=prec)
    cd = torch.complex64 if prec == "f32" else torch.complex128
    Z = torch.tensor(rng.standard_normal(total) + 1j * rng.standard_normal(total), dtype=cd, device="cuda")
    Y = torch.tensor(rng.standard_normal(total) + 1j * rng.standard_normal(total), dtype=cd, device="cuda")
    # balls that cut some channels and contain others
    eps = torch.tensor([10.0, 1.0, 1e3, 2.0, 40.0], dtype=torch.float64, device="cuda")
    offs = torch.tensor(off, device="cuda")
    for dual in (False, True):
        ref, rho_ref = plan.proj_l2ball(Z, Y, eps, dual)
        hs.proj_l2ball_static(offs, Z, Y, eps, dual, prec=prec)   # first call: set-up
        torch.cuda.synchronize()
        free0 = torch.cuda.mem_get_info()[0]
        for _ in range(2):
            out, rho = hs.proj_l2ball_static(offs, Z, Y, eps, dual, prec=prec)
            torch.cuda.synchronize()
            a, b = out.cpu().numpy(), ref.cpu().numpy()
            assert np.max(np.abs(a - b)) <= tol * max(1.0, np.max(np.abs(b))), (prec, dual)
            np.testing.assert_allclose(rho.cpu().numpy(), rho_ref.cpu().numpy(), rtol=1e-12, atol=0)
        assert torch.cuda.mem_get_info()[0] == free0
    # rho is the channel norm of z - y (the difference is formed in the plan's precision)
    d = Z.cpu().numpy().astype(np.complex128) - Y.cpu().numpy().astype(np.complex128)
    want = [np.linalg.norm(d[off[l]:off[l + 1]]) for l in range(len(M))]
    np.testing.assert_allclose(rho.cpu().numpy(), want, rtol=max(tol, 1e-12), atol=1e-300)


def test_static_in_place(hs):
    import torch
    rng = np.random.default_rng(5)
    off = np.array([0, 300, 900], dtype=np.int64)
    Z = torch.tensor(rng.standard_normal(900) + 1j * rng.standard_normal(900), dtype=torch.complex64,
                     device="cuda")
    Y = torch.zeros_like(Z)
    eps = torch.tensor([1.0, 2.0], dtype=torch.float64, device="cuda")
    offs = torch.tensor(off, device="cuda")
    want, _ = hs.proj_l2ball_static(offs, Z, Y, eps)
    Zc = Z.clone()
    hs.proj_l2ball_static(offs, Zc, Y, eps, out=Zc)
    torch.cuda.synchronize()
    assert torch.equal(Zc, want)
    n = torch.linalg.vector_norm(Zc[300:]).item()
    assert abs(n - 2.0) <= 1e-5
