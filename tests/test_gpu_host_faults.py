"""Failures made on the host and reported by the library without touching the
GPU's state: plan creation rejects non-finite and out-of-band coordinates and
non-positive preconditioner entries (host-built inputs, detected before any
kernel), the library's device-memory cap makes allocations fail with
HS_ERR_NOMEM and releases the partial plan, and a state stays usable after a
rejected call."""

import numpy as np
import pytest

from gpu_util import dev, make_plan, ragged_case

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def hs(cuda_device):
    import __graft_entry__ as ge
    ge.build()
    from paper_1806_04596_gb300 import hypersara
    return hypersara


@pytest.mark.parametrize("bad", ["nan", "inf", "pi", "below"])
def test_bad_coordinates_rejected(hs, bad):
    c = ragged_case(n=32, L=2, M=(200, 100), seed=3)
    uv = c["uv"].copy()
    uv[57, 1] = {"nan": np.nan, "inf": np.inf, "pi": np.pi, "below": -3.2}[bad]
    with pytest.raises(hs.HSError) as e:
        make_plan(dict(c, uv=uv), "f64")
    assert e.value.status == hs.HS_ERR_ARG and "uv[57]" in str(e.value)


@pytest.mark.parametrize("val", [0.0, -1.0, np.nan])
def test_non_positive_preconditioner_rejected(hs, val):
    c = ragged_case(n=32, L=2, M=(200, 100), seed=4)
    U = np.ones(300)
    U[123] = val
    with pytest.raises(hs.HSError) as e:
        make_plan(c, "f64", precond=U)
    assert e.value.status == hs.HS_ERR_ARG and "precond[123]" in str(e.value)


def test_device_limit_gives_nomem_and_releases(hs):
    import torch
    c = ragged_case(n=64, L=3, M=(500, 400, 300), seed=5)
    before = hs.device_bytes()
    try:
        hs.set_device_limit(before + (1 << 20))   # 1 MiB more than held now: the plan needs more
        with pytest.raises(hs.HSError) as e:
            make_plan(c, "f32")
        assert e.value.status == hs.HS_ERR_NOMEM and "limit" in str(e.value)
        assert hs.device_bytes() == before       # the partial plan was released
    finally:
        hs.set_device_limit(0)
    plan = make_plan(c, "f32")                    # without the cap it succeeds
    assert hs.device_bytes() == before + plan.info["device_bytes"]
    Y = plan.phi_fwd(dev(c["X"], "f32"))
    assert torch.isfinite(Y).all()


def test_rejected_call_leaves_state_usable(hs):
    import torch
    c = ragged_case(n=32, L=2, M=(200, 100), seed=6)
    plan = make_plan(c, "f64")
    Y = dev(c["Y"], "f64", True)
    eps = torch.ones(2, dtype=torch.float64, device="cuda")
    st = hs.PDState(plan, Y, eps, kappa3=1e-3, mu=0.01)
    st.solve(2, graph=False)
    with pytest.raises(ValueError):
        st.set_data(Y[:-1].clone(), eps)         # wrong size: rejected before the call
    with pytest.raises(hs.HSError) as e:
        st.solve(-1, graph=False)                 # rejected by the library (HS_ERR_ARG)
    assert e.value.status == hs.HS_ERR_ARG
    st.solve(2, graph=False)
    X, beta, rho = st.get()
    assert np.isfinite(beta) and torch.isfinite(X).all()
