"""Non-finite values in the data never turn into out-of-range indices.

The nuclear prox (Eq. "prox-L*") ranks the eigenvalues of the Gram matrix on
the device and takes the active eigenvectors' indices from that ranking; a NaN
in the cube makes eigenvalues NaN, and NaN compares false with everything. The
library ranks NaN below every number, so the ranking stays a permutation: the
prox and a PD iteration on a cube or data with a NaN complete (their outputs
carry the NaN), and the same plan then serves finite inputs as before."""

import numpy as np
import pytest

from gpu_util import dev, host, make_plan, ragged_case, rel

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def hs(cuda_device):
    import __graft_entry__ as ge
    ge.build()
    from paper_1806_04596_gb300 import hypersara
    return hypersara


@pytest.mark.parametrize("prec", ["f32", "f64"])
def test_nuclear_prox_with_nan_completes(hs, prec):
    import torch
    c = ragged_case(n=32, L=5, M=(300, 200, 250, 100, 150), seed=12)
    plan = make_plan(c, prec)
    X = dev(c["X"], prec)
    ref, sv_ref = plan.prox_nuclear(X, 0.5)
    ref = host(ref)
    Xn = X.clone()
    Xn[2, 7, 9] = float("nan")
    out, sv = plan.prox_nuclear(Xn, 0.5)
    torch.cuda.synchronize()
    assert torch.isnan(out).any()
    again, sv2 = plan.prox_nuclear(X, 0.5)
    assert rel(host(again), ref) <= 1e-12
    assert torch.equal(sv2, sv_ref)


def test_pd_iterations_with_nan_data_complete(hs):
    import torch
    c = ragged_case(n=32, L=3, M=(300, 200, 250), seed=13)
    plan = make_plan(c, "f32")
    Y = dev(c["Y"], "f32", True)
    eps = torch.ones(3, dtype=torch.float64, device="cuda")
    Yn = Y.clone()
    Yn[17] = complex(float("nan"), 0.0)
    st = hs.PDState(plan, Yn, eps, kappa3=1e-3, mu=0.01)
    st.solve(4, graph=False)
    X, beta, rho = st.get()
    torch.cuda.synchronize()
    # the NaN block's radius is NaN, and max(0, 1 - eps / rho) takes 0: that block's
    # dual stays zero, the other blocks proceed
    assert not np.isfinite(rho[0]) and np.isfinite(rho[1:]).all()
    ok = hs.PDState(plan, Y, eps, kappa3=1e-3, mu=0.01)
    ok.solve(4, graph=True)
    X2, beta2, _ = ok.get()
    assert np.isfinite(beta2) and torch.isfinite(X2).all()
