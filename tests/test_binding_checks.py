"""The Python binding rejects tensors whose dtype or size does not match what
the C functions will read and write, before anything is launched (the C side
receives bare pointers and cannot check). Runs on the CPU: every rejection
happens before a device is touched."""

import pytest

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def hs():
    import __graft_entry__ as ge
    ge.build()
    from paper_1806_04596_gb300 import hypersara
    return hypersara


def _static_args(n=10, L=2, cdt=torch.complex64):
    off = torch.tensor([0, 4, n], dtype=torch.int64)
    Z = torch.zeros(n, dtype=cdt)
    return off, Z, Z.clone(), torch.ones(L, dtype=torch.float64)


@pytest.mark.parametrize("prec,wrong", [("f32", torch.complex128), ("f64", torch.complex64)])
def test_static_projection_rejects_wrong_precision(hs, prec, wrong):
    off, Z, Y, eps = _static_args(cdt=wrong)
    with pytest.raises(ValueError, match="dtype"):
        hs.proj_l2ball_static(off, Z, Y, eps, prec=prec)


def test_static_projection_rejects_bad_offsets_eps_and_sizes(hs):
    off, Z, Y, eps = _static_args()
    with pytest.raises(ValueError, match="offsets must have dtype"):
        hs.proj_l2ball_static(off.to(torch.int32), Z, Y, eps)
    with pytest.raises(ValueError, match="eps must have dtype"):
        hs.proj_l2ball_static(off, Z, Y, eps.float())
    with pytest.raises(ValueError, match="eps must have 2 elements"):
        hs.proj_l2ball_static(off, Z, Y, torch.ones(3, dtype=torch.float64))
    with pytest.raises(ValueError, match="Yd must have 10 elements"):
        hs.proj_l2ball_static(off, Z, Y[:9].clone(), eps)
    with pytest.raises(ValueError, match="out must have dtype"):
        hs.proj_l2ball_static(off, Z, Y, eps, out=torch.zeros(10, dtype=torch.complex128))
    with pytest.raises(ValueError, match="CUDA"):       # right dtypes and sizes, host tensors
        hs.proj_l2ball_static(off, Z, Y, eps)


def _fake_plan(hs, prec="f32"):
    p = object.__new__(hs.Plan)
    p.nx, p.ny, p.L, p.M, p.h = 8, 8, 3, 50, None
    p.nblocks = 3
    p.rdtype = torch.float32 if prec == "f32" else torch.float64
    p.cdtype = torch.complex64 if prec == "f32" else torch.complex128
    return p


@pytest.mark.parametrize("prec", ["f32", "f64"])
def test_plan_operators_reject_mismatched_tensors(hs, prec):
    p = _fake_plan(hs, prec)
    other_r = torch.float64 if prec == "f32" else torch.float32
    other_c = torch.complex128 if prec == "f32" else torch.complex64
    X = torch.zeros((3, 8, 8), dtype=p.rdtype)
    Y = torch.zeros(50, dtype=p.cdtype)
    A = torch.zeros((9, 3, 8, 8), dtype=p.rdtype)
    with pytest.raises(ValueError, match="dtype"):
        p.phi_fwd(X.to(other_r), Y)
    with pytest.raises(ValueError, match="dtype"):
        p.phi_fwd(X, Y.to(other_c))
    with pytest.raises(ValueError, match="elements"):
        p.phi_adj(Y[:49].clone(), X)
    with pytest.raises(ValueError, match="elements"):
        p.psi_fwd(X, A[:, :2].clone())
    with pytest.raises(ValueError, match="elements"):
        p.psi_adj(A, X[:2].clone())
    with pytest.raises(ValueError, match="w_rows"):
        p.prox_l21(A, 1.0, w_rows=torch.ones(8, dtype=p.rdtype), out=A.clone())
    with pytest.raises(ValueError, match="eps"):
        p.proj_l2ball(Y, Y.clone(), torch.ones(3, dtype=torch.float32), out=Y.clone())
