"""GPU parity of every operator against the FP64 oracle, through the C ABI.

Cases span several 32 x 32 gridding tiles (grid 128 x 128), uneven and empty
channels, a rectangular image, weights, and wrap-around windows. Tolerances
(relative 2-norm over the whole output): 1e-12 for FP64 plans, 1e-5 for FP32
plans (inputs rounded to FP32 on both sides), and every element within ten
times that of the largest reference magnitude; channels without visibilities
map to exact zeros."""

import numpy as np
import pytest

from gpu_util import TOL, assert_close, dev, host, make_plan, oracle_op, ragged_case, rel, rounded
from oracle import nufft, prox, wavelets

pytestmark = pytest.mark.gpu

PRECS = ["f64", "f32"]
CASES = {
    "ragged64": dict(n=64, L=4, M=(2000, 1503, 0, 911), seed=11),
    "rect": dict(nx=64, ny=32, L=3, M=(700, 333, 1200), seed=12),
    "wide_uv": dict(n=32, L=2, M=(900, 1000), seed=13, uv_std=1.4),
    # coverage packed around u = v = 0: strips with thousands of windows in a few rows
    # (gridding work items cut short), windows wrapping around both grid edges
    "dense": dict(n=64, L=2, M=(6000, 3000), seed=17, uv_std=0.15),
    # large grids: every compile-time FFT size (K = 1024 rows and columns; K = 2048 and 4096
    # along either axis)
    "big512": dict(n=512, L=2, M=(500, 300), seed=14),
    "big_rect_x": dict(nx=2048, ny=1024, L=1, M=(400,), seed=15),
    "big_rect_y": dict(nx=1024, ny=2048, L=1, M=(400,), seed=16),
}


@pytest.fixture(scope="module", autouse=True)
def _built(cuda_device):
    import __graft_entry__ as ge
    ge.build()


def _case(name, prec):
    kw = dict(CASES[name])
    return rounded(ragged_case(**kw), prec)


@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("name", list(CASES))
def test_phi_fwd(prec, name):
    c = _case(name, prec)
    plan = make_plan(c, prec)
    Y = host(plan.phi_fwd(dev(c["X"], prec)))
    ref = oracle_op(c).forward(c["X"])
    assert_close(Y, ref, prec)


@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("name", list(CASES))
@pytest.mark.parametrize("compensated", [False, True])
def test_phi_adj(prec, name, compensated):
    c = _case(name, prec)
    plan = make_plan(c, prec, compensated=compensated)
    X = host(plan.phi_adj(dev(c["Y"], prec, True)))
    ref = oracle_op(c).adjoint(c["Y"])
    assert_close(X, ref, prec)
    for l in range(c["L"]):   # a channel without visibilities maps to exactly zero
        if c["off"][l + 1] == c["off"][l]:
            assert not np.any(X[l])


@pytest.mark.parametrize("prec", PRECS)
def test_phi_with_weights(prec):
    c = _case("ragged64", prec)
    w = np.random.default_rng(1).uniform(0.5, 2.0, c["off"][-1])
    if prec == "f32":
        w = w.astype(np.float32).astype(np.float64)
    plan = make_plan(c, prec, weights=w)
    op = nufft.WidebandOperator(c["nx"], c["ny"], c["uv"], c["off"], weights=w)
    assert_close(host(plan.phi_fwd(dev(c["X"], prec))), op.forward(c["X"]), prec)
    assert_close(host(plan.phi_adj(dev(c["Y"], prec, True))), op.adjoint(c["Y"]), prec)


@pytest.mark.parametrize("prec", PRECS)
def test_adjoint_identity_on_gpu(prec):
    c = _case("ragged64", prec)
    plan = make_plan(c, prec)
    Yx = host(plan.phi_fwd(dev(c["X"], prec)))
    Xy = host(plan.phi_adj(dev(c["Y"], prec, True)))
    lhs = np.real(np.vdot(Yx, c["Y"]))
    rhs = np.sum(c["X"] * Xy)
    assert abs(lhs - rhs) <= (1e-12 if prec == "f64" else 1e-5) * abs(lhs)


def test_compensated_gridding_matches_and_is_not_worse():
    c = _case("ragged64", "f32")
    ref = oracle_op(c).adjoint(c["Y"])
    e_plain = rel(host(make_plan(c, "f32").phi_adj(dev(c["Y"], "f32", True))), ref)
    e_comp = rel(host(make_plan(c, "f32", compensated=True).phi_adj(dev(c["Y"], "f32", True))), ref)
    assert e_comp <= TOL["f32"]
    assert e_comp <= 1.5 * e_plain + 1e-9


@pytest.mark.parametrize("prec", PRECS)
def test_gpu_deterministic(prec):
    """Both gridding kernels (the register sweep and the compensated tiles) add
    in a fixed order: repeated adjoints are bitwise equal; the two kernels agree
    to rounding."""
    c = _case("ragged64", prec)
    plan = make_plan(c, prec, compensated=True)
    a = host(plan.phi_adj(dev(c["Y"], prec, True)))
    b = host(plan.phi_adj(dev(c["Y"], prec, True)))
    assert np.array_equal(a, b)
    plan2 = make_plan(c, prec)
    d1 = host(plan2.phi_adj(dev(c["Y"], prec, True)))
    d2 = host(plan2.phi_adj(dev(c["Y"], prec, True)))
    assert np.array_equal(d1, d2)
    assert rel(d1, a) <= (1e-14 if prec == "f64" else 1e-6)


@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("levels", [4, 2])
def test_psi_fwd_adj(prec, levels):
    c = _case("rect", prec)
    plan = make_plan(c, prec, levels=levels)
    A = host(plan.psi_fwd(dev(c["X"], prec)))
    refA = wavelets.psi_adjoint_cube(c["X"], levels)
    assert_close(A, refA, prec)
    B = np.random.default_rng(2).standard_normal(refA.shape)
    if prec == "f32":
        B = B.astype(np.float32).astype(np.float64)
    X = host(plan.psi_adj(dev(B, prec)))
    refX = wavelets.psi_cube(B, levels)
    assert_close(X, refX, prec)


@pytest.mark.parametrize("prec", PRECS)
def test_psi_256(prec):
    """256 x 256 at 3 levels: 64 level-0 tiles and 16 level-1 tiles per wavelet
    and channel, the chunked staging on every level."""
    rng = np.random.default_rng(21)
    c = rounded(dict(X=rng.uniform(0.0, 1.0, (2, 256, 256)), uv=np.zeros((1, 2)), Y=np.zeros(1, complex)), prec)
    from paper_1806_04596_gb300 import hypersara as hs
    plan = hs.Plan(256, 256, np.array([0, 1, 1]), dev(np.zeros((1, 2)), prec), levels=3, prec=prec)
    A = host(plan.psi_fwd(dev(c["X"], prec)))
    refA = wavelets.psi_adjoint_cube(c["X"], 3)
    assert_close(A, refA, prec)
    B = rng.standard_normal(refA.shape)
    if prec == "f32":
        B = B.astype(np.float32).astype(np.float64)
    X = host(plan.psi_adj(dev(B, prec)))
    refX = wavelets.psi_cube(B, 3)
    assert_close(X, refX, prec)


@pytest.mark.parametrize("prec", PRECS)
def test_psi_unaligned_buffers(prec):
    """Image and coefficient arrays starting one element past an aligned address
    are staged element by element; the results equal those of aligned buffers."""
    import torch
    c = _case("rect", prec)
    plan = make_plan(c, prec, levels=3)

    def shifted(t):
        s = torch.empty(t.numel() + 1, dtype=t.dtype, device=t.device)[1:].view_as(t)
        s.copy_(t)
        return s

    X = dev(c["X"], prec)
    A = plan.psi_fwd(X)
    assert np.array_equal(host(plan.psi_fwd(shifted(X))), host(A))
    assert np.array_equal(host(plan.psi_adj(shifted(A))), host(plan.psi_adj(A)))


def test_psi_small_levels_long_filters():
    """64 x 64 at 4 levels: the coarsest level is 8 x 8, shorter than db8."""
    c = _case("ragged64", "f64")
    plan = make_plan(c, "f64", levels=4)
    A = host(plan.psi_fwd(dev(c["X"], "f64")))
    assert rel(A, wavelets.psi_adjoint_cube(c["X"], 4)) <= 1e-12
    back = host(plan.psi_adj(dev(A, "f64")))
    assert rel(back, c["X"]) <= 1e-12


@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("dual", [False, True])
def test_prox_l21(prec, dual):
    c = _case("ragged64", prec)
    plan = make_plan(c, prec)
    rng = np.random.default_rng(3)
    A = rng.standard_normal((9, c["L"], c["ny"], c["nx"]))
    w = rng.uniform(0.0, 2.0, (9, c["ny"], c["nx"]))
    A[:, :, 0, 0] = 0.0   # zero rows
    if prec == "f32":
        A = A.astype(np.float32).astype(np.float64)
        w = w.astype(np.float32).astype(np.float64)
    thr = 1.3
    out = host(plan.prox_l21(dev(A, prec), thr, dev(w, prec), dual=dual))
    ref = prox.l21_dual(A, w, thr) if dual else prox.prox_l21(A, w, thr)
    assert_close(out, ref, prec)
    out1 = host(plan.prox_l21(dev(A, prec), thr, None, dual=dual))
    ref1 = prox.l21_dual(A, 1.0, thr) if dual else prox.prox_l21(A, 1.0, thr)
    assert_close(out1, ref1, prec)


@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("dual", [False, True])
@pytest.mark.parametrize("L", [4, 13])
def test_prox_nuclear(prec, dual, L):
    import torch
    c = _case("ragged64", prec)
    c = dict(c)
    c["L"] = L
    c["off"] = np.zeros(L + 1, dtype=np.int64)
    plan = make_plan(dict(c, uv=np.zeros((0, 2))), prec)
    rng = np.random.default_rng(4)
    # rank-3 signal plus small noise, positive like the cubes
    S = rng.uniform(0, 1, (3, c["ny"] * c["nx"]))
    H = rng.uniform(0.5, 1.5, (L, 3))
    X = (H @ S + 0.01 * rng.standard_normal((L, c["ny"] * c["nx"]))).reshape(L, c["ny"], c["nx"])
    if prec == "f32":
        X = X.astype(np.float32).astype(np.float64)
    w = np.linspace(0.5, 1.5, L)
    thr = 2.0
    out, sv = plan.prox_nuclear(dev(X, prec), thr, torch.tensor(w, dtype=torch.float64, device="cuda"),
                                dual=dual)
    out = host(out)
    ref_s = np.linalg.svd(X.reshape(L, -1).T, compute_uv=False)
    if dual:
        ref, _ = prox.nuclear_dual(X, w, thr)
    else:
        ref = prox.prox_nuclear(X, w, thr)
    tol = 1e-11 if prec == "f64" else 1e-5
    assert rel(out, ref) <= tol, rel(out, ref)
    assert np.max(np.abs(out - ref)) <= 10 * tol * np.max(np.abs(ref))
    svh = host(sv)
    if prec == "f64":
        assert rel(svh, ref_s) <= 1e-12
    else:
        # FP32 plans: singular values above the threshold are refined in FP64; the
        # others are resolved to the FP32 Gram eigen-precision, ~1e-7 sigma_max^2
        act = ref_s > thr * w * 1.01
        np.testing.assert_allclose(svh[act], ref_s[act], rtol=2e-6)
        assert np.max(np.abs(svh[~act] ** 2 - ref_s[~act] ** 2)) <= 4e-6 * ref_s[0] ** 2


@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("dual", [False, True])
def test_proj_l2ball(prec, dual):
    import torch
    c = _case("ragged64", prec)
    plan = make_plan(c, prec)
    rng = np.random.default_rng(5)
    M = int(c["off"][-1])
    Z = c["Y"]
    Yd = rng.standard_normal(M) + 1j * rng.standard_normal(M)
    if prec == "f32":
        Yd = Yd.astype(np.complex64).astype(np.complex128)
    # one channel inside its ball, others outside; the empty channel has norm 0
    eps = np.array([5.0, 1e6, 3.0, 10.0])
    out, rho = plan.proj_l2ball(dev(Z, prec, True), dev(Yd, prec, True),
                                torch.tensor(eps, dtype=torch.float64, device="cuda"), dual=dual)
    out = host(out)
    ref = np.empty_like(Z)
    for l in range(c["L"]):
        a, b = c["off"][l], c["off"][l + 1]
        ref[a:b] = prox.l2ball_dual(Z[a:b], Yd[a:b], eps[l]) if dual else \
            prox.proj_l2ball(Z[a:b], Yd[a:b], eps[l])
    assert_close(out, ref, prec)
    ref_rho = [np.linalg.norm(Z[c["off"][l]:c["off"][l + 1]] - Yd[c["off"][l]:c["off"][l + 1]])
               for l in range(c["L"])]
    np.testing.assert_allclose(host(rho), ref_rho, rtol=1e-12 if prec == "f64" else 1e-6)


@pytest.mark.parametrize("prec", PRECS)
def test_op_norm2(prec):
    """Power iteration against the exact spectral norm of the dense operator
    (built column by column with the oracle), uneven and empty channels."""
    c = rounded(ragged_case(n=16, L=3, M=(300, 0, 420), seed=14), prec)
    plan = make_plan(c, prec, levels=2)
    op = oracle_op(c)
    best = 0.0
    for ch in op.ch:
        if ch.M == 0:
            continue
        E = np.stack([ch.forward(e.reshape(16, 16)) for e in np.eye(256)], axis=1)
        best = max(best, np.linalg.norm(np.vstack([E.real, E.imag]), 2) ** 2)
    got = plan.op_norm2(iters=5000, tol=1e-13, seed=3)
    assert got == pytest.approx(best, rel=1e-7 if prec == "f64" else 1e-5)


@pytest.mark.parametrize("prec", PRECS)
def test_norm_l21(prec):
    c = _case("ragged64", prec)
    plan = make_plan(c, prec)
    A = np.random.default_rng(6).standard_normal((9, c["L"], c["ny"], c["nx"]))
    if prec == "f32":
        A = A.astype(np.float32).astype(np.float64)
    got = plan.norm_l21(dev(A, prec))
    assert got == pytest.approx(np.sum(prox.row_norms(A)), rel=1e-12 if prec == "f64" else 1e-6)


@pytest.mark.parametrize("prec", PRECS)
def test_time_stage_runs_every_stage(prec):
    c = _case("ragged64", prec)
    plan = make_plan(c, prec)
    X = dev(c["X"], prec)
    Y = dev(c["Y"], prec, True)
    Xo = plan.cube()
    A = plan.cube(9)
    io = {"fft_fwd": (X, None), "degrid": (None, Y), "grid": (Y, None), "fft_adj": (None, Xo),
          "psi_fwd": (X, A), "psi_adj": (A, Xo)}
    for name, (i, o) in io.items():
        assert plan.time_stage(name, i, o, reps=2) > 0.0
    # the stages compose to the operators: grid then adjoint FFT is phi_adj
    plan.time_stage("grid", Y, None, reps=1)
    plan.time_stage("fft_adj", None, Xo, reps=1)
    ref = host(plan.phi_adj(Y))
    assert rel(host(Xo), ref) <= (1e-14 if prec == "f64" else 1e-6)
