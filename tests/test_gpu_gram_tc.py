"""Gram matrix of the nuclear prox (Eq. "prox-L*", Algorithm 2 step 5) on the
tensor cores (FP32 plans: tcgen05 on exact BF16 digits), through the C ABI.

hs_gram is checked entry by entry against the FP64 product of the same
FP32-rounded cube, relative to sqrt(S_ii S_jj), for L from 1 to the maximum
64 (including L not a multiple of 8), grids whose 64-pixel chunks split
unevenly over the CTAs (4 to 1024 chunks), channels whose magnitudes differ by
six orders, an all-zero channel, Z = X + Xa (the form of the PD iteration),
the CUDA-core form of the same plan (HS_PLAN_GRAM_FMA) and a buffer one
element off the 16-byte alignment the tensor-core form needs (CUDA-core
fallback). The nuclear prox built on it is checked against the oracle, and
its singular values against the FP64 SVD."""

import numpy as np
import pytest

from gpu_util import dev, host
from oracle import prox

pytestmark = pytest.mark.gpu

GRAM_TOL = 2e-7      # |S - S_exact|_ij / sqrt(S_ii S_jj)


def _plan(nx, ny, L, gram_fma=False):
    import __graft_entry__ as ge
    ge.build()
    import torch
    from paper_1806_04596_gb300 import hypersara as hs
    off = np.zeros(L + 1, dtype=np.int64)
    return hs.Plan(nx, ny, off, torch.zeros((0, 2), dtype=torch.float32, device="cuda"), levels=1,
                   prec="f32", gram_fma=gram_fma)


def _cube(L, ny, nx, seed, spread=False, noise=0.02):
    rng = np.random.default_rng(seed)
    S = rng.uniform(0, 1, (4, ny * nx))
    H = rng.uniform(0.5, 1.5, (L, 4))
    X = H @ S + noise * rng.standard_normal((L, ny * nx))
    if spread:   # channel magnitudes over six orders, one channel zero
        X *= 10.0 ** rng.uniform(-3, 3, (L, 1))
        X[L // 2] = 0.0
    return X.reshape(L, ny, nx).astype(np.float32).astype(np.float64)


def _gram_err(S, Z):
    Zm = Z.reshape(Z.shape[0], -1)
    ref = Zm @ Zm.T
    d = np.sqrt(np.diag(ref))
    den = np.outer(d, d)
    den[den == 0] = 1.0
    return np.max(np.abs(S - ref) / den)


@pytest.mark.parametrize("nx,ny", [(16, 16), (64, 32), (256, 256)])
@pytest.mark.parametrize("L", [1, 3, 60, 64])
def test_gram_matches_fp64_product(cuda_device, nx, ny, L):
    X = _cube(L, ny, nx, seed=nx + L, spread=L > 1)
    for fma in (False, True):
        plan = _plan(nx, ny, L, gram_fma=fma)
        S = host(plan.gram(dev(X, "f32")))
        plan.check()
        assert _gram_err(S, X) <= GRAM_TOL, fma
        assert np.array_equal(S, S.T)


@pytest.mark.parametrize("L", [5, 64])
def test_gram_of_sum(cuda_device, L):
    """Z = X + Xa formed in FP32 inside the kernel, as the PD iteration uses it."""
    nx = ny = 128
    X = _cube(L, ny, nx, seed=11)
    Xa = _cube(L, ny, nx, seed=12) - 0.5
    Z = (X.astype(np.float32) + Xa.astype(np.float32)).astype(np.float64)
    plan = _plan(nx, ny, L)
    S = host(plan.gram(dev(X, "f32"), dev(Xa, "f32")))
    plan.check()
    assert _gram_err(S, Z) <= GRAM_TOL


def test_unaligned_buffer_falls_back(cuda_device):
    import torch
    L, nx, ny = 12, 64, 64
    X = _cube(L, ny, nx, seed=3)
    plan = _plan(nx, ny, L)
    flat = torch.zeros(L * nx * ny + 1, dtype=torch.float32, device="cuda")
    flat[1:] = dev(X, "f32").reshape(-1)
    Xv = flat[1:].view(L, ny, nx)                       # 4 bytes off a 16-byte boundary
    S = host(plan.gram(Xv))
    plan.check()
    assert _gram_err(S, X) <= GRAM_TOL


@pytest.mark.parametrize("L", [8, 60, 64])
@pytest.mark.parametrize("dual", [False, True])
def test_nuclear_prox_on_tensor_core_gram(cuda_device, L, dual):
    """Rank-4 cube plus noise whose singular values (about 0.64) stay clear of
    the thresholds 1.5 .. 4.5: the prox is then well conditioned."""
    import torch
    nx = ny = 128
    X = _cube(L, ny, nx, seed=7 * L, noise=0.005)
    w = np.linspace(0.5, 1.5, L)
    thr = 3.0
    plan = _plan(nx, ny, L)
    out, sv = plan.prox_nuclear(dev(X, "f32"), thr, torch.tensor(w, dtype=torch.float64, device="cuda"),
                                dual=dual)
    plan.check()
    out = host(out)
    ref = prox.nuclear_dual(X, w, thr)[0] if dual else prox.prox_nuclear(X, w, thr)
    # the dual form is X - prox(X), much smaller than X here: its FP32 error is
    # bounded relative to the input, the prox form's relative to itself
    scale = X if dual else ref
    assert np.linalg.norm(out - ref) <= 1e-5 * np.linalg.norm(scale)
    assert np.max(np.abs(out - ref)) <= 1e-5 * np.max(np.abs(scale))
    s = host(sv)
    ref_s = np.linalg.svd(X.reshape(L, -1).T, compute_uv=False)
    assert abs(s[0] - ref_s[0]) <= 1e-6 * ref_s[0]
    assert np.max(np.abs(s ** 2 - ref_s ** 2)) <= 4e-6 * ref_s[0] ** 2
