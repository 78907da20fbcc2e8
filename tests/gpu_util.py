"""Shared helpers for the GPU parity tests: seeded cases, device transfer, and
error measures. Inputs of FP32 runs are rounded to FP32 first and the oracle
receives the same rounded values in FP64."""

from __future__ import annotations

import numpy as np

import synth
from oracle import nufft


def rel(a, b) -> float:
    a = np.asarray(a)
    b = np.asarray(b)
    nb = np.linalg.norm(b)
    return float(np.linalg.norm(a - b) / (nb if nb > 0 else 1.0))


def ragged_case(n=64, L=4, M=(2000, 1503, 0, 911), seed=123, nx=None, ny=None, uv_std=np.pi / 4):
    """Coverage with uneven (and empty) channels, scaled per channel like the paper's."""
    nx = nx or n
    ny = ny or n
    rng = np.random.Generator(np.random.PCG64(seed))
    freqs = synth.channel_freqs(L, 1.0, 2.0)
    pool = synth.uv_coverage(rng, max(M) if max(M) > 0 else 1, freqs, uv_std, np.pi)
    off = np.zeros(L + 1, dtype=np.int64)
    off[1:] = np.cumsum(M)
    uv = np.concatenate([pool[:M[l]] * freqs[l] / freqs[0] for l in range(L)], axis=0) \
        if off[-1] > 0 else np.zeros((0, 2))
    X = rng.uniform(0.0, 1.0, (L, ny, nx))
    Yr = rng.standard_normal(off[-1]) + 1j * rng.standard_normal(off[-1])
    return dict(nx=nx, ny=ny, L=L, off=off, uv=uv, X=X, Y=Yr, rng=rng)


def rounded(case, prec):
    """Round the case's inputs to the plan precision (returned in FP64)."""
    if prec == "f64":
        return case
    c = dict(case)
    c["uv"] = case["uv"].astype(np.float32).astype(np.float64)
    c["X"] = case["X"].astype(np.float32).astype(np.float64)
    c["Y"] = case["Y"].astype(np.complex64).astype(np.complex128)
    return c


def oracle_op(case):
    return nufft.WidebandOperator(case["nx"], case["ny"], case["uv"], case["off"])


def dev(arr, prec, complex_=False):
    import torch
    if complex_:
        dt = torch.complex64 if prec == "f32" else torch.complex128
    else:
        dt = torch.float32 if prec == "f32" else torch.float64
    return torch.tensor(np.ascontiguousarray(arr), dtype=dt, device="cuda")


def host(t) -> np.ndarray:
    import torch
    torch.cuda.synchronize()
    return t.detach().cpu().numpy().astype(np.complex128 if t.is_complex() else np.float64)


def make_plan(case, prec, levels=4, compensated=False, weights=None, precond=None):
    from paper_1806_04596_gb300 import hypersara as hs
    w = None if weights is None else dev(weights, prec)
    u = None if precond is None else dev(precond, prec)
    return hs.Plan(case["nx"], case["ny"], case["off"], dev(case["uv"], prec), weights=w, precond=u,
                   levels=levels, prec=prec, compensated=compensated)


TOL = {"f64": 1e-12, "f32": 1e-5}


def assert_close(out, ref, prec, elem=10.0):
    """Relative 2-norm within the precision's tolerance, and every element
    within elem * tolerance of the largest reference magnitude (so a few wrong
    entries cannot hide under the norm)."""
    out = np.asarray(out)
    ref = np.asarray(ref)
    r = rel(out, ref)
    assert r <= TOL[prec], r
    scale = float(np.max(np.abs(ref))) if ref.size else 0.0
    if ref.size:
        worst = float(np.max(np.abs(out - ref)))
        assert worst <= elem * TOL[prec] * (scale if scale > 0 else 1.0), (worst, scale)
