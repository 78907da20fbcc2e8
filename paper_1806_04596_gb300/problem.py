"""Synthetic problem set-up on the device with the library's own operators.

Given the seeded random inputs (truth cube, uv coverage, unit noise draws from
the `synth` module), this builds the measurement plan and computes, on the
GPU:
  y = Phi(X_true) + sigma * noise, sigma from the input SNR on the whole cube,
  eps_l = sigma sqrt(M_l + 2 sqrt(M_l))         (chi-square mean + 2 std),
  X_dirty,l = eta_l Phi_l^dagger y_l,  eta_l = 1 / max(Phi_l^dagger Phi_l delta),
  mu = ||X_dirty||_* / ||Psi^dagger X_dirty||_{2,1}                (Sec. 2.3),
  kappa_3 = 1 / max_l ||U_l^{1/2} Phi_l||^2 by power iteration    (Sec. 3.4).
mu (the dirty cube's PSF normalisation, nuclear and l2,1 norms) comes from
hs_estimate_mu; the noise level sigma is the norm of the clean visibilities (a
torch reduction: part of synthesising the data); every operator application is
a library call.
"""

from __future__ import annotations

from dataclasses import dataclass

import numpy as np

from . import hypersara as hs


@dataclass
class DeviceProblem:
    plan: hs.Plan
    truth: object      # CUDA tensor (L, ny, nx)
    y: object          # CUDA complex tensor (M,)
    eps: object        # CUDA float64 tensor (L,)
    sigma: float
    mu: float
    kappa3: float
    op_norm2: float


def build(inp, prec: str = "f32", levels: int = 4, compensated: bool = False,
          power_iters: int = 200, power_tol: float = 1e-6) -> DeviceProblem:
    import torch
    rdt = torch.float32 if prec == "f32" else torch.float64
    cdt = torch.complex64 if prec == "f32" else torch.complex128
    uv = torch.tensor(inp.uv, dtype=rdt, device="cuda")
    plan = hs.Plan(inp.nx, inp.ny, inp.offsets, uv, levels=levels, prec=prec, compensated=compensated)
    X = torch.tensor(inp.truth, dtype=rdt, device="cuda")
    y = plan.phi_fwd(X)
    M = int(inp.offsets[-1])
    nrm = float(torch.linalg.vector_norm(y.to(torch.complex128)))
    sigma = nrm / np.sqrt(max(M, 1)) * 10.0 ** (-inp.insnr / 20.0)
    y = y + (sigma * torch.tensor(inp.noise, dtype=torch.complex128, device="cuda")).to(cdt)
    Ml = np.diff(inp.offsets).astype(np.float64)
    eps = torch.tensor(sigma * np.sqrt(Ml + 2.0 * np.sqrt(Ml)), dtype=torch.float64, device="cuda")
    # mu from the dirty cube (PSF normalisation, nuclear and l2,1 norms: hs_estimate_mu)
    mu = plan.estimate_mu(y)[0] if plan.L <= 64 else 0.0
    on2 = plan.op_norm2(iters=power_iters, tol=power_tol, seed=0)
    torch.cuda.synchronize()
    return DeviceProblem(plan=plan, truth=X, y=y, eps=eps, sigma=sigma, mu=mu,
                         kappa3=1.0 / on2 if on2 > 0 else 1.0, op_norm2=on2)
