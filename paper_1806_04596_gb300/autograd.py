"""Differentiable operators of the HyperSARA hot path (torch.autograd).

The measurement operator Phi (Sec. 2.1, Eq. "inverse") and the SARA
dictionary Psi (Sec. 2.3) are linear, so each one's backward pass is its
adjoint, and both directions run in the library's kernels:

  phi(plan, X)            Y = Phi X        backward: Phi^dagger (gridding, F^H, Z^T, Re)
  phi_adj(plan, Y)        X = Phi^dagger Y backward: Phi (Z, F, de-gridding)
  psi_analysis(plan, X)   A = Psi^dagger X backward: Psi (synthesis kernels)
  psi_synthesis(plan, A)  X = Psi A        backward: Psi^dagger (analysis kernels)
  l21_norm(plan, A)       sum_n w_n ||a_n|| backward: w_n a_n / ||a_n|| (hs_l21_grad)

Gradients follow torch's convention for complex tensors (for a real loss,
grad = dL/dRe + i dL/dIm): the real-inner-product adjoint Phi^dagger y =
Re(Z^T F^H G^H Theta y) is then exactly the vector-Jacobian product of Phi.

`objective` is f(X) = 0.5 ||Phi X - y||^2 + ||Psi^dagger X||_{2,1}, and
`unrolled_pd` runs Algorithm 2 (fixed bounds, JAS or LRJAS priors) as a
differentiable function of the data y and the initial image, with
torch.utils.checkpoint over blocks of iterations so that only block
boundaries are kept for the backward pass. In the unrolled solve the linear
operators are the kernels above; the per-element and per-row nonlinearities
(positivity, l2,1 row scaling, l2-ball scaling, nuclear factor) are torch
expressions so that their derivatives come from autograd, and the nuclear
dual uses the library's Gram matrix (hs_gram) with a differentiable FP64
eigendecomposition of the L x L matrix.
"""

from __future__ import annotations

from typing import Optional

import torch

from . import hypersara as hs


def _c(t):
    return t if t.is_contiguous() else t.contiguous()


class _Phi(torch.autograd.Function):
    @staticmethod
    def forward(ctx, X, plan):
        ctx.plan = plan
        return plan.phi_fwd(_c(X))

    @staticmethod
    def backward(ctx, gY):
        return ctx.plan.phi_adj(_c(gY)), None


class _PhiAdj(torch.autograd.Function):
    @staticmethod
    def forward(ctx, Y, plan):
        ctx.plan = plan
        return plan.phi_adj(_c(Y))

    @staticmethod
    def backward(ctx, gX):
        return ctx.plan.phi_fwd(_c(gX)), None


class _PsiAnalysis(torch.autograd.Function):
    @staticmethod
    def forward(ctx, X, plan):
        ctx.plan = plan
        return plan.psi_fwd(_c(X))

    @staticmethod
    def backward(ctx, gA):
        return ctx.plan.psi_adj(_c(gA)), None


class _PsiSynthesis(torch.autograd.Function):
    @staticmethod
    def forward(ctx, A, plan):
        ctx.plan = plan
        return plan.psi_adj(_c(A))

    @staticmethod
    def backward(ctx, gX):
        return ctx.plan.psi_fwd(_c(gX)), None


class _L21Norm(torch.autograd.Function):
    @staticmethod
    def forward(ctx, A, plan, w_rows):
        ctx.plan, ctx.w_rows = plan, w_rows
        ctx.save_for_backward(A)
        val = plan.norm_l21(_c(A), w_rows)
        return torch.tensor(val, dtype=A.dtype, device=A.device)

    @staticmethod
    def backward(ctx, g):
        (A,) = ctx.saved_tensors
        d = ctx.plan.l21_grad(_c(A), ctx.w_rows)
        return d * g, None, None


class _Gram(torch.autograd.Function):
    """S = Z Z^T (L x L, FP64) of the channel-major cube Z; dZ = (dS + dS^T) Z."""

    @staticmethod
    def forward(ctx, Z, plan):
        ctx.save_for_backward(Z)
        return plan.gram(_c(Z))

    @staticmethod
    def backward(ctx, gS):
        (Z,) = ctx.saved_tensors
        L = Z.shape[0]
        G = (gS + gS.T).to(Z.dtype)
        return (G @ Z.reshape(L, -1)).reshape(Z.shape), None


def phi(plan: hs.Plan, X):
    return _Phi.apply(X, plan)


def phi_adj(plan: hs.Plan, Y):
    return _PhiAdj.apply(Y, plan)


def psi_analysis(plan: hs.Plan, X):
    return _PsiAnalysis.apply(X, plan)


def psi_synthesis(plan: hs.Plan, A):
    return _PsiSynthesis.apply(A, plan)


def l21_norm(plan: hs.Plan, A, w_rows=None):
    return _L21Norm.apply(A, plan, w_rows)


def gram(plan: hs.Plan, Z):
    return _Gram.apply(Z, plan)


def objective(plan: hs.Plan, X, Y, w_rows=None):
    """f(X) = 0.5 ||Phi X - Y||^2 + ||Psi^dagger X||_{2,1} (weighted by w_rows)."""
    r = phi(plan, X) - Y
    return 0.5 * torch.sum(r.real ** 2 + r.imag ** 2) + l21_norm(plan, psi_analysis(plan, X), w_rows)


# ------------------------------------------------------------ unrolled Algorithm 2
def _channel_ids(plan: hs.Plan, device):
    off = torch.tensor(plan.offsets, dtype=torch.int64)
    return torch.repeat_interleave(torch.arange(plan.L), off[1:] - off[:-1]).to(device)


def _ball_dual(vbar, Y, eps, ch, L):
    """v = vbar - P_B(vbar), one ball B(y_l, eps_l) per channel (Algorithm 2 step 11, U = I)."""
    d = vbar - Y
    n2 = torch.zeros(L, dtype=eps.dtype, device=d.device).index_add_(0, ch, (d.real ** 2 + d.imag ** 2).to(eps.dtype))
    nrm = torch.sqrt(n2)
    f = torch.where(nrm > eps, 1.0 - eps / torch.where(nrm > 0, nrm, torch.ones_like(nrm)),
                    torch.zeros_like(nrm))
    return d * f.to(d.real.dtype)[ch]


def _l21_dual(Q, lam):
    """Rows scaled by min(1, lam / ||q_n||) (Algorithm 2 step 7)."""
    nrm = torch.sqrt(torch.sum(Q * Q, dim=1, keepdim=True))
    f = torch.where(nrm > lam, lam / torch.where(nrm > 0, nrm, torch.ones_like(nrm)), torch.ones_like(nrm))
    return Q * f


def _nuclear_dual(plan, Z, thr):
    """Z V diag(min(1, thr / sigma_j)) V^T (Algorithm 2 step 5) from the Gram matrix."""
    L = Z.shape[0]
    S = gram(plan, Z)
    lam, V = torch.linalg.eigh(S)
    sig = torch.sqrt(torch.clamp(lam, min=0.0))
    f = torch.where(sig > thr, thr / torch.where(sig > 0, sig, torch.ones_like(sig)), torch.ones_like(sig))
    M = (V * f) @ V.T
    return (M.to(Z.dtype) @ Z.reshape(L, -1)).reshape(Z.shape)


def unrolled_pd(plan: hs.Plan, Y, eps, *, iters: int, mu: float, kappa3: float, tau: float = 0.33,
                use_nuclear: bool = False, X0: Optional[torch.Tensor] = None, checkpoint_every: int = 0):
    """`iters` iterations of Algorithm 2 (fixed bounds, U = I, unit weights,
    kappa_1 = kappa_2 = 1) as a differentiable function of Y (complex, caller
    order), eps (FP64 per channel) and the initial image X0. Returns X.
    checkpoint_every = k > 0 recomputes each block of k iterations in the
    backward pass instead of storing its intermediates."""
    L, ny, nx = plan.L, plan.ny, plan.nx
    dev = Y.device
    rdt = plan.rdtype
    ch = _channel_ids(plan, dev)
    X = torch.zeros((L, ny, nx), dtype=rdt, device=dev) if X0 is None else X0
    Xt = X
    P = torch.zeros_like(X)
    A = torch.zeros((9, L, ny, nx), dtype=rdt, device=dev)
    v = torch.zeros_like(Y)

    def step(X, Xt, P, A, v):
        if use_nuclear:
            P = _nuclear_dual(plan, P + Xt, 1.0)
        A = _l21_dual(A + psi_analysis(plan, Xt), mu)
        At = psi_synthesis(plan, A)
        v = _ball_dual(v + phi(plan, Xt), Y, eps, ch, L)
        G = At + kappa3 * phi_adj(plan, v)
        if use_nuclear:
            G = G + P
        Xn = torch.relu(X - tau * G)
        return Xn, 2.0 * Xn - X, P, A, v

    def block(k, X, Xt, P, A, v):
        for _ in range(k):
            X, Xt, P, A, v = step(X, Xt, P, A, v)
        return X, Xt, P, A, v

    done = 0
    while done < iters:
        k = min(checkpoint_every, iters - done) if checkpoint_every > 0 else iters - done
        if checkpoint_every > 0 and torch.is_grad_enabled():
            X, Xt, P, A, v = torch.utils.checkpoint.checkpoint(block, k, X, Xt, P, A, v, use_reentrant=False)
        else:
            X, Xt, P, A, v = block(k, X, Xt, P, A, v)
        done += k
    return X
