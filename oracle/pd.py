"""Preconditioned primal-dual iteration, Algorithm 2 with fixed l2 bounds.

Reading (checked against the Condat-Vu condition of Sec. 3.4): the dual
variables are the paper's scaled ones, so that with kappa_1 = 1,
kappa_2 = 1 / ||Psi^dagger||^2 and kappa_3 = 1 / ||U^{1/2} Phi||^2 the updates are

  step 4   u_l   = F Z x~_l                      (inside Phi below)
  step 5   P     = (I - S*_w)(P + X~)
  step 7   A_d   = (I - S^{l21}_{w mu ||Psi||^2})(A_d + Psi_d^dagger X~)
  step 8   A~    = sum_d Psi_d A_d
  step 10  vbar  = v + U Theta G u = v + U Phi_l x~_l
  step 11  v     = U^{1/2} (I - P_B(y, eps)) (U^{-1/2} vbar)
  step 12/20  G  = kappa_1 P + kappa_2 A~ + kappa_3 Phi^dagger v
  step 21  X     = P_+(X - tau G)
  step 22  X~    = 2 X - X_prev
  step 23  beta  = ||X - X_prev|| / ||X||

Variants of Sec. 4.2 through the flags: LR (use_l21 = False), JAS
(use_nuclear = False), and SARA (use_nuclear = False, sparsity = "l1": step 7
with the per-coefficient l1 dual (I - S^{l1}) in place of the l2,1 one, which
decouples the channels into L single-channel problems).

Data blocks (Sec. 2.1, M_l^b): `blocks` are offsets into the visibility
vector (caller order) containing every channel boundary; each block has its
own bound epsilon_l^b and ball projection (steps 10-11). Without blocks, one
block per channel.

Adaptive bounds (steps 13-19, Sec. 3.6), enabled by `adapt`: with
rho_b = ||y_b - Phibar_b X~^{(t-1)}|| (the data residual of the block at the
extrapolated image this iteration uses), if beta^{(t-1)} < lambda_1 and
t - vartheta_b > vartheta_bar and |rho_b - eps_b| / eps_b > lambda_2 then
eps_b <- lambda_3 rho_b + (1 - lambda_3) eps_b and vartheta_b <- t. Readings:
t counts iterations from 1, vartheta starts at 0, beta^{(0)} is undefined (the
first iteration never adjusts), and the new bounds serve from the next
iteration (step 11 uses eps^{(t-1)}).

Initial state: everything zero (the paper's "Given" does not fix it). By
default the bounds stay fixed (as in the paper's simulations, Sec. 4.1) and
there is one data block per channel (M_l^b = I); `adapt` and `blocks` above
switch on steps 13-19 and several blocks per channel.

Preconditioning (Sec. 3.3): with diagonal U the data-term updates are exactly
the unpreconditioned ones applied to the operator U^{1/2} Phi, written in the
variable v = U^{1/2} w of that problem's dual w; kappa_3 = 1 / ||U^{1/2} Phi||^2
keeps the Condat-Vu condition of Sec. 3.4.
"""

from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

from . import prox, wavelets


@dataclass
class PDParams:
    mu: float
    tau: float = 0.33
    kappa1: float = 1.0
    kappa2: float = 1.0            # 1 / ||Psi^dagger||^2 = 1 for the normalised frame
    kappa3: float = 1.0
    psi_norm2: float = 1.0         # ||Psi^dagger||_S^2
    levels: int = 4
    w_nuc: object = 1.0            # scalar or (L,) nuclear weights
    w_l21: object = 1.0            # scalar or (9, ny, nx) l2,1 row weights
    use_nuclear: bool = True
    use_l21: bool = True
    sparsity: str = "l21"          # "l21" (joint, rows across channels) or "l1" (per channel, SARA)


@dataclass
class AdaptParams:
    """Steps 13-19 (values of Sec. 3.6 / Appendix A used in the paper's runs)."""
    lambda1: float = 5e-4
    lambda2: float = 0.01
    lambda3: float = 0.618
    min_gap: int = 100             # vartheta_bar


@dataclass
class PDState:
    X: np.ndarray
    Xt: np.ndarray
    P: np.ndarray
    A: np.ndarray
    v: np.ndarray
    t: int = 0
    beta: float = float("nan")
    rho: np.ndarray = field(default_factory=lambda: np.zeros(0))
    eps: np.ndarray | None = None      # current bounds per block (adaptive runs)
    theta: np.ndarray | None = None    # iteration of each block's last bound update
    resid: np.ndarray = field(default_factory=lambda: np.zeros(0))


def init_state(L: int, ny: int, nx: int, M_total: int) -> PDState:
    z = np.zeros((L, ny, nx))
    return PDState(X=z.copy(), Xt=z.copy(), P=z.copy(),
                   A=np.zeros((wavelets.N_BASES, L, ny, nx)),
                   v=np.zeros(M_total, dtype=np.complex128))


def pd_step(st: PDState, op, y: np.ndarray, eps: np.ndarray, prm: PDParams, U=None, blocks=None,
            adapt: AdaptParams | None = None) -> PDState:
    """One iteration of Algorithm 2 (returns a new state). eps: one bound per
    block (per channel without blocks); with `adapt` the state carries the
    current bounds."""
    L = st.X.shape[0]
    Xt = st.Xt
    # step 5: low rankness dual
    if prm.use_nuclear:
        P, _ = prox.nuclear_dual(st.P + Xt, prm.w_nuc, 1.0 / prm.kappa1)
    else:
        P = np.zeros_like(st.P)
    # steps 7-8: joint average sparsity dual and its synthesis
    if prm.use_l21:
        Q = st.A + wavelets.psi_adjoint_cube(Xt, prm.levels)
        if prm.sparsity == "l1":
            A = prox.l1_dual(Q, prm.w_l21, prm.mu * prm.psi_norm2)
        else:
            A = prox.l21_dual(Q, prm.w_l21, prm.mu * prm.psi_norm2)
        At = wavelets.psi_cube(A, prm.levels)
    else:
        A = np.zeros_like(st.A)
        At = np.zeros_like(st.X)
    # steps 4, 10-12: data fidelity duals, one ball per block
    PhiXt = op.forward(Xt)
    bo = np.asarray(op.offsets if blocks is None else blocks)
    nb = len(bo) - 1
    eps_cur = np.asarray(eps, dtype=np.float64) if st.eps is None else st.eps
    v = np.empty_like(st.v)
    rho = np.empty(nb)
    resid = np.empty(nb)
    for k in range(nb):
        a, b = bo[k], bo[k + 1]
        Ul = None if U is None else U[a:b]
        vbar = st.v[a:b] + (PhiXt[a:b] if Ul is None else Ul * PhiXt[a:b])
        z = vbar if Ul is None else vbar / np.sqrt(Ul)
        rho[k] = np.sqrt(np.sum(np.abs(z - y[a:b]) ** 2))
        resid[k] = np.sqrt(np.sum(np.abs(y[a:b] - PhiXt[a:b]) ** 2))
        v[a:b] = prox.l2ball_dual(vbar, y[a:b], eps_cur[k], Ul)
    # steps 13-19: adjust the bounds (used from the next iteration)
    t = st.t + 1
    eps_new, theta = eps_cur, st.theta
    if adapt is not None:
        theta = np.zeros(nb, dtype=np.int64) if st.theta is None else st.theta.copy()
        eps_new = eps_cur.copy()
        for k in range(nb):
            if (st.beta < adapt.lambda1 and t - theta[k] > adapt.min_gap
                    and abs(resid[k] - eps_cur[k]) / eps_cur[k] > adapt.lambda2):
                eps_new[k] = adapt.lambda3 * resid[k] + (1.0 - adapt.lambda3) * eps_cur[k]
                theta[k] = t
    # steps 20-23: primal update
    Gd = op.adjoint(v)
    G = prm.kappa1 * P + prm.kappa2 * At + prm.kappa3 * Gd
    Xn = prox.proj_positive(st.X - prm.tau * G)
    Xtn = 2.0 * Xn - st.X
    nx_ = np.sqrt(np.sum(Xn * Xn))
    beta = np.sqrt(np.sum((Xn - st.X) ** 2)) / nx_ if nx_ > 0 else float("inf")
    return PDState(X=Xn, Xt=Xtn, P=P, A=A, v=v, t=t, beta=beta, rho=rho,
                   eps=eps_new if adapt is not None else st.eps, theta=theta, resid=resid)


def pd_solve(op, y, eps, prm: PDParams, iters: int, U=None, state: PDState | None = None,
             callback=None, blocks=None, adapt: AdaptParams | None = None) -> PDState:
    st = state if state is not None else init_state(op.L, op.ny, op.nx, int(op.offsets[-1]))
    for _ in range(iters):
        st = pd_step(st, op, y, eps, prm, U, blocks, adapt)
        if callback is not None:
            callback(st)
    return st


def metric_norm2(dX, dP, dA, dv, op, prm: PDParams, U=None) -> float:
    """Squared norm of a state difference in the primal-dual metric
        M = [[I / tau, -K^*], [-K, diag(1 / sigma_i)]],  K = [I; Psi^dagger; U^{1/2} Phi],
    written for the scaled duals (y_i = kappa_i D_i, sigma_i = kappa_i):
        ||dX||^2 / tau - 2 sum_i kappa_i <K_i dX, dD_i> + sum_i kappa_i ||dD_i||^2.
    The data dual of the U^{1/2} Phi problem is w = U^{-1/2} v, so its terms are
    ||U^{-1/2} dv||^2 - 2 Re<Phi dX, dv>. The iteration is a proximal-point step
    in M, so the residual between consecutive pairs (X^{t-1}, D^t) is
    nonincreasing."""
    s = np.sum(dX * dX) / prm.tau
    s += prm.kappa1 * (np.sum(dP * dP) - 2.0 * np.sum(dX * dP))
    KdX = wavelets.psi_adjoint_cube(dX, prm.levels)
    s += prm.kappa2 * (np.sum(dA * dA) - 2.0 * np.sum(KdX * dA))
    PhidX = op.forward(dX)
    dv2 = np.abs(dv) ** 2 if U is None else np.abs(dv) ** 2 / np.asarray(U, dtype=np.float64)
    s += prm.kappa3 * (np.sum(dv2) - 2.0 * np.sum(np.real(np.conj(PhidX) * dv)))
    return float(s)
