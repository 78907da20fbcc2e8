"""Re-weighting outer loop of HyperSARA (Sec. 3.5, Algorithm 1) - test
infrastructure only, like the rest of `oracle/`.

Weights (Sec. 3.5, Eqs. "weights-l21" and "weights-n"):
  l2,1:    w_n = gamma_bar / (gamma_bar + ||(Psi^dagger X)_n||_2), n a row
           (basis d, pixel) of the coefficient cube, the norm taken across the
           L channels;
  nuclear: w_j = gamma / (gamma + sigma_j(X)), sigma_j the singular values of
           the N x L matrix X in descending order.

Readings (the paper fixes neither): gamma and gamma_bar start at 1 and the
weights computed after outer iteration k use the current values, which are then
multiplied by the decay factor (0.8, inside the paper's 0.5-0.9); the first
inner loop runs with unit weights ("starting from weights equal to 1"); each
inner loop starts from the previous one's primal and dual variables.
"""

from __future__ import annotations

import dataclasses

import numpy as np

from . import pd, prox, wavelets


def weights_l21(X: np.ndarray, levels: int, gamma_bar: float) -> np.ndarray:
    """(9, ny, nx) row weights from Psi^dagger X (X is L x ny x nx)."""
    A = wavelets.psi_adjoint_cube(X, levels)
    return gamma_bar / (gamma_bar + prox.row_norms(A))


def weights_l1(X: np.ndarray, levels: int, gamma_bar: float) -> np.ndarray:
    """(9, L, ny, nx) per-coefficient weights of the SARA prior (the l1 analogue
    of Eq. "weights-l21": each coefficient on its own)."""
    A = wavelets.psi_adjoint_cube(X, levels)
    return gamma_bar / (gamma_bar + np.abs(A))


def weights_nuclear(X: np.ndarray, gamma: float) -> np.ndarray:
    """(L,) weights from the singular values of the N x L matrix of X."""
    L = X.shape[0]
    s = np.linalg.svd(X.reshape(L, -1).T, compute_uv=False)
    return gamma / (gamma + s)


def reweighted_solve(op, y, eps, prm: pd.PDParams, outer: int, inner: int, decay: float = 0.8,
                     U=None, state: pd.PDState | None = None):
    """Algorithm 1: `outer` re-weights of `inner` PD iterations each.
    Returns (state, w_l21, w_nuc) after the last weight update."""
    st = state if state is not None else pd.init_state(op.L, op.ny, op.nx, int(op.offsets[-1]))
    gamma = gamma_bar = 1.0
    p = prm
    w21 = wn = None
    for _ in range(outer):
        st = pd.pd_solve(op, y, eps, p, inner, U=U, state=st)
        if prm.sparsity == "l1":
            w21 = weights_l1(st.X, prm.levels, gamma_bar)
        else:
            w21 = weights_l21(st.X, prm.levels, gamma_bar)
        wn = weights_nuclear(st.X, gamma)
        p = dataclasses.replace(prm, w_l21=w21, w_nuc=wn)
        gamma *= decay
        gamma_bar *= decay
    return st, w21, wn
