"""Oracle: a plain, slow FP64 CPU restatement of the HyperSARA primal-dual hot path.

TEST INFRASTRUCTURE ONLY. Only tests/, __graft_entry__.smoke() and bench.py's
cpu_baseline / reference leg may import, call or execute anything here. The
product path (the CUDA library and its Python binding) never does, and this
package never imports the product path. The two share no code: the only
common input is the seeded generator in the top-level `synth` module, which
holds none of the method's arithmetic.

Contents (each function cites the passage it follows):
  kaiser_bessel  interpolation kernel phi, its Fourier transform, the Z scaling
  nufft          Phi_l = Theta_l G_l F Z and its adjoint (Sec. 2.1, Eq. "inverse";
                 adjoint Sec. 3.2), direct NUDFT (Eq. "RIdata1", w = 0)
  wavelets       Daubechies 1-8 filters by spectral factorisation, periodic
                 orthonormal 2-D DWT, SARA dictionary Psi / Psi^dagger (Sec. 2.3)
  prox           positivity, nuclear, l2,1, l2-ball proximity operators and their
                 Moreau duals (Sec. 3.3, Eqs. "proj-plus", "prox-L*", "prox-L21", "md")
  pd             preconditioned primal-dual iteration (Algorithm 2, fixed bounds)
  problem        data synthesis y = Phi(X) + noise, sigma, epsilon, mu, kappa_3
  metrics        SNR_l and aSNR (Sec. 4.3)
  grad           gradient of 0.5 ||Phi X - y||^2 + ||Psi^dagger X||_{2,1}

Parity status: every function is pinned by tests in tests/test_oracle_*.py
(closed forms, brute force, invariants). The whole PD solve has no external
implementation to compare against; it is pinned through its components and the
monotone fixed-point residual of the iteration.
"""

from . import kaiser_bessel, nufft, wavelets, prox, pd, problem, metrics, grad  # noqa: F401
