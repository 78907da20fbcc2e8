"""Pins for the oracle's primal-dual iteration (Algorithm 2, Sec. 3.4).

* The PD iteration with kappa_1 = 1, kappa_2 = 1/||Psi||^2, kappa_3 = 1/||Phi||^2
  and tau < 1/3 is a proximal-point step in the metric
  M = [[I/tau, -K^*], [-K, diag(1/kappa_i)]]; consecutive pairs (X^{t-1}, D^t)
  therefore have a nonincreasing M-norm difference. A wrong update order, sign
  or threshold can break this.
* With both priors off, full Fourier sampling and a tight bound, the problem
  reduces to finding a positive image consistent with the data; the exact
  image is recovered.
* The solve drives every channel residual toward its l2 ball.
* SNR / aSNR closed forms (Sec. 4.3)."""

import numpy as np
import pytest

import synth
from oracle import metrics, nufft, pd, problem, prox, wavelets


def _small_problem(n=16, L=3, M=120, seed=77):
    inp = synth.make_inputs(1, n=n, L=L, M=M, seed=seed)
    prob = problem.make_problem(inp)
    return inp, prob


def test_snr_closed_form():
    x = np.ones((4, 4))
    xh = x * 0.9
    assert metrics.snr(x, xh) == pytest.approx(20.0, abs=1e-12)
    X = np.stack([x, x])
    Xh = np.stack([x * 0.9, x * 0.99])
    assert metrics.asnr(X, Xh) == pytest.approx(30.0, abs=1e-12)


def test_generator_shapes_and_scaling():
    inp = synth.make_inputs(1)
    assert inp.truth.shape == (4, 64, 64)
    assert inp.truth.max() == pytest.approx(1.0)
    assert np.all(inp.truth >= 0)
    assert inp.uv.shape == (8000, 2)
    assert np.max(np.abs(inp.uv)) < np.pi
    # rank <= Q = 3
    s = np.linalg.svd(inp.truth.reshape(4, -1), compute_uv=False)
    assert s[3] <= 1e-12 * s[0]
    # channel l is channel 0 scaled by nu_l / nu_0
    M = 2000
    np.testing.assert_allclose(inp.uv[M:2 * M], inp.uv[:M] * inp.freqs[1] / inp.freqs[0])


def test_noise_level_matches_input_snr():
    inp, prob = _small_problem(M=4000, L=2)
    y_clean = prob.op.forward(prob.truth)
    snr_in = 20 * np.log10(np.linalg.norm(y_clean) / np.linalg.norm(prob.y - y_clean))
    assert snr_in == pytest.approx(inp.insnr, abs=0.3)
    # the chi-square bound holds for the drawn noise with high probability
    for l in range(2):
        a, b = inp.offsets[l], inp.offsets[l + 1]
        assert np.linalg.norm(prob.y[a:b] - y_clean[a:b]) <= prob.eps[l]


def test_fixed_point_residual_nonincreasing():
    inp, prob = _small_problem()
    op = prob.op
    mu = problem.estimate_mu(op, prob.y, levels=2)
    k3 = 1.0 / problem.op_norm2(op)
    prm = pd.PDParams(mu=mu, tau=0.33, kappa3=k3, levels=2)
    hist = []
    pd.pd_solve(op, prob.y, prob.eps, prm, 40,
                callback=lambda s: hist.append((s.X.copy(), s.P.copy(), s.A.copy(), s.v.copy())))
    # pairs z_t = (X^{t-1}, D^t)
    X0 = np.zeros_like(hist[0][0])
    Xs = [X0] + [h[0] for h in hist]
    res = []
    for t in range(1, len(hist)):
        dX = Xs[t] - Xs[t - 1]
        dP = hist[t][1] - hist[t - 1][1]
        dA = hist[t][2] - hist[t - 1][2]
        dv = hist[t][3] - hist[t - 1][3]
        res.append(pd.metric_norm2(dX, dP, dA, dv, op, prm))
    res = np.array(res)
    assert np.all(res >= -1e-12 * res[0])
    assert np.all(res[1:] <= res[:-1] * (1 + 1e-9) + 1e-14 * res[0])
    assert res[-1] < res[0]


def test_full_sampling_no_priors_recovers_image():
    n = 8
    g = (np.arange(n) - n // 2) * 2 * np.pi / n
    uu, vv = np.meshgrid(g, g)
    uv = np.stack([uu.ravel(), vv.ravel()], axis=1)
    rng = np.random.default_rng(3)
    x_true = rng.uniform(0.2, 1.0, (1, n, n))
    op = nufft.WidebandOperator(n, n, uv, np.array([0, n * n]))
    y = op.forward(x_true)
    eps = np.array([1e-7 * np.linalg.norm(y)])
    prm = pd.PDParams(mu=0.0, tau=0.33, kappa3=1.0 / problem.op_norm2(op), levels=1,
                      use_nuclear=False, use_l21=False)
    st = pd.pd_solve(op, y, eps, prm, 3000)
    assert np.linalg.norm(st.X - x_true) <= 1e-4 * np.linalg.norm(x_true)


@pytest.mark.slow
def test_solve_approaches_data_fidelity_and_snr():
    """Channel residuals shrink toward their l2 bounds and the cube is recovered.
    (Unpreconditioned PD approaches the ball slowly: ~10% above epsilon after
    200 iterations on this problem, ~1.5% after 1200.)"""
    inp = synth.make_inputs(1, n=32, L=4, M=1500)
    prob = problem.make_problem(inp)
    op = prob.op
    mu = problem.estimate_mu(op, prob.y, levels=3)
    prm = pd.PDParams(mu=mu, tau=0.33, kappa3=1.0 / problem.op_norm2(op), levels=3)

    def ratios(st):
        r = prob.y - op.forward(st.X)
        return np.array([np.linalg.norm(r[op.offsets[l]:op.offsets[l + 1]]) / prob.eps[l]
                         for l in range(op.L)])

    st1 = pd.pd_solve(op, prob.y, prob.eps, prm, 100)
    r1 = ratios(st1)
    st2 = pd.pd_solve(op, prob.y, prob.eps, prm, 100, state=st1)
    r2 = ratios(st2)
    assert np.all(r2 < r1)
    assert np.all(r2 < 1.2)
    assert metrics.asnr(prob.truth, st2.X) > 35.0
    assert np.all(st2.X >= 0)


def test_opnorm_matches_dense_operator():
    inp, prob = _small_problem()
    op = prob.op
    # power iteration against the dense operator's largest singular value
    n = op.nx
    best = 0.0
    for ch in op.ch:
        E = np.zeros((ch.M, n * n), dtype=complex)
        for k in range(n * n):
            e = np.zeros(n * n)
            e[k] = 1
            E[:, k] = ch.forward(e.reshape(n, n))
        Er = np.vstack([E.real, E.imag])
        best = max(best, np.linalg.norm(Er, 2) ** 2)
    assert problem.op_norm2(op) == pytest.approx(best, rel=1e-8)


def _density_precond(op):
    """U_m = 1 / (visibilities of the channel in the same cell of the
    oversampled grid): uniform-weighting density, not constant."""
    U = np.empty(int(op.offsets[-1]))
    for l, ch in enumerate(op.ch):
        cell = ch.iy[:, 3] * ch.Kx + ch.ix[:, 3]
        _, inv, cnt = np.unique(cell, return_inverse=True, return_counts=True)
        U[op.offsets[l]:op.offsets[l + 1]] = 1.0 / cnt[inv]
    return U


def test_constant_preconditioner_is_a_rescaled_problem():
    """U = c I on (y, eps) is the unpreconditioned iteration on (y / sqrt(c),
    eps / sqrt(c)): v = c u at every step, ||U^{1/2} Phi||^2 = c ||Phi||^2, and
    the primal iterates coincide."""
    inp, prob = _small_problem()
    op = prob.op
    c = 3.7
    U = np.full(int(op.offsets[-1]), c)
    n2 = problem.op_norm2(op)
    assert problem.op_norm2(op, U) == pytest.approx(c * n2, rel=1e-8)
    mu = problem.estimate_mu(op, prob.y, levels=2)
    prm_u = pd.PDParams(mu=mu, tau=0.33, kappa3=1.0 / (c * n2), levels=2)
    prm_1 = pd.PDParams(mu=mu, tau=0.33, kappa3=1.0 / n2, levels=2)
    su = pd.pd_solve(op, prob.y, prob.eps, prm_u, 25, U=U)
    s1 = pd.pd_solve(op, prob.y / np.sqrt(c), prob.eps / np.sqrt(c), prm_1, 25)
    np.testing.assert_allclose(su.X, s1.X, rtol=1e-10, atol=1e-13 * np.abs(s1.X).max())
    np.testing.assert_allclose(su.v, c * s1.v, rtol=1e-10, atol=1e-13 * np.abs(su.v).max())


def test_preconditioned_fixed_point_residual_nonincreasing():
    """Non-constant diagonal U (density weights): the iteration is the
    unpreconditioned one on U^{1/2} Phi, so its residual in that problem's PD
    metric is nonincreasing."""
    inp, prob = _small_problem(M=300)
    op = prob.op
    U = _density_precond(op)
    assert U.min() < 1.0 and U.max() == 1.0
    mu = problem.estimate_mu(op, prob.y, levels=2)
    k3 = 1.0 / problem.op_norm2(op, U)
    prm = pd.PDParams(mu=mu, tau=0.33, kappa3=k3, levels=2)
    hist = []
    pd.pd_solve(op, prob.y, prob.eps, prm, 40, U=U,
                callback=lambda s: hist.append((s.X.copy(), s.P.copy(), s.A.copy(), s.v.copy())))
    Xs = [np.zeros_like(hist[0][0])] + [h[0] for h in hist]
    res = []
    for t in range(1, len(hist)):
        res.append(pd.metric_norm2(Xs[t] - Xs[t - 1], hist[t][1] - hist[t - 1][1],
                                   hist[t][2] - hist[t - 1][2], hist[t][3] - hist[t - 1][3],
                                   op, prm, U=U))
    res = np.array(res)
    assert np.all(res >= -1e-12 * res[0])
    assert np.all(res[1:] <= res[:-1] * (1 + 1e-9) + 1e-14 * res[0])
    assert res[-1] < 0.5 * res[0]
