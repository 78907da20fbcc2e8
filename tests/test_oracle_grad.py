"""Pins for the oracle's objective gradient (oracle/grad.py): central finite
differences of the objective along random directions (FP64, tiny problem),
each term on its own and together, and the l2,1 term's closed form on a cube
whose coefficient rows have known norms (a constant image: only the coarsest
approximation band is non-zero)."""

import numpy as np
import pytest

import synth
from oracle import grad, nufft, problem, wavelets


def _setup(n=16, L=3, M=150, seed=5):
    inp = synth.make_inputs(1, n=n, L=L, M=M, seed=seed)
    prob = problem.make_problem(inp)
    rng = np.random.default_rng(seed)
    X = rng.uniform(0.0, 1.0, (L, n, n))
    return prob.op, prob.y, X, rng


@pytest.mark.parametrize("levels", [1, 2])
def test_gradient_matches_central_differences(levels):
    op, y, X, rng = _setup()
    g = grad.gradient(op, X, y, levels)
    for _ in range(4):
        D = rng.standard_normal(X.shape)
        h = 1e-5
        fd = (grad.objective(op, X + h * D, y, levels) - grad.objective(op, X - h * D, y, levels)) / (2 * h)
        assert np.sum(g * D) == pytest.approx(fd, rel=1e-7, abs=1e-9)


def test_data_term_alone_is_adjoint_of_residual():
    op, y, X, rng = _setup()
    D = rng.standard_normal(X.shape)
    h = 1e-5
    f = lambda Z: 0.5 * np.sum(np.abs(op.forward(Z) - y) ** 2)   # noqa: E731
    fd = (f(X + h * D) - f(X - h * D)) / (2 * h)
    g = op.adjoint(op.forward(X) - y)
    assert np.sum(g * D) == pytest.approx(fd, rel=1e-8)


def test_l21_term_on_constant_image():
    """X = c 1 (x) h: Psi^dagger X has non-zero rows only in the Dirac basis
    (n^2 rows of norm c ||h|| / 3) and in the coarsest band of each wavelet
    ((n / 2^levels)^2 rows of norm 2^levels c ||h|| / 3), so the l2,1 norm is
    closed form; the term is 1-homogeneous, so <grad, X> equals it (Euler)."""
    n, L, levels = 16, 4, 2
    h = np.array([1.0, 0.5, -0.25, 2.0])
    X = 0.7 * h[:, None, None] * np.ones((n, n))[None]
    A = wavelets.psi_adjoint_cube(X, levels)
    nrm = 0.7 * np.linalg.norm(h)
    expect = (n * n * nrm + 8 * (n / 2 ** levels) ** 2 * 2 ** levels * nrm) / 3.0
    assert np.sum(np.sqrt(np.sum(A * A, axis=1))) == pytest.approx(expect, rel=1e-12)
    op = nufft.WidebandOperator(n, n, np.zeros((0, 2)), np.zeros(L + 1, dtype=np.int64))
    y = np.zeros(0, dtype=complex)
    g = grad.gradient(op, X, y, levels)
    assert np.sum(g * X) == pytest.approx(expect, rel=1e-12)
