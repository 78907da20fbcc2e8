"""The pins of the oracle's set-up and preconditioning catch planted mistakes.

Each test plants one plausible error in the oracle (on the CPU, for the
duration of the test only) and checks that the pin written for that part
fails: a PSF normalisation off by 1 %, the nuclear norm replaced by the
Frobenius norm in mu (Sec. 4.3), the preconditioner dropped from the data
dual's projection (Sec. 3.3, Algorithm 2 step 11) and from the operator norm
that sets kappa_3.
"""

import numpy as np
import pytest

from oracle import problem, prox

import test_oracle_pd as tpd
import test_oracle_problem as tprob


def test_psf_normalisation_error_is_caught(monkeypatch):
    good = problem.psf_peak_norm
    monkeypatch.setattr(problem, "psf_peak_norm", lambda op, *a, **k: 1.01 * good(op, *a, **k))
    with pytest.raises(AssertionError):
        tprob.test_psf_peak_is_sum_of_squared_weights(False)
    with pytest.raises(AssertionError):
        tprob.test_dirty_cube_is_eta_times_adjoint()


def test_mu_with_frobenius_norm_is_caught(monkeypatch):
    monkeypatch.setattr(problem, "nuclear_norm", lambda X: float(np.linalg.norm(np.asarray(X).ravel())))
    with pytest.raises(AssertionError):
        tprob.test_mu_closed_form_rank_two_cube(32, 2)


def test_projection_without_preconditioner_is_caught(monkeypatch):
    good = prox.l2ball_dual
    monkeypatch.setattr(prox, "l2ball_dual", lambda vbar, y, eps, U=None: good(vbar, y, eps, None))
    with pytest.raises(AssertionError):
        tpd.test_constant_preconditioner_is_a_rescaled_problem()


def test_operator_norm_without_preconditioner_is_caught(monkeypatch):
    good = problem.op_norm2
    monkeypatch.setattr(problem, "op_norm2", lambda op, U=None, *a, **k: good(op, None, *a, **k))
    with pytest.raises(AssertionError):
        tpd.test_constant_preconditioner_is_a_rescaled_problem()


def test_pins_pass_without_planted_errors():
    """The same pins, unmodified oracle (the control of the tests above)."""
    tprob.test_psf_peak_is_sum_of_squared_weights(False)
    tprob.test_dirty_cube_is_eta_times_adjoint()
    tprob.test_mu_closed_form_rank_two_cube(32, 2)
    tpd.test_constant_preconditioner_is_a_rescaled_problem()
