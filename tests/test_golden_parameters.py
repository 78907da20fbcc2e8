"""The parameter values the paper prints (tests/golden/paper_parameters.txt,
each line citing where) against the defaults of the oracle and of the Python
binding: the adaptive-bound constants of Appendix A, kappa_1 and the step-size
range of Sec. 3.4, and the re-weighting schedule of Sec. 3.5."""

import inspect
import os

import pytest

from oracle import pd, reweight

HERE = os.path.dirname(os.path.abspath(__file__))


@pytest.fixture(scope="module")
def paper():
    vals = {}
    with open(os.path.join(HERE, "golden", "paper_parameters.txt")) as f:
        for line in f:
            if line.strip() and not line.startswith("#"):
                name, value = line.split()[:2]
                vals[name] = float(value)
    return vals


def _defaults(fn):
    return {k: v.default for k, v in inspect.signature(fn).parameters.items()
            if v.default is not inspect.Parameter.empty}


def test_adaptive_bound_constants(paper):
    a = pd.AdaptParams()
    assert (a.lambda1, a.lambda2, a.lambda3, a.min_gap) == (
        paper["lambda1"], paper["lambda2"], paper["lambda3"], paper["vartheta_bar"])
    from paper_1806_04596_gb300 import hypersara as hs
    d = _defaults(hs.PDState.set_adaptive)
    assert (d["lambda1"], d["lambda2"], d["lambda3"], d["min_gap"]) == (
        paper["lambda1"], paper["lambda2"], paper["lambda3"], paper["vartheta_bar"])


def test_step_sizes(paper):
    p = pd.PDParams(mu=1.0)
    assert p.kappa1 == paper["kappa1"]
    assert 0 < p.tau < paper["tau_sup"]
    from paper_1806_04596_gb300 import hypersara as hs
    d = _defaults(hs.PDState.__init__)
    assert d["kappa1"] == paper["kappa1"] and 0 < d["tau"] < paper["tau_sup"]


def test_reweighting_schedule(paper):
    from paper_1806_04596_gb300 import hypersara as hs
    for fn in (reweight.reweighted_solve, hs.reweighted_solve):
        assert paper["decay_lo"] <= _defaults(fn)["decay"] <= paper["decay_hi"]
    # the first weights use gamma = gamma_bar = the paper's initial value
    import numpy as np
    import synth
    from oracle import problem
    inp = synth.make_inputs(1, n=16, L=2, M=120, seed=5)
    prob = problem.make_problem(inp)
    prm = pd.PDParams(mu=0.05, levels=2, kappa3=1.0 / problem.op_norm2(prob.op, iters=100, tol=1e-8))
    st, w21, wn = reweight.reweighted_solve(prob.op, prob.y, prob.eps, prm, outer=1, inner=3)
    g = paper["gamma_init"]
    assert np.array_equal(wn, reweight.weights_nuclear(st.X, g))
    assert np.array_equal(w21, reweight.weights_l21(st.X, 2, g))
