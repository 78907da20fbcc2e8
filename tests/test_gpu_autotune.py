"""Plan-time autotuner: the chosen parameters and the candidate times appear in
hs_plan_info, a second plan of the same shape takes them from the process
cache, and the operators of a tuned plan agree with those of an untuned one
(different work lists and Gram form, same results to FP32 rounding)."""

import numpy as np
import pytest

from gpu_util import TOL, dev, host, make_plan, ragged_case, rel, rounded

pytestmark = pytest.mark.gpu


def test_tuned_plan_reports_choice_and_matches_untuned(cuda_device):
    import __graft_entry__ as ge
    ge.build()
    case = rounded(ragged_case(n=128, L=5, M=(20000, 3000, 0, 9000, 15000), seed=21), "f32")
    tuned = make_plan(case, "f32")
    info = tuned.info
    assert info["tuned"] in (1, 2)
    assert info["sweep_hmax"] in (32, 64, 128) and info["sweep_cap"] in (512, 1024, 2048)
    assert info["gram_tc"] in (0, 1)
    if info["tuned"] == 1:
        assert all(t > 0 for t in info["tune_grid_ms"]) and all(t > 0 for t in info["tune_gram_ms"])
        best = int(np.argmin(info["tune_grid_ms"]))
        assert (info["sweep_hmax"], info["sweep_cap"]) == [(32, 512), (64, 1024), (128, 2048)][best]
        assert info["gram_tc"] == int(info["tune_gram_ms"][0] <= info["tune_gram_ms"][1])
    again = make_plan(case, "f32")
    assert again.info["tuned"] == 2
    assert again.info["sweep_hmax"] == info["sweep_hmax"] and again.info["gram_tc"] == info["gram_tc"]
    from paper_1806_04596_gb300 import hypersara as hs
    plain = hs.Plan(case["nx"], case["ny"], case["off"], dev(case["uv"], "f32"), levels=4, prec="f32",
                    autotune=False)
    assert plain.info["tuned"] == 0 and plain.info["sweep_hmax"] == 64 and plain.info["gram_tc"] == 1
    Yin = dev(case["Y"], "f32", True)
    a, b = host(tuned.phi_adj(Yin)), host(plain.phi_adj(Yin))
    assert rel(a, b) <= TOL["f32"]
    X = dev(case["X"], "f32")
    assert rel(host(tuned.gram(X)), host(plain.gram(X))) <= 1e-7


@pytest.mark.parametrize("prec", ["f32", "f64"])
def test_chunked_adjoint_fft_equals_single_pass(cuda_device, prec):
    """F^H in L2-sized channel chunks (row passes on the plan's second stream,
    overlapping the next chunk's column pass) gives bit-identical results to the
    single pass over all channels: same kernels and arithmetic, only the launch
    grouping differs. 256^2 image, L = 30: chunks of 20 and 10 channels (FP32)."""
    import torch
    import __graft_entry__ as ge
    ge.build()
    from paper_1806_04596_gb300 import hypersara as hs
    M = tuple(1500 + 97 * (l % 7) for l in range(30))
    case = rounded(ragged_case(n=256, L=30, M=M, seed=41), prec)
    uv = dev(case["uv"], prec)
    one = hs.Plan(256, 256, case["off"], uv, levels=4, prec=prec, autotune=False)
    chunked = hs.Plan(256, 256, case["off"], uv, levels=4, prec=prec, autotune=False, fft_chunked=True)
    assert one.info["fft_adj_chunk"] == 0
    C = chunked.info["fft_adj_chunk"]
    assert 1 <= C < 30
    Y = dev(case["Y"], prec, True)
    a = one.phi_adj(Y)
    b = chunked.phi_adj(Y)
    torch.cuda.synchronize()
    assert torch.equal(a, b)
    # again inside other work on the same stream: the side stream joins back before the result is read
    Z = chunked.phi_adj(Y) * 2
    assert torch.equal(Z, 2 * a)
