"""Write the expected values of the full 256 x 256, L = 60, M = 32768 per channel
problem after 500 primal-dual iterations, computed by the FP64 oracle only.

The inputs are those the FP32 GPU path receives: the seeded generator's draws
with uv, the truth cube and the data y rounded to FP32 (the oracle then works
in FP64 on the rounded values). mu (dirty-cube ratio, Sec. 2.3) and
kappa_3 = 1 / max_l ||Phi_l||^2 (Sec. 3.4) are the oracle's; the GPU parity test
passes the same values to the library, so both sides solve the same problem.

Stored (tests/golden/c2_pd500.json): mu, kappa_3, the input noise level and
bounds summary, aSNR every 50 iterations, the per-channel SNR, norm and sum of
the final cube, beta, and a 16 x 16 block-sum checksum of the final cube
summed over channels.

Run from the repository root (about an hour on one CPU core for the 500
iterations; the per-channel power iterations use a process pool):
    python tests/golden/make_c2_golden.py
"""

from __future__ import annotations

import json
import multiprocessing as mp
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import synth  # noqa: E402
from oracle import metrics, nufft, pd, problem  # noqa: E402

ITERS = 500
OUT = os.path.join(os.path.dirname(os.path.abspath(__file__)), "c2_pd500.json")


def rounded_inputs():
    inp = synth.make_inputs(2)
    inp.uv = inp.uv.astype(np.float32).astype(np.float64)
    inp.truth = inp.truth.astype(np.float32).astype(np.float64)
    prob = problem.make_problem(inp)
    prob.y = prob.y.astype(np.complex64).astype(np.complex128)
    return inp, prob


def _channel_norm2(args):
    nx, ny, uv = args
    op = nufft.WidebandOperator(nx, ny, uv, np.array([0, uv.shape[0]], dtype=np.int64))
    return problem.op_norm2(op)


def main():
    t0 = time.time()
    inp, prob = rounded_inputs()
    op = prob.op
    mu = problem.estimate_mu(op, prob.y, levels=4)
    jobs = [(inp.nx, inp.ny, inp.uv[inp.offsets[l]:inp.offsets[l + 1]]) for l in range(inp.L)]
    with mp.get_context("spawn").Pool(min(8, os.cpu_count() or 1)) as pool:
        norms = pool.map(_channel_norm2, jobs)
    on2 = float(max(norms))
    k3 = 1.0 / on2
    print(f"mu {mu:.10e}  ||Phi||^2 {on2:.10e}  ({time.time() - t0:.0f} s)", flush=True)
    prm = pd.PDParams(mu=mu, tau=0.33, kappa3=k3, levels=4)
    asnr_hist = {}

    def cb(st):
        if st.t % 50 == 0:
            asnr_hist[st.t] = metrics.asnr(prob.truth, st.X)
            print(f"it {st.t}: aSNR {asnr_hist[st.t]:.4f} dB, beta {st.beta:.3e} "
                  f"({time.time() - t0:.0f} s)", flush=True)

    st = pd.pd_solve(op, prob.y, prob.eps, prm, ITERS, callback=cb)
    X = st.X
    L, ny, nx = X.shape
    blocks = X.sum(axis=0).reshape(16, ny // 16, 16, nx // 16).sum(axis=(1, 3))
    out = dict(
        workload="256x256 image, L=60 channels over 1-2 GHz, M=32768 visibilities per channel, "
                 "40 dB input SNR, seed 2000; uv, truth and y rounded to FP32",
        iterations=ITERS, tau=0.33, kappa1=1.0, kappa2=1.0, levels=4,
        mu=mu, kappa3=k3, op_norm2=on2, sigma=prob.sigma,
        asnr_every_50={str(k): v for k, v in sorted(asnr_hist.items())},
        asnr=metrics.asnr(prob.truth, X),
        snr=[metrics.snr(prob.truth[l], X[l]) for l in range(L)],
        x_norm=[float(np.linalg.norm(X[l])) for l in range(L)],
        x_sum=[float(X[l].sum()) for l in range(L)],
        beta=float(st.beta),
        rho=[float(r) for r in st.rho],
        block_sums_16x16=blocks.ravel().tolist(),
        seconds=time.time() - t0,
    )
    with open(OUT, "w") as f:
        json.dump(out, f, indent=1)
    print(f"wrote {OUT}: aSNR {out['asnr']:.4f} dB in {out['seconds']:.0f} s")


if __name__ == "__main__":
    main()
