#!/usr/bin/env python3
"""Benchmark of the HyperSARA primal-dual hot path on GB300.

Workload (default, --config 2): the 256 x 256, L = 60 channels over 1-2 GHz,
M = 32768 visibilities per channel problem, FP32 operators with FP64 norms and
FP64 Gram eigendecomposition, every PD iteration replayed as one CUDA graph.
One "step" is one full iteration of Algorithm 2 (steps 2-12 and 20-23) over
all channels.

Printed (one JSON line, rank 0):
  value      PD iterations / s (inputs resident in HBM; the iteration's working
             set, ~0.9 GB, is larger than the 129 MB L2, so no flush is needed)
  e2e        the same metric through the C ABI with host buffers: each step
             uploads y from pinned host memory (hs_pd_set_data_host), runs the
             iteration and copies the image cube X back to host memory
             (hs_pd_get_host)
  phi_vis_per_s   Phi + Phi^dagger throughput (visibilities / s over all channels)
  roofline   the slowest stage of the iteration, launched alone and timed with
             CUDA events on its stream, against the measured HBM copy bandwidth
             (algorithmic bytes per launch as listed in `stages`, each with the
             resource that limits it in practice); `phi_pair` gives the same for
             Phi + Phi^dagger, 2 (68 N + 16 M) L bytes (FP32)
  fp64       the plain FP64 GPU form of the same iteration, both forms run for
             the workload's iteration count: time and reconstruction SNR of each
  cpu_baseline   the FP64 NumPy oracle, full iterations of the whole workload

Other workloads (--config): 3 differentiation (autograd objective and the
checkpointed unrolled solve, peak memory), 4 precision sweep (per-operator and
per-cube error of FP64, FP32 and FP32 with compensated gridding), 5 the large
re-weighted solve (2048 x 2048, L = 64, ~86M visibilities, memory budget).

`--impl reference` times the oracle alone (the reference arm: this work has no
other implementation to compare against).
"""

from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "pd_iter_per_s"
UNIT = "iter/s"


def _args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=1000)
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--config", type=int, default=2)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-fp64", action="store_true")
    ap.add_argument("--gram", default="", help="n,L: time the Gram matrix alone on an n x n x L cube")
    return ap.parse_args()


def _workload(cfg_id: int) -> dict:
    import synth
    c = synth.CONFIGS[cfg_id]
    M = c["M"]
    return {"workload": c["name"], "n": c["n"], "L": c["L"],
            "M_per_channel": list(M) if isinstance(M, tuple) else M,
            "band_ghz": [c["f_lo"], c["f_hi"]], "insnr_db": c["insnr"], "levels": 4,
            "kernel": "Kaiser-Bessel 8x8, oversampling 2", "sara": "Dirac + db1..db8",
            "l2_policy": "inputs larger than L2 (iteration working set ~0.9 GB vs 129 MB L2)"}


# ---------------------------------------------------------------- clocks
class ClockSampler:
    """nvidia-smi samples during the timed region (read-only query)."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, val in zip(names, parts[5:9]):
                if val.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "samples": len(sm), "reasons": sorted(reasons)}


# ---------------------------------------------------------------- oracle (CPU)
def _oracle_problem(cfg_id: int, channels: int | None = None):
    """The workload's oracle problem on its first `channels` channels (all by
    default) and its step sizes: mu and kappa_3 as the oracle computed them for
    the 256 x 256 workload (tests/golden/c2_pd500.json, written by
    tests/golden/make_c2_golden.py), otherwise mu from the dirty cube and
    kappa_3 from a short power iteration (step sizes change the iterates, not
    the cost of an iteration)."""
    import synth
    from oracle import pd as opd
    from oracle import problem as oprob
    inp = synth.make_inputs(cfg_id)
    if channels is not None and channels < inp.L:
        inp.truth = inp.truth[:channels]
        inp.offsets = inp.offsets[:channels + 1]
        inp.uv = inp.uv[:inp.offsets[-1]]
        inp.noise = inp.noise[:inp.offsets[-1]]
    prob = oprob.make_problem(inp)
    gold = os.path.join(ROOT, "tests", "golden", "c2_pd500.json")
    if cfg_id == 2 and os.path.exists(gold):
        g = json.load(open(gold))
        mu, k3, src = g["mu"], g["kappa3"], "oracle values of the full workload (tests/golden/c2_pd500.json)"
    else:
        mu = oprob.estimate_mu(prob.op, prob.y, 4)
        k3 = 1.0 / oprob.op_norm2(prob.op, iters=5, tol=1e-3)
        src = "mu from the dirty cube, kappa_3 from 5 power iterations"
    prm = opd.PDParams(mu=mu, tau=0.33, kappa3=k3, levels=4)
    return inp, prob, prm, src


def _oracle_steps(cfg_id: int, channels: int | None, n: int):
    """Wall times of n consecutive oracle PD iterations (after one untimed one)."""
    from oracle import pd as opd
    inp, prob, prm, src = _oracle_problem(cfg_id, channels)
    st = opd.init_state(inp.L, inp.ny, inp.nx, int(inp.offsets[-1]))
    st = opd.pd_step(st, prob.op, prob.y, prob.eps, prm)
    times = []
    for _ in range(n):
        t0 = time.perf_counter()
        st = opd.pd_step(st, prob.op, prob.y, prob.eps, prm)
        times.append(time.perf_counter() - t0)
    return times, inp.L, src


def cpu_baseline(cfg_id: int, iters: int = 3) -> dict:
    import synth
    L = synth.CONFIGS[cfg_id]["L"]
    chans = L if cfg_id <= 2 else 1
    times, used, src = _oracle_steps(cfg_id, chans, iters)
    per = float(np.mean(times))
    return {"value": (used / L) / per, "unit": UNIT, "cores": os.cpu_count(), "kind": "oracle",
            "sample": f"FP64 NumPy oracle, {iters} full PD iterations on {used} of {L} channels "
                      f"({per:.2f} s each{'' if used == L else ', rate scaled by the channel fraction'}); "
                      f"{src}; NumPy FFT single-threaded, BLAS with its default threads"}


def run_reference(a):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    import synth
    L = synth.CONFIGS[a.config]["L"]
    total = a.steps + a.warmup
    # whole-workload iterations when the run stays within a few minutes, else
    # each step is one iteration on a fraction of the channels
    chans = L if (a.config <= 2 and total <= 30) else max(1, min(L, (30 * L) // max(total, 1)))
    if a.config > 2:
        chans = 1
    times, used, src = _oracle_steps(a.config, chans, total)
    t = times[a.warmup:] or times
    per = float(np.mean(t))
    v = (used / L) / per
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": a.gpus,
            "steps": a.steps, "warmup": a.warmup, "ms_per_step": per * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": _workload(a.config),
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": os.cpu_count(), "kind": "oracle",
                             "sample": f"each step: one oracle PD iteration on {used} of {L} channels"
                                       f"{'' if used == L else ' (rate scaled by the channel fraction)'}; {src}"},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def synth_L(cfg_id):
    import synth
    return synth.CONFIGS[cfg_id]["L"]


# DRAM bytes per launch of each stage (dram__bytes_read.sum + dram__bytes_write.sum
# of its kernels, one ncu capture of this bench's stage launches), recorded in
# profiles/stage_traffic.txt together with the SHA-256 of the sources of those
# kernels: a stage whose sources changed since the capture reports null.
STAGE_SOURCES = {"fft_fwd": ["hs_fft.cu"], "fft_adj": ["hs_fft.cu"], "degrid": ["hs_nufft.cu", "hs_plan.cpp"],
                 "grid": ["hs_nufft.cu", "hs_plan.cpp"], "psi_fwd": ["hs_dwt.cu"], "psi_adj": ["hs_dwt.cu"],
                 "gram_tc": ["hs_gram_tc.cu", "hs_prox.cu"], "gram_fma": ["hs_gram_tc.cu", "hs_prox.cu"]}


def stage_source_hash(stage: str) -> str:
    h = hashlib.sha256()
    for f in STAGE_SOURCES[stage]:
        with open(os.path.join(ROOT, "paper_1806_04596_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def _stage_traffic(stage: str, cfg_id: int):
    path = os.path.join(ROOT, "profiles", "stage_traffic.txt")
    try:
        for line in open(path):
            f = line.split()
            if len(f) == 4 and f[0] == f"C{cfg_id}" and f[1] == stage and f[3] == stage_source_hash(stage):
                return float(f[2])
    except OSError:
        pass
    return None


# ---------------------------------------------------------------- GPU arm
def job_rate(ms: float, steps: int, world: int, device: str = "cuda"):
    """Whole-job rate of `world` replicas that each ran `steps` steps: the
    slowest rank's time (MAX all-reduce when world > 1) and steps * world / it."""
    if world > 1:
        import torch
        import torch.distributed as td
        t = torch.tensor([ms], dtype=torch.float64, device=device)
        td.all_reduce(t, op=td.ReduceOp.MAX)
        ms = float(t.item())
    return ms, steps * world / (ms / 1e3)


# Resource that limits each stage in practice (ncu: profiles/kernel_sections_c2.md,
# profiles/stage_traffic.txt); the roofline each is measured against is HBM.
LIMITER = {
    "fft_fwd": "HBM: spectrum write plus the row-pass intermediate",
    "degrid": "shared-memory data pipe and instruction issue (8 lanes per visibility, staged window rows)",
    "grid": "instruction issue and shared-memory data pipe (12 row taps per lane per window group)",
    "fft_adj": "HBM: the row-pass intermediate round trip (1.57x algorithmic bytes)",
    "psi_fwd": "instruction issue of the first level (filter taps of 8 wavelets, staging, barriers)",
    "psi_adj": "instruction issue of the first level; instruction fetch in the shared-memory tail",
    "gram": "instruction issue (digit split and accumulator drain per 64-pixel chunk)",
}


def _peak_hbm():
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
        return float(peaks["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def _events_ms(stream, fn, reps):
    import torch
    fn()
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(reps):
        fn()
    e1.record(stream)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / reps


def _asnr(truth, X):
    Xh = X.detach().cpu().numpy().astype(np.float64)
    return float(np.mean([20 * np.log10(np.linalg.norm(truth[l]) / np.linalg.norm(truth[l] - Xh[l]))
                          for l in range(truth.shape[0])]))


def run_ours(a):
    if a.config == 3:
        return run_diff(a)
    if a.config == 4:
        return run_precision(a)
    import torch
    import synth
    from paper_1806_04596_gb300 import problem as dprob
    from paper_1806_04596_gb300 import hypersara as hs

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    dist = world > 1
    torch.cuda.set_device(local)
    if dist:
        import torch.distributed as td
        td.init_process_group("nccl")
    import __graft_entry__ as ge
    ge.build()
    big = a.config == 5

    # oracle CPU baseline first (before heavy GPU work, rank 0 at N = 1 only)
    cpu = None
    if rank == 0 and world == 1 and not a.no_cpu_baseline:
        cpu = cpu_baseline(a.config)

    # replicas: each rank solves its own problem (weak scaling, no data-path collective)
    torch.cuda.reset_peak_memory_stats()
    t_setup = time.perf_counter()
    inp = synth.make_inputs(a.config, realisation=rank)
    P = dprob.build(inp, prec="f32", power_iters=60 if big else 200, power_tol=1e-4 if big else 1e-6)
    setup_s = time.perf_counter() - t_setup
    plan = P.plan
    L, N, M = plan.L, plan.nx * plan.ny, plan.M
    info = plan.info
    w21 = wnu = None
    if big:   # Algorithm 1: the state references weight buffers that re-weighting rewrites
        w21 = torch.ones((9, plan.ny, plan.nx), dtype=torch.float32, device="cuda")
        wnu = torch.ones(L, dtype=torch.float64, device="cuda")
    st = hs.PDState(plan, P.y, P.eps, tau=0.33, kappa3=P.kappa3, mu=P.mu, w_nuc=wnu, w_l21=w21)
    stream = torch.cuda.current_stream()

    def barrier():
        if dist:
            torch.distributed.barrier()

    # warm-up (captures the iteration graph)
    st.solve(max(a.warmup, 1), graph=True)
    torch.cuda.synchronize()
    kern_per_step = st.graph_kernels

    clk = ClockSampler(local)
    clk.start()
    time.sleep(0.3)
    barrier()
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    torch.cuda.nvtx.range_push("timed")
    e0.record(stream)
    st.solve(a.steps, graph=True)
    e1.record(stream)
    torch.cuda.nvtx.range_pop()
    torch.cuda.synchronize()
    barrier()
    ms = e0.elapsed_time(e1)
    clocks = clk.stop()
    ms, value = job_rate(ms, a.steps, world)
    plan.check()

    # Phi + Phi^dagger throughput
    Xin = P.truth.clone()
    Y = plan.vis()
    Xo = plan.cube()
    A9 = plan.cube(9)
    reps = max(10, min(a.steps, 500 if not big else 20))

    def pair():
        plan.phi_fwd(Xin, Y)
        plan.phi_adj(Y, Xo)
    torch.cuda.nvtx.range_push("phi_pair")
    pair_ms = _events_ms(stream, pair, reps)
    torch.cuda.nvtx.range_pop()
    phi_vis = M / (pair_ms / 1e3)
    hbm, peak_src = _peak_hbm()
    pair_bytes = 2 * (68 * N * L + 16 * M)
    pair_gbs = pair_bytes / (pair_ms / 1e3) / 1e9

    # every stage of the iteration launched alone (CUDA events on this stream);
    # algorithmic bytes per launch (FP32): spectrum 32 B / grid cell (4N cells
    # per channel), image 4 B / pixel, 16 B per visibility (coordinates + value);
    # the Gram matrix reads the two cubes it sums (8 B / pixel and channel)
    NL = N * L
    stage_bytes = {"fft_fwd": 36 * NL, "degrid": 32 * NL + 16 * M, "grid": 16 * M + 32 * NL,
                   "fft_adj": 36 * NL, "psi_fwd": 40 * NL, "psi_adj": 40 * NL}
    stage_io = {"fft_fwd": (Xin, None), "degrid": (None, Y), "grid": (Y, None), "fft_adj": (None, Xo),
                "psi_fwd": (Xin, A9), "psi_adj": (A9, Xo)}
    stages = {}
    sreps = max(5, min(a.steps // 2, 200 if not big else 20))
    for name, (si, so) in stage_io.items():
        torch.cuda.nvtx.range_push(f"stage_{name}")
        ms_s = plan.time_stage(name, si, so, reps=sreps)
        torch.cuda.nvtx.range_pop()
        gbs = stage_bytes[name] / (ms_s / 1e3) / 1e9
        stages[name] = {"ms": ms_s, "alg_bytes": stage_bytes[name], "GB_s": gbs, "frac": gbs / hbm,
                        "limiter": LIMITER[name]}
    if L <= 64:
        Xa = Xo.clone()
        forms = {}
        for form, tag in (("tensor_cores", "tc"), ("cuda_cores", "fma")):
            torch.cuda.nvtx.range_push(f"stage_gram_{tag}")
            forms[form] = _events_ms(stream, lambda: plan.gram(Xin, Xa, form), sreps)
            torch.cuda.nvtx.range_pop()
        g_ms = forms["tensor_cores" if info["gram_tc"] else "cuda_cores"]
        gbs = 8 * NL / (g_ms / 1e3) / 1e9
        stages["gram"] = {"ms": g_ms, "alg_bytes": 8 * NL, "GB_s": gbs, "frac": gbs / hbm,
                          "form": "tensor cores (tcgen05)" if info["gram_tc"] else "CUDA cores",
                          "forms_ms": forms,
                          "limiter": LIMITER["gram"] if info["gram_tc"] else "instruction issue (two-sum FMA)"}
    dom = max((k for k in stages if k != "gram"), key=lambda k: stages[k]["ms"])
    traffic = _stage_traffic(dom, a.config)
    for k in stages:
        tk = ("gram_tc" if info["gram_tc"] else "gram_fma") if k == "gram" else k
        stages[k]["traffic"] = _stage_traffic(tk, a.config)

    # end to end through the C ABI with host buffers (pinned): y in, X out
    y_host = P.y.cpu().pin_memory()
    eps_host = P.eps.cpu().numpy().astype(np.float64)
    X_host = torch.empty((L, plan.ny, plan.nx), dtype=torch.float32).pin_memory()
    st.solve(1, graph=True)
    torch.cuda.synchronize()
    e2e_steps = max(5, min(a.steps // 2, 300 if not big else 10))
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        st.set_data_host(y_host, eps_host)
        st.solve(1, graph=True)
        st.get_host(X_host)
    e2e_s = (time.perf_counter() - t0) / e2e_steps
    h2d = M * y_host.element_size() + 8 * plan.nblocks
    d2h = X_host.numel() * X_host.element_size() + 8 + 8 * plan.nblocks

    def _iter_rate(state, k):
        state.solve(2, graph=True)
        torch.cuda.synchronize()
        g0 = torch.cuda.Event(enable_timing=True)
        g1 = torch.cuda.Event(enable_timing=True)
        g0.record(stream)
        state.solve(k, graph=True)
        g1.record(stream)
        torch.cuda.synchronize()
        return k / (g0.elapsed_time(g1) / 1e3)

    variants = None
    fp64 = None
    if not big:
        # model variants and the re-weighting step on the same problem (FP32, graph replay)
        kv = max(5, min(a.steps // 4, 200))
        variants = {}
        for name, kw in (("lr", dict(use_l21=False)), ("jas", dict(use_nuclear=False)),
                         ("sara", dict(use_nuclear=False, sparsity="l1"))):
            sv_ = hs.PDState(plan, P.y, P.eps, tau=0.33, kappa3=P.kappa3, mu=P.mu, **kw)
            variants[name] = {"value": _iter_rate(sv_, kv), "unit": UNIT}
            sv_.close()
        w21v = torch.ones((9, plan.ny, plan.nx), dtype=torch.float32, device="cuda")
        wnuv = torch.ones(L, dtype=torch.float64, device="cuda")
        st_rw = hs.PDState(plan, P.y, P.eps, tau=0.33, kappa3=P.kappa3, mu=P.mu, w_nuc=wnuv, w_l21=w21v)
        st_rw.solve(20, graph=True)
        variants["reweight_ms"] = _events_ms(stream, lambda: st_rw.reweight(0.8, 0.8, w21v, wnuv), 5)
        variants["reweighted_lrjas_iter_per_s"] = _iter_rate(st_rw, kv)
        st_rw.close()

        # FP32 and the plain FP64 GPU form run for the workload's iteration count
        # from the same (zero) start: time and reconstruction SNR of each
        if not a.no_fp64:
            T = int(synth.CONFIGS[a.config]["iters"])
            g0, g1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)

            def run_T(state):
                state.solve(1, graph=True)     # first iteration captures the graph (untimed)
                torch.cuda.synchronize()
                g0.record(stream)
                state.solve(T - 1, graph=True)
                g1.record(stream)
                torch.cuda.synchronize()
                Xs, _, _ = state.get()
                return g0.elapsed_time(g1) / 1e3, _asnr(inp.truth, Xs)

            s32 = hs.PDState(plan, P.y, P.eps, tau=0.33, kappa3=P.kappa3, mu=P.mu)
            t32, snr32 = run_T(s32)
            s32.close()
            P64 = dprob.build(inp, prec="f64", power_iters=60, power_tol=1e-4)
            s64 = hs.PDState(P64.plan, P64.y, P64.eps, tau=0.33, kappa3=P.kappa3, mu=P.mu)
            t64, snr64 = run_T(s64)
            fp64 = {"iters": T, "fp32": {"s": t32, "asnr_db": snr32, "iter_per_s": (T - 1) / t32},
                    "fp64": {"s": t64, "asnr_db": snr64, "iter_per_s": (T - 1) / t64},
                    "asnr_gap_db": snr32 - snr64, "speedup_fp32_over_fp64": t64 / t32,
                    "note": "both forms from a zero start with the same mu and kappa_3 (the FP32 problem's), "
                            "graph replay of iterations 2..T; speed-up at equal iteration count, SNRs stated"}
            s64.close()
            P64.plan.close()
    X, beta, rho = st.get()
    asnr = _asnr(inp.truth, X)

    rw = None
    if big:   # Algorithm 1 on the large workload: re-weights of inner PD loops, all graph-replayed
        outer, inner = 5, 20
        st_rw = hs.PDState(plan, P.y, P.eps, tau=0.33, kappa3=P.kappa3, mu=P.mu, w_nuc=wnu, w_l21=w21)
        g0, g1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        wnu.fill_(1.0)
        w21.fill_(1.0)
        g0.record(stream)
        hs.reweighted_solve(st_rw, outer, inner, decay=0.8, graph=True)
        g1.record(stream)
        torch.cuda.synchronize()
        t_rw = g0.elapsed_time(g1) / 1e3
        Xr, _, _ = st_rw.get()
        rw = {"outer": outer, "inner": inner, "iterations": outer * inner, "s": t_rw,
              "iter_per_s": outer * inner / t_rw, "asnr_db": _asnr(inp.truth, Xr)}
        st_rw.close()

    mem = {"peak_allocated_GB": torch.cuda.max_memory_allocated() / 1e9,
           "plan_GB": info["device_bytes"] / 1e9,
           "device_total_GB": torch.cuda.get_device_properties(local).total_memory / 1e9,
           "budget_GB": 180.0}
    mem["state_and_buffers_GB"] = mem["peak_allocated_GB"]
    mem["total_GB"] = mem["plan_GB"] + mem["peak_allocated_GB"]
    mem["frac_of_budget"] = mem["total_GB"] / mem["budget_GB"]

    if rank != 0:
        return
    cfg = _workload(a.config)
    cfg["tuned"] = {"gram": "tensor cores" if info["gram_tc"] else "CUDA cores",
                    "sweep_rows_per_item": info["sweep_hmax"], "sweep_list_cap": info["sweep_cap"],
                    "grid_candidates_ms": info["tune_grid_ms"], "fft_adj_chunk": info["fft_adj_chunk"],
                    "fft_adj_candidates_ms": info["tune_fft_ms"], "tune_s": info["tune_ms"] / 1e3}
    cfg["visibilities"] = M
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": a.steps,
        "warmup": a.warmup, "ms_per_step": ms / a.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": cfg,
        "roofline": {"bound": "hbm", "achieved": stages[dom]["GB_s"], "peak": hbm, "unit": "GB/s",
                     "frac": stages[dom]["frac"], "traffic": traffic, "kernel": dom,
                     "limiter": stages[dom]["limiter"],
                     "alg_bytes_per_launch": stages[dom]["alg_bytes"], "launch_ms": stages[dom]["ms"],
                     "peak_source": peak_src},
        "stages": stages,
        "phi_pair": {"ms": pair_ms, "alg_bytes": pair_bytes, "GB_s": pair_gbs, "frac": pair_gbs / hbm,
                     "target_frac": 0.60},
        "phi_vis_per_s": phi_vis, "phi_pair_ms": pair_ms,
        "e2e": {"value": 1.0 / e2e_s, "unit": UNIT, "h2d_bytes_per_step": h2d,
                "d2h_bytes_per_step": d2h, "api": "hs_pd_set_data_host + hs_pd_solve + hs_pd_get_host"},
        "gpu_launches": kern_per_step * a.steps,
        "kernels_per_step": kern_per_step,
        "clocks": clocks,
        "asnr_db": asnr, "asnr_after_iterations": a.warmup + a.steps + 1 + e2e_steps,
        "beta": beta, "mu": P.mu, "kappa3": P.kappa3,
        "fp64": fp64,
        "variants": variants,
        "reweighted": rw,
        "memory": mem,
        "setup_s": setup_s,
        "cpu_baseline": cpu,
    }
    print(json.dumps(line), flush=True)


def _gpu_setup():
    import torch
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    import __graft_entry__ as ge
    ge.build()
    return local


def run_diff(a):
    """Differentiation workload (512 x 512, L = 32, M_l ~ U[1e5, 4e5], FP32): one
    step is the objective 0.5 ||Phi X - y||^2 + ||Psi^dagger X||_{2,1} and its
    gradient through the autograd Functions (forward + backward kernels). Also
    the unrolled 50-iteration Algorithm 2 with checkpoints every 10 iterations
    (forward + backward time, peak memory with and without checkpointing), and
    the gradient against the oracle's (all channels) and central differences."""
    import torch
    import synth
    from paper_1806_04596_gb300 import autograd as ag
    from paper_1806_04596_gb300 import problem as dprob
    local = _gpu_setup()
    inp = synth.make_inputs(3)
    P = dprob.build(inp, prec="f32", power_iters=60, power_tol=1e-4)
    plan = P.plan
    stream = torch.cuda.current_stream()
    rng = np.random.default_rng(1)
    X0 = torch.tensor(rng.uniform(0, 1, inp.truth.shape), dtype=torch.float32, device="cuda")

    def step():
        X = X0.clone().requires_grad_(True)
        f = ag.objective(plan, X, P.y)
        (g,) = torch.autograd.grad(f, X)
        return f, g
    for _ in range(max(a.warmup, 1)):
        step()
    torch.cuda.synchronize()
    clk = ClockSampler(local)
    clk.start()
    time.sleep(0.3)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(a.steps):
        f, g = step()
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    clocks = clk.stop()

    # gradient against the FP64 oracle (all channels: the l2,1 term couples them)
    # and against central differences with step 1e-3
    from oracle import grad as ograd
    from oracle import nufft
    Xh = X0.cpu().numpy().astype(np.float64)
    uv = inp.uv.astype(np.float32).astype(np.float64)
    op = nufft.WidebandOperator(inp.nx, inp.ny, uv, inp.offsets)
    yh = P.y.cpu().numpy().astype(np.complex128)
    t0 = time.perf_counter()
    gref = ograd.gradient(op, Xh, yh, 4)
    t_oracle = time.perf_counter() - t0
    gh = g.cpu().numpy().astype(np.float64)
    grad_rel = float(np.linalg.norm(gh - gref) / np.linalg.norm(gref))
    # central differences need the objective (~1e17 here) to far better than FP32
    # rounding: they run on an FP64 plan of the same problem, and its gradient
    # is compared with the FP32 one too
    from paper_1806_04596_gb300 import hypersara as hs
    plan64 = hs.Plan(inp.nx, inp.ny, inp.offsets, torch.tensor(uv, dtype=torch.float64, device="cuda"),
                     levels=4, prec="f64")
    X64 = X0.double().requires_grad_(True)
    Y64 = P.y.to(torch.complex128)
    (g64,) = torch.autograd.grad(ag.objective(plan64, X64, Y64), X64)
    fd = []
    for k in range(2):
        D = torch.tensor(rng.standard_normal(inp.truth.shape), dtype=torch.float64, device="cuda")
        with torch.no_grad():
            fp = float(ag.objective(plan64, X64.detach() + 1e-3 * D, Y64))
            fm = float(ag.objective(plan64, X64.detach() - 1e-3 * D, Y64))
        fd.append({"fd": (fp - fm) / 2e-3, "grad_dot_fp64": float(torch.sum(g64 * D)),
                   "grad_dot_fp32": float(torch.sum(g.double() * D))})
    plan64.close()

    # unrolled Algorithm 2, gradient of a loss of the final image with respect to y
    eps = P.eps
    unrolled = {}
    Yw = P.y.clone().requires_grad_(True)   # warm-up (allocator growth, first launches)
    torch.sum(ag.unrolled_pd(plan, Yw, eps, iters=4, mu=P.mu, kappa3=P.kappa3, checkpoint_every=2)).backward()
    del Yw
    for ck in (10, 0):
        torch.cuda.synchronize()
        torch.cuda.reset_peak_memory_stats()
        base = torch.cuda.memory_allocated()
        Y = P.y.clone().requires_grad_(True)
        u0, u1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        u0.record(stream)
        X = ag.unrolled_pd(plan, Y, eps, iters=50, mu=P.mu, kappa3=P.kappa3, checkpoint_every=ck)
        loss = 0.5 * torch.sum((X - P.truth) ** 2)
        loss.backward()
        u1.record(stream)
        torch.cuda.synchronize()
        unrolled[f"checkpoint_every_{ck}" if ck else "no_checkpoint"] = {
            "s": u0.elapsed_time(u1) / 1e3, "peak_GB": (torch.cuda.max_memory_allocated() - base) / 1e9}
        del X, Y, loss
    line = {"metric": "objective_grad_per_s", "value": a.steps / (ms / 1e3), "unit": "grad/s",
            "n_gpus": 1, "steps": a.steps, "warmup": a.warmup, "ms_per_step": ms / a.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic", "config": dict(_workload(3), visibilities=plan.M),
            "clocks": clocks, "grad_rel_err_vs_oracle": grad_rel, "oracle_grad_s": t_oracle,
            "central_differences_step_1e-3": fd, "unrolled_pd_50": unrolled,
            "plan_GB": plan.info["device_bytes"] / 1e9}
    print(json.dumps(line), flush=True)


def run_precision(a):
    """Precision sweep (1024 x 1024, L = 16, M = 1e6, 50 sources plus a diffuse
    field, 30 dB): per-operator error of the FP64, FP32 and FP32 compensated-
    gridding plans against the FP64 oracle (channels 0 and 15 for Phi, Phi^dagger,
    Psi^dagger, Psi; the whole cube for the proxes), and per-cube error after the
    workload's 100 PD iterations (aSNR, and distance to the FP64 GPU cube, which
    tracks the oracle to ~1e-12 per iteration)."""
    import torch
    import synth
    from oracle import nufft, prox, wavelets
    from paper_1806_04596_gb300 import hypersara as hs
    from paper_1806_04596_gb300 import problem as dprob
    local = _gpu_setup()
    stream = torch.cuda.current_stream()
    inp = synth.make_inputs(4)
    T = int(synth.CONFIGS[4]["iters"])
    chans = (0, inp.L - 1)
    rng = np.random.default_rng(3)
    Xr = rng.uniform(0, 1, (inp.L, inp.ny, inp.nx))
    Ar = rng.standard_normal((9, inp.L, inp.ny, inp.nx))
    ops = {}
    probs = {}
    for name, prec, comp in (("fp64", "f64", False), ("fp32", "f32", False), ("fp32_compensated", "f32", True)):
        Pp = dprob.build(inp, prec=prec, compensated=comp, power_iters=60, power_tol=1e-4)
        probs[name] = Pp
    # every form receives the FP64 problem's data (y rounded to the form's precision)
    P64 = probs["fp64"]
    y64 = P64.y.cpu().numpy()
    uv32 = inp.uv.astype(np.float32).astype(np.float64)
    errs = {}
    for name, Pp in probs.items():
        plan = Pp.plan
        f32 = plan.prec == "f32"
        uvv = uv32 if f32 else inp.uv
        X_in = Xr.astype(np.float32).astype(np.float64) if f32 else Xr
        A_in = Ar.astype(np.float32).astype(np.float64) if f32 else Ar
        y_in = y64.astype(np.complex64).astype(np.complex128) if f32 else y64
        rdt, cdt = plan.rdtype, plan.cdtype
        Yd = plan.phi_fwd(torch.tensor(X_in, dtype=rdt, device="cuda")).cpu().numpy()
        Xa = plan.phi_adj(torch.tensor(y_in, dtype=cdt, device="cuda")).cpu().numpy()
        Aw = plan.psi_fwd(torch.tensor(X_in, dtype=rdt, device="cuda")).cpu().numpy()
        Xs = plan.psi_adj(torch.tensor(A_in, dtype=rdt, device="cuda")).cpu().numpy()
        e = {"phi": [], "phi_adj": [], "psi_analysis": None, "psi_synthesis": None}
        for l in chans:
            a_, b_ = inp.offsets[l], inp.offsets[l + 1]
            chop = nufft.ChannelOperator(inp.nx, inp.ny, uvv[a_:b_])
            r1 = chop.forward(X_in[l])
            e["phi"].append(float(np.linalg.norm(Yd[a_:b_] - r1) / np.linalg.norm(r1)))
            r2 = chop.adjoint(y_in[a_:b_])
            e["phi_adj"].append(float(np.linalg.norm(Xa[l] - r2) / np.linalg.norm(r2)))
        rA = wavelets.psi_adjoint_cube(X_in[list(chans)], 4)
        e["psi_analysis"] = float(np.linalg.norm(Aw[:, list(chans)] - rA) / np.linalg.norm(rA))
        rX = wavelets.psi_cube(A_in[:, list(chans)], 4)
        e["psi_synthesis"] = float(np.linalg.norm(Xs[list(chans)] - rX) / np.linalg.norm(rX))
        thr = 0.5 * float(np.median(np.sqrt(np.sum(A_in ** 2, axis=1))))
        Pl = plan.prox_l21(torch.tensor(A_in, dtype=rdt, device="cuda"), thr).cpu().numpy()
        rl = prox.prox_l21(A_in, 1.0, thr)
        e["prox_l21"] = float(np.linalg.norm(Pl - rl) / np.linalg.norm(rl))
        sv = np.linalg.svd(X_in.reshape(inp.L, -1).T, compute_uv=False)
        thr_n = float(sv[min(3, len(sv) - 1)])
        Pn, _ = plan.prox_nuclear(torch.tensor(X_in, dtype=rdt, device="cuda"), thr_n)
        rn = prox.prox_nuclear(X_in, 1.0, thr_n)
        e["prox_nuclear"] = float(np.linalg.norm(Pn.cpu().numpy() - rn) / np.linalg.norm(rn))
        errs[name] = e
    # per cube: T iterations of each form with the FP64 problem's step sizes and data
    cubes, rates, snrs = {}, {}, {}
    for name, Pp in probs.items():
        plan = Pp.plan
        Y = P64.y.to(plan.cdtype)
        st = hs.PDState(plan, Y, P64.eps, tau=0.33, kappa3=P64.kappa3, mu=P64.mu)
        st.solve(1, graph=True)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        st.solve(T - 1, graph=True)
        e1.record(stream)
        torch.cuda.synchronize()
        rates[name] = (T - 1) / (e0.elapsed_time(e1) / 1e3)
        X, _, _ = st.get()
        cubes[name] = X.cpu().numpy().astype(np.float64)
        snrs[name] = _asnr(inp.truth, X)
        st.close()
    ref = cubes["fp64"]
    cube = {name: {"asnr_db": snrs[name], "rel_to_fp64_cube": float(np.linalg.norm(c - ref) / np.linalg.norm(ref)),
                   "iter_per_s": rates[name]} for name, c in cubes.items()}
    line = {"metric": METRIC, "value": rates["fp32"], "unit": UNIT, "n_gpus": 1, "steps": T - 1, "warmup": 1,
            "ms_per_step": 1e3 / rates["fp32"], "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": dict(_workload(4), sources=50, diffuse=True, visibilities=int(inp.offsets[-1])),
            "precision": {"operators_rel_err_vs_oracle": errs, "cube_after_iterations": T, "cube": cube,
                          "operator_channels": list(chans)}}
    print(json.dumps(line), flush=True)


def run_gram(a):
    """The nuclear prox's Gram matrix alone (hs_gram) on an n x n x L cube
    Z = X + Xa (the PD form), both forms, CUDA events: `--gram n,L`."""
    import torch
    from paper_1806_04596_gb300 import hypersara as hs
    _gpu_setup()
    n, L = (int(v) for v in a.gram.split(","))
    stream = torch.cuda.current_stream()
    plan = hs.Plan(n, n, np.zeros(L + 1, dtype=np.int64), torch.zeros((0, 2), dtype=torch.float32, device="cuda"),
                   levels=1, prec="f32")
    X = torch.rand((L, n, n), dtype=torch.float32, device="cuda")
    Xa = torch.rand((L, n, n), dtype=torch.float32, device="cuda")
    hbm, src = _peak_hbm()
    out = {}
    for form, tag in (("tensor_cores", "tc"), ("cuda_cores", "fma")):
        torch.cuda.nvtx.range_push(f"gram_{tag}")
        ms = _events_ms(stream, lambda: plan.gram(X, Xa, form), max(a.steps, 3))
        torch.cuda.nvtx.range_pop()
        gbs = 8.0 * n * n * L / (ms / 1e3) / 1e9
        out[form] = {"ms": ms, "GB_s": gbs, "frac": gbs / hbm}
    plan.check()
    print(json.dumps({"gram": {"n": n, "L": L, "alg_bytes": 8 * n * n * L, "peak_GB_s": hbm, "peak_source": src,
                               "forms": out}}), flush=True)


def main():
    a = _args()
    if a.gram:
        return run_gram(a)
    if a.impl == "reference":
        run_reference(a)
    else:
        run_ours(a)


if __name__ == "__main__":
    main()
