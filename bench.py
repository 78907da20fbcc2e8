#!/usr/bin/env python3
"""Benchmark of the HyperSARA primal-dual hot path on GB300.

Workload (default): the 256 x 256, L = 60 channels over 1-2 GHz, M = 32768
visibilities per channel problem, FP32 operators with FP64 norms and FP64
Gram eigendecomposition, every PD iteration replayed as one CUDA graph. One
"step" is one full iteration of Algorithm 2 (steps 2-12 and 20-23) over all
channels.

Printed (one JSON line, rank 0):
  value      PD iterations / s (inputs resident in HBM; the iteration's working
             set, ~0.9 GB, is larger than the 129 MB L2, so no flush is needed)
  e2e        the same metric through the public API with host buffers: each step
             uploads the data y from pinned host memory (set_data) and reads the
             iteration's beta and per-channel residual norms back
  phi_vis_per_s   Phi + Phi^dagger throughput (visibilities / s over all channels)
  roofline   the slowest stage of the iteration, launched alone and timed with
             CUDA events on its stream, against the measured HBM copy bandwidth
             (algorithmic bytes per launch as listed in `stages`); `phi_pair`
             gives the same for Phi + Phi^dagger, 2 (68 N + 16 M) L bytes (FP32)
  fp64       the plain FP64 GPU form of the same iteration (iterations / s)
  cpu_baseline   the FP64 NumPy oracle on a bounded sample of the workload

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
    ap.add_argument("--cpu-channels", type=int, default=3)
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
def _oracle_sample(cfg_id: int, channels: int, iters: int):
    """Time `iters` oracle PD iterations on the first `channels` channels of the
    workload; returns seconds per full-workload iteration (scaled by L / channels)."""
    import synth
    from oracle import pd as opd
    from oracle import problem as oprob
    c = synth.CONFIGS[cfg_id]
    inp = synth.make_inputs(cfg_id)
    keep = channels
    inp.truth = inp.truth[:keep]
    inp.offsets = inp.offsets[:keep + 1]
    inp.uv = inp.uv[:inp.offsets[-1]]
    inp.noise = inp.noise[:inp.offsets[-1]]
    prob = oprob.make_problem(inp)
    prm = opd.PDParams(mu=0.01, tau=0.33, kappa3=1.0, levels=4)
    st = opd.init_state(keep, inp.ny, inp.nx, int(inp.offsets[-1]))
    st = opd.pd_step(st, prob.op, prob.y, prob.eps, prm)   # warm caches
    times = []
    for _ in range(iters):
        t0 = time.perf_counter()
        st = opd.pd_step(st, prob.op, prob.y, prob.eps, prm)
        times.append(time.perf_counter() - t0)
    per = float(np.mean(times))
    return per * c["L"] / keep, per, times


def cpu_baseline(cfg_id: int, channels: int) -> dict:
    full, per, _ = _oracle_sample(cfg_id, channels, 2)
    return {"value": 1.0 / full, "unit": UNIT, "cores": os.cpu_count(), "kind": "oracle",
            "sample": f"FP64 NumPy oracle, 2 PD iterations on {channels} of the workload's channels "
                      f"({per:.2f} s each), scaled linearly to all channels; NumPy FFT single-threaded, "
                      f"BLAS with its default threads"}


def run_reference(a):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    cfg = _workload(a.config)
    full, per, times = _oracle_sample(a.config, a.cpu_channels, a.steps + a.warmup)
    t = times[a.warmup:] or times
    per_full = float(np.mean(t)) * synth_L(a.config) / a.cpu_channels
    v = 1.0 / per_full
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": a.gpus,
            "steps": a.steps, "warmup": a.warmup, "ms_per_step": per_full * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": cfg,
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": os.cpu_count(), "kind": "oracle",
                             "sample": f"each step: one oracle PD iteration on {a.cpu_channels} of "
                                       f"{synth_L(a.config)} channels, scaled linearly"},
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
                 "grid": ["hs_nufft.cu", "hs_plan.cpp"], "psi_fwd": ["hs_dwt.cu"], "psi_adj": ["hs_dwt.cu"]}


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


def run_ours(a):
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

    # oracle CPU baseline first (before heavy GPU work, rank 0 at N = 1 only)
    cpu = None
    if rank == 0 and world == 1 and not a.no_cpu_baseline:
        cpu = cpu_baseline(a.config, a.cpu_channels)

    # replicas: each rank solves its own problem (weak scaling, no data-path collective)
    inp = synth.make_inputs(a.config, realisation=rank)
    P = dprob.build(inp, prec="f32")
    plan = P.plan
    L, N, M = plan.L, plan.nx * plan.ny, plan.M
    st = hs.PDState(plan, P.y, P.eps, tau=0.33, kappa3=P.kappa3, mu=P.mu)
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
    X, beta, rho = st.get()
    torch.cuda.synchronize()
    Xh = X.cpu().numpy().astype(np.float64)
    asnr = float(np.mean([20 * np.log10(np.linalg.norm(inp.truth[l]) /
                                        np.linalg.norm(inp.truth[l] - Xh[l])) for l in range(L)]))

    # Phi + Phi^dagger throughput
    Xin = P.truth.clone()
    Y = plan.vis()
    Xo = plan.cube()
    A9 = plan.cube(9)
    for _ in range(3):
        plan.phi_fwd(Xin, Y)
        plan.phi_adj(Y, Xo)
    reps = max(10, min(a.steps, 500))
    torch.cuda.synchronize()
    f0 = torch.cuda.Event(enable_timing=True)
    f1 = torch.cuda.Event(enable_timing=True)
    torch.cuda.nvtx.range_push("phi_pair")
    f0.record(stream)
    for _ in range(reps):
        plan.phi_fwd(Xin, Y)
        plan.phi_adj(Y, Xo)
    f1.record(stream)
    torch.cuda.nvtx.range_pop()
    torch.cuda.synchronize()
    pair_ms = f0.elapsed_time(f1) / reps
    phi_vis = M / (pair_ms / 1e3)
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
        hbm = float(peaks["hbm_gbs"])
        peak_src = "measured"
    except Exception:
        hbm, peak_src = 6800.0, "fallback"
    pair_bytes = 2 * (68 * N + 16 * (M / L)) * L
    pair_gbs = pair_bytes / (pair_ms / 1e3) / 1e9

    # every stage of the iteration launched alone (CUDA events on this stream);
    # algorithmic bytes per launch (FP32): spectrum 32 B / grid cell (4N cells
    # per channel), image 4 B / pixel, 16 B per visibility (coordinates + value)
    NL = N * L
    stage_bytes = {"fft_fwd": 36 * NL, "degrid": 32 * NL + 16 * M, "grid": 16 * M + 32 * NL,
                   "fft_adj": 36 * NL, "psi_fwd": 40 * NL, "psi_adj": 40 * NL}
    stage_io = {"fft_fwd": (Xin, None), "degrid": (None, Y), "grid": (Y, None), "fft_adj": (None, Xo),
                "psi_fwd": (Xin, A9), "psi_adj": (A9, Xo)}
    stages = {}
    for name, (si, so) in stage_io.items():
        torch.cuda.nvtx.range_push(f"stage_{name}")
        ms_s = plan.time_stage(name, si, so, reps=max(5, min(a.steps // 2, 200)))
        torch.cuda.nvtx.range_pop()
        gbs = stage_bytes[name] / (ms_s / 1e3) / 1e9
        stages[name] = {"ms": ms_s, "alg_bytes": stage_bytes[name], "GB_s": gbs, "frac": gbs / hbm}
    dom = max(stages, key=lambda k: stages[k]["ms"])
    traffic = _stage_traffic(dom, a.config)

    # end to end through the public API with host buffers
    y_host = P.y.cpu().pin_memory()
    eps = P.eps
    y_dev = torch.empty_like(P.y)
    st.solve(1, graph=True)
    torch.cuda.synchronize()
    e2e_steps = max(5, min(a.steps // 2, 300))
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        y_dev.copy_(y_host, non_blocking=True)
        st.set_data(y_dev, eps)
        st.solve(1, graph=True)
        _, b_, r_ = st.get(X=Xo)
    torch.cuda.synchronize()
    e2e_s = (time.perf_counter() - t0) / e2e_steps
    h2d = M * y_dev.element_size()
    d2h = 8 + 8 * L

    # model variants and the re-weighting step on the same problem (FP32, graph replay)
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

    kv = max(5, min(a.steps // 4, 200))
    variants = {}
    for name, kw in (("lr", dict(use_l21=False)), ("jas", dict(use_nuclear=False)),
                     ("sara", dict(use_nuclear=False, sparsity="l1"))):
        sv_ = hs.PDState(plan, P.y, P.eps, tau=0.33, kappa3=P.kappa3, mu=P.mu, **kw)
        variants[name] = {"value": _iter_rate(sv_, kv), "unit": UNIT}
        sv_.close()
    w21 = torch.ones((9, plan.ny, plan.nx), dtype=torch.float32, device="cuda")
    wnu = torch.ones(L, dtype=torch.float64, device="cuda")
    st_rw = hs.PDState(plan, P.y, P.eps, tau=0.33, kappa3=P.kappa3, mu=P.mu, w_nuc=wnu, w_l21=w21)
    st_rw.solve(20, graph=True)
    torch.cuda.synchronize()
    r0 = torch.cuda.Event(enable_timing=True)
    r1 = torch.cuda.Event(enable_timing=True)
    r0.record(stream)
    for _ in range(5):
        st_rw.reweight(0.8, 0.8, w21, wnu)
    r1.record(stream)
    torch.cuda.synchronize()
    variants["reweight_ms"] = r0.elapsed_time(r1) / 5
    variants["reweighted_lrjas_iter_per_s"] = _iter_rate(st_rw, kv)
    st_rw.close()

    # plain FP64 GPU form of the same iteration
    fp64 = None
    if not a.no_fp64:
        P64 = dprob.build(inp, prec="f64", power_iters=60, power_tol=1e-4)
        st64 = hs.PDState(P64.plan, P64.y, P64.eps, tau=0.33, kappa3=P64.kappa3, mu=P64.mu)
        st64.solve(2, graph=True)
        torch.cuda.synchronize()
        k64 = max(3, min(a.steps // 10, 50))
        g0 = torch.cuda.Event(enable_timing=True)
        g1 = torch.cuda.Event(enable_timing=True)
        g0.record(stream)
        st64.solve(k64, graph=True)
        g1.record(stream)
        torch.cuda.synchronize()
        fp64 = {"value": k64 / (g0.elapsed_time(g1) / 1e3), "unit": UNIT, "steps": k64,
                "speedup_fp32_over_fp64": value / world / (k64 / (g0.elapsed_time(g1) / 1e3))}
        st64.close()
        P64.plan.close()

    if rank != 0:
        return
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": a.steps,
        "warmup": a.warmup, "ms_per_step": ms / a.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": _workload(a.config),
        "roofline": {"bound": "hbm", "achieved": stages[dom]["GB_s"], "peak": hbm, "unit": "GB/s",
                     "frac": stages[dom]["frac"], "traffic": traffic, "kernel": dom,
                     "alg_bytes_per_launch": stages[dom]["alg_bytes"], "launch_ms": stages[dom]["ms"],
                     "peak_source": peak_src},
        "stages": stages,
        "phi_pair": {"ms": pair_ms, "alg_bytes": pair_bytes, "GB_s": pair_gbs, "frac": pair_gbs / hbm},
        "phi_vis_per_s": phi_vis, "phi_pair_ms": pair_ms,
        "e2e": {"value": 1.0 / e2e_s, "unit": UNIT, "h2d_bytes_per_step": h2d,
                "d2h_bytes_per_step": d2h},
        "gpu_launches": kern_per_step * a.steps,
        "kernels_per_step": kern_per_step,
        "clocks": clocks,
        "asnr_db": asnr, "beta": beta, "mu": P.mu, "kappa3": P.kappa3,
        "fp64": fp64,
        "variants": variants,
        "cpu_baseline": cpu,
    }
    print(json.dumps(line), flush=True)


def main():
    a = _args()
    if a.impl == "reference":
        run_reference(a)
    else:
        run_ours(a)


if __name__ == "__main__":
    main()
