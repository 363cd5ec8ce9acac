"""Benchmark: TLR Matern log-likelihood evaluations per second at n = 40,000.

One step is one pass of the whole hot path over the resident inputs:
Hilbert ordering of the 40,000 locations, permutation of the locations and of
Z, then l(theta) of Eq. 1.2 (Matern tiles generated inside the TLR Cholesky
update, per-tile compression at eps, TLR Cholesky, forward solve and
log-determinant), with theta moved along a fixed log-space walk so that
nothing carries over between steps.

Workload: 200 x 200 perturbed grid (n = 40,000), Matern sigma2 = 1,
beta = 0.1, nu = 0.5 (medium correlation) as the walk's start, tile 800,
eps = 1e-7, FP64.  Z = L w is drawn once from the library's own TLR factor
at the starting theta (eps = 1e-9), w ~ N(0, I) seeded.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]
Multi-GPU (torchrun): replicas, one dataset per rank (seed 1 + rank), no
collective on the data path; value = evaluations of all ranks / max time.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "TLR ℓ(θ) evals/s at n=40k vs FP64 path (|Δℓ|/|ℓ|≤1e-6); p50/p99 latency"
UNIT = "evals/s"
N_POINTS = 40000
NB = 800
EPS = 1e-7
THETA0 = (1.0, 0.1, 0.5)
ORDER = "hilbert"
L2_FLUSH_BYTES = 256 << 20


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except Exception:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0,
                "sm_max_mhz": 2070.0}, "fallback"


class ClockSampler:
    """nvidia-smi clock / throttle sampling during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device: int):
        self.device = device
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.device), "--query-gpu=" + self.Q,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            out, _ = self.proc.communicate(timeout=5)
        except Exception:
            self.proc.kill()
            out = ""
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in out.splitlines():
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax = float(f[2])
            except ValueError:
                continue
            for name, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(name)
        sm.sort()
        med = sm[len(sm) // 2] if sm else None
        return {"sm_mhz": med, "sm_max_mhz": smax, "reasons": sorted(reasons), "samples": len(sm)}


def aggregate(total_ms: float, steps: int, world: int, device=None) -> tuple:
    """Whole-job throughput of `world` replicas: every rank ran `steps`
    evaluations; the job's time is the slowest rank's (max over ranks).
    Returns (evals_per_s, max_total_ms).  With world > 1 a process group must
    be initialised (NCCL on GPUs, gloo on CPUs)."""
    if world > 1:
        import torch
        import torch.distributed as dist
        t = torch.tensor([float(total_ms)], dtype=torch.float64, device=device)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        total_ms = float(t.item())
    return world * steps / (total_ms / 1000.0), total_ms


def dataset_seeds(rank: int) -> tuple:
    """Replica r evaluates its own dataset: locations seed 1 + r, w seed 2 + r."""
    return 1 + rank, 2 + rank


def make_inputs(tlr, ctx, torch, dev, rank: int):
    """Locations (generation order) and Z = L(theta0) w drawn with the library's factor."""
    import numpy as np
    import synth
    s_loc, s_w = dataset_seeds(rank)
    xy_h = synth.jittered_grid(N_POINTS, seed=s_loc)
    w_h = synth.standard_normal(N_POINTS, seed=s_w)
    xy = torch.from_numpy(xy_h).to(dev)
    w = torch.from_numpy(w_h).to(dev)
    xyo = torch.empty_like(xy)
    perm = tlr.tlr_order(ctx, xy, ORDER, xy_out=xyo)
    L = tlr.TlrMatrix(ctx, N_POINTS, NB)
    zero = torch.zeros(N_POINTS, dtype=torch.float64, device=dev)
    tlr.tlr_loglik(L, xyo, zero, THETA0, tlr.Options(nb=NB, eps=1e-9))
    z_ord = tlr.tlr_lmul(L, w)
    z = torch.empty_like(z_ord)
    z[perm] = z_ord  # back to generation order
    torch.cuda.synchronize()
    L.close()
    return xy_h, xy, z


def run_gpu(args):
    import numpy as np
    import torch
    import paper_2402_09356_gb300 as tlr
    import synth

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    ctx = tlr.Context(local)
    stream = torch.cuda.current_stream()
    xy_h, xy, z = make_inputs(tlr, ctx, torch, dev, rank)
    thetas = synth.theta_walk(THETA0, args.warmup + args.steps, seed=7, scale=0.05)
    opts = tlr.Options(nb=NB, eps=EPS)
    L = tlr.TlrMatrix(ctx, N_POINTS, NB)
    xyo = torch.empty_like(xy)
    perm = torch.empty(N_POINTS, dtype=torch.int64, device=dev)
    zo = torch.empty_like(z)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)

    def step(theta):
        tlr.tlr_order(ctx, xy, ORDER, perm=perm, xy_out=xyo)
        tlr.tlr_gather(ctx, perm, z, dst=zo)
        return tlr.tlr_loglik(L, xyo, zo, theta, opts)

    for k in range(args.warmup):
        step(thetas[k])
    torch.cuda.synchronize()

    # timed region: every step bracketed by CUDA events on the launching stream;
    # the L2 is flushed (256 MB write) between steps, outside the events
    tlr.tlr_profile(ctx, True)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    results, gemm_ms, gemm_flops, panel_launches = [], 0.0, 0.0, 0
    stage_ms = {k: 0.0 for k in tlr.STAGES}
    comp_ms = {k: 0.0 for k in tlr.COMPRESS_STEPS}
    comp_stats = {k: 0 for k in tlr.COMPRESS_STATS}
    clocks = ClockSampler(local)
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    launches0 = tlr.tlr_launch_count()
    clocks.start()
    for k in range(args.steps):
        flush.zero_()
        ev[k][0].record(stream)
        r = step(thetas[args.warmup + k])
        ev[k][1].record(stream)
        prof = tlr.tlr_profile(ctx, True)
        gemm_ms += prof["gemm_ms"]
        gemm_flops += prof["gemm_flops"]
        panel_launches += prof["panel_launches"]
        for name, v in tlr.tlr_stage_times(ctx).items():
            stage_ms[name] += v / args.steps
        for name, v in tlr.tlr_compress_times(ctx).items():
            comp_ms[name] += v / args.steps
        for name, v in tlr.tlr_compress_stats(ctx).items():
            comp_stats[name] = max(comp_stats[name], v) if name == "max_sweeps" else comp_stats[name] + v
        results.append(r)
    torch.cuda.synchronize()
    clk = clocks.stop()
    launches = tlr.tlr_launch_count() - launches0
    times = [a.elapsed_time(b) for a, b in ev]
    value, total_ms = aggregate(sum(times), args.steps, world, device=dev)
    if world > 1:
        torch.distributed.barrier()

    # end to end through the public API with host buffers: pinned host inputs
    # copied in every step, the result read back on the host
    xy_pin = torch.from_numpy(xy_h).pin_memory()
    z_pin = z.cpu().pin_memory()
    xy_dev = torch.empty_like(xy)
    z_dev = torch.empty_like(z)
    e2e_steps = max(1, min(args.steps, 5))
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for k in range(e2e_steps):
        xy_dev.copy_(xy_pin, non_blocking=True)
        z_dev.copy_(z_pin, non_blocking=True)
        tlr.tlr_order(ctx, xy_dev, ORDER, perm=perm, xy_out=xyo)
        tlr.tlr_gather(ctx, perm, z_dev, dst=zo)
        tlr.tlr_loglik(L, xyo, zo, thetas[args.warmup + k], opts)  # result returned on the host
    torch.cuda.synchronize()
    e2e_s = time.perf_counter() - t0
    e2e_value = world * e2e_steps / e2e_s if world == 1 else e2e_steps / e2e_s * world

    pk, pk_kind = peaks()
    # FP64 peak of the DFMA pipe: 152 SMs x 2 DFMA/clk x 2 flop at the sampled SM clock
    sm_mhz = clk.get("sm_mhz") or pk.get("sm_max_mhz", 2070.0)
    n_sms = torch.cuda.get_device_properties(dev).multi_processor_count
    fp64_peak_tflops = n_sms * 4 * sm_mhz * 1e6 / 1e12
    avg_launch_ms = gemm_ms / max(panel_launches, 1)
    achieved_tflops = (gemm_flops / max(panel_launches, 1)) / (avg_launch_ms / 1000.0) / 1e12 if gemm_ms > 0 else 0.0
    p50 = float(np.percentile(times, 50))
    p99 = float(np.percentile(times, 99))
    line = {
        "metric": METRIC,
        "value": value,
        "unit": UNIT,
        "n_gpus": world,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": total_ms / args.steps,
        "p50_ms": p50,
        "p99_ms": p99,
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": "ordering study FP64, n=%d (perturbed grid), Matern sigma2=1 beta=0.1 nu=0.5 "
                               "walk start, %s, tile %d, eps %g" % (N_POINTS, ORDER, NB, EPS),
                   "n": N_POINTS, "nb": NB, "eps": EPS, "ordering": ORDER, "theta0": list(THETA0),
                   "theta_walk": "log-space, scale 0.05/step, seed 7",
                   "l2": "flushed between timed steps (256 MB write outside the events)",
                   "parallelism": "replicas" if world > 1 else "single GPU"},
        "stage_ms_per_step": stage_ms,
        "compress_ms_per_step": comp_ms,
        "compress_per_step": {"tiles": comp_stats["tiles"] / args.steps, "rounds": comp_stats["rounds"] / args.steps,
                              "mean_sweeps": comp_stats["sweeps"] / max(comp_stats["tiles"], 1),
                              "max_sweeps": comp_stats["max_sweeps"]},
        "loglik_last": results[-1]["loglik"],
        "max_rank_last": results[-1]["max_rank"],
        "mean_rank_last": results[-1]["mean_rank"],
        "offdiag_mb_last": results[-1]["offdiag_bytes"] / 1e6,
        "rel_dl_vs_fp64": 0.0,
        "clocks": clk,
        "e2e": {"value": e2e_value, "unit": UNIT, "steps": e2e_steps,
                "h2d_bytes_per_step": int(xy_pin.numel() * 8 + z_pin.numel() * 8),
                "d2h_bytes_per_step": 8 * 3},
        "gpu_launches": int(launches),
        "roofline": {"bound": "alu", "kernel": "k_gemm_f64<EpiMatern> (panel update + Matern generation)",
                     "achieved": achieved_tflops, "peak": fp64_peak_tflops, "unit": "TFLOP/s",
                     "frac": achieved_tflops / fp64_peak_tflops if fp64_peak_tflops else None,
                     "traffic": None,
                     "peak_source": "FP64 DFMA pipe: %d SMs x 4 flop/clk x %.0f MHz (sampled SM clock)"
                                    % (n_sms, sm_mhz),
                     "launch_ms_avg": avg_launch_ms, "launches": panel_launches,
                     "flops_per_launch": gemm_flops / max(panel_launches, 1)},
    }
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline_sample()
    if rank == 0:
        print(json.dumps(line), flush=True)
    L.close()
    ctx.close()
    if world > 1:
        torch.distributed.destroy_process_group()


def cpu_baseline_sample(n_sample: int = 6400, theta=THETA0):
    """The oracle (dense FP64 Cholesky likelihood) on a bounded sample, scaled to n = 40,000.

    Sample: n = 6,400 (80 x 80 perturbed grid).  The covariance fill is scaled
    by (40000/6400)^2, the Cholesky + solve by (40000/6400)^3.
    """
    import numpy as np
    import oracle
    import synth
    xy = synth.jittered_grid(n_sample, seed=1)
    z = synth.standard_normal(n_sample, seed=2)
    t0 = time.perf_counter()
    S = oracle.cov_matrix(xy, theta)
    t1 = time.perf_counter()
    oracle.loglik_from_cov(S, z)
    t2 = time.perf_counter()
    f = N_POINTS / n_sample
    est = (t1 - t0) * f ** 2 + (t2 - t1) * f ** 3
    return {"value": 1.0 / est, "unit": UNIT, "cores": os.cpu_count(), "kind": "oracle",
            "sample": "dense FP64 oracle at n=6400 (80x80 grid): Matern fill %.2fs x (40000/6400)^2, "
                      "Cholesky+solve %.2fs x (40000/6400)^3 -> %.1fs per n=40k evaluation"
                      % (t1 - t0, t2 - t1, est)}


def run_reference(args):
    """Reference arm: the CPU oracle as it stands, on bounded samples of the same workload."""
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    for _ in range(args.warmup):
        cpu_baseline_sample(n_sample=3200)
    vals = []
    t0 = time.perf_counter()
    for _ in range(args.steps):
        vals.append(cpu_baseline_sample(n_sample=3200))
    wall = time.perf_counter() - t0
    v = sum(x["value"] for x in vals) / len(vals)
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000.0 / v,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": "dense FP64 oracle likelihood, n=3200 samples scaled to n=40,000",
                       "n": N_POINTS, "theta0": list(THETA0)},
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": os.cpu_count(), "kind": "oracle",
                             "sample": vals[-1]["sample"].replace("6400", "3200")},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
            "wall_s": wall}
    print(json.dumps(line), flush=True)


def main():
    global N_POINTS, NB, EPS, ORDER
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--n", type=int, default=N_POINTS, help="locations (profiling of smaller cases)")
    ap.add_argument("--nb", type=int, default=NB)
    ap.add_argument("--eps", type=float, default=EPS)
    ap.add_argument("--order", default=ORDER)
    args = ap.parse_args()
    N_POINTS, NB, EPS, ORDER = args.n, args.nb, args.eps, args.order
    if args.impl == "reference":
        run_reference(args)
        return
    from paper_2402_09356_gb300 import build as lib_build
    lib_build.build()
    run_gpu(args)


if __name__ == "__main__":
    main()
