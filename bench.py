"""Benchmark: TLR Matern log-likelihood evaluations per second at n = 40,000.

One step is one pass of the whole hot path over the resident inputs:
Hilbert ordering of the 40,000 locations, permutation of the locations and of
Z, then l(theta) of Eq. 1.2 (Matern tiles generated inside the TLR Cholesky
update, per-tile compression at eps, TLR Cholesky, forward solve and
log-determinant), with theta moved along a fixed log-space walk so that
nothing carries over between steps.

Workload: 200 x 200 perturbed grid (n = 40,000), Matern sigma2 = 1,
beta = 0.1, nu = 0.5 (medium correlation) as the walk's start, tile 800,
eps = 1e-7.  Z = L w is drawn once from the library's own TLR factor at the
starting theta (eps = 1e-9), w ~ N(0, I) seeded.

Both precision paths run the same K steps at the same thetas: FP64 and mixed
(paired-FP32 off-diagonal products).  The headline value is the mixed path
when every step keeps |l_mixed - l_fp64| <= 1e-6 |l_fp64|, else the FP64 path.

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
# DRAM bytes (read + write) per launch from ncu captures of unchanged kernels,
# by (kernel, tile size); the capture and its command are in profiles/
NCU_TRAFFIC = {("k_potrf_inv<16, 1>", 800): (3.34e6, "profiles/k_potrf_inv_n16000.md")}


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


def aggregate_units(units: float, seconds: float, world: int, device=None) -> tuple:
    """Whole-job throughput of a sharded workload: every rank evaluated its own
    `units` in `seconds`; the job's units are the sum over ranks and its time
    the slowest rank's.  Returns (units_per_s, total_units, max_seconds)."""
    if world > 1:
        import torch
        import torch.distributed as dist
        u = torch.tensor([float(units)], dtype=torch.float64, device=device)
        t = torch.tensor([float(seconds)], dtype=torch.float64, device=device)
        dist.all_reduce(u, op=dist.ReduceOp.SUM)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        units, seconds = float(u.item()), float(t.item())
    return units / seconds, units, seconds


def shard_batched(sizes, world: int, maxrank: int = 0, nb: int = 512):
    """Rank of every dataset of the batched workload: placed by HBM footprint
    (tlr_pool_footprint at the nominal tile size: resident data, factor,
    workspace) with the library's largest-first rule.  Every rank computes
    the same placement; nothing is exchanged."""
    import paper_2402_09356_gb300 as tlr
    fp = []
    for n in sizes:
        f = tlr.tlr_pool_footprint(int(n), nb, maxrank if maxrank > 0 else 0)
        fp.append(f["base"] + f["factor"] + f["work"])
    return tlr.tlr_shard_place(fp, world), fp


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


def algorithmic_flops(ranks, n: int, nb: int) -> dict:
    """The method's work per evaluation counted from a rank map (the factor's
    r_ij, i > j), term by term as the TLR Cholesky of Sec. 2 needs it:
      compression  4 m_i m_j r_ij per off-diagonal tile (RRQR-class);
      POTRF        m_k^3 / 3 per diagonal tile;
      TRSM         m_i m_k r_ik (V_ik <- L_kk^-1 V_ik);
      SYRK         2 m_i m_k r_ik (D_ii -= U_ik (V_ik' V_ik) U_ik');
      GEMM         2 m_k r_ik r_jk (V_ik' V_jk) + 8 m (r_ij + r_ik)^2 for the
                   recompression of A_ij -= U_ik (V_ik' V_jk) U_jk', i > j > k.
    Executed work differs (explicit inverses, densified panels, sampling)."""
    import numpy as np
    r = np.asarray(ranks, dtype=np.float64)
    nt = r.shape[0]
    m = np.array([min(nb, n - t * nb) for t in range(nt)], dtype=np.float64)
    low = np.tril(r, -1)
    comp = float((4.0 * m[:, None] * m[None, :] * low).sum())
    potrf = float((m ** 3 / 3.0).sum())
    trsm = float((m[:, None] * m[None, :] * low).sum())
    syrk = 2.0 * trsm
    gemm = 0.0
    for k in range(nt - 2):
        rk = low[k + 1:, k]                       # r_ik, i > k
        mi = m[k + 1:]
        prod = 2.0 * m[k] * np.outer(rk, rk)      # V_ik' V_jk, i > j > k
        rij = low[k + 1:, k + 1:]                 # r_ij for rows i, cols j (both > k)
        rec = 8.0 * mi[:, None] * (rij + rk[:, None]) ** 2
        mask = np.tril(np.ones((nt - k - 1, nt - k - 1)), -1)
        gemm += float(((prod + rec) * mask).sum())
    total = comp + potrf + trsm + syrk + gemm
    return {"total": total, "compression": comp, "potrf": potrf, "trsm": trsm, "syrk": syrk, "gemm": gemm}


def draw_z_lw(tlr, ctx, xy_h, w_h, theta, order, nb):
    """Data drawn from the model, Z = L(theta) w (generation order, host array):
    L is the library's own TLR factor at eps 1e-9 (maxrank nb), so that the
    quadratic term has the size the model gives it (|w|^2 ~ n).  A covariance
    too ill-conditioned for that factor is retried at eps 1e-7; if that fails
    too, Z = w is returned and the second value is False."""
    import numpy as np
    import torch
    dev = torch.device("cuda", ctx.device)
    n = w_h.size
    xy = torch.from_numpy(xy_h).to(dev)
    xyo = torch.empty_like(xy)
    perm = tlr.tlr_order(ctx, xy, order, xy_out=xyo)
    zero = torch.zeros(n, dtype=torch.float64, device=dev)
    for eps in (1e-9, 1e-7):
        L = tlr.TlrMatrix(ctx, n, nb, maxrank=nb)
        try:
            tlr.tlr_loglik(L, xyo, zero, tuple(theta), tlr.Options(nb=nb, eps=eps, maxrank=nb))
            zo = tlr.tlr_lmul(L, tlr.tlr_gather(ctx, perm, torch.from_numpy(w_h).to(dev)))
            z = torch.empty_like(zo)
            z[perm] = zo
            return z.cpu().numpy(), True
        except tlr.TlrError:
            torch.cuda.synchronize()
        finally:
            L.close()
    return np.array(w_h, dtype=np.float64), False


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
    if args.qr_sizes or args.svd_sizes:
        bk = tlr.tlr_ctx_get_buckets(ctx)
        if args.qr_sizes:
            bk["qr_size"] = [int(v) for v in args.qr_sizes.split(",")]
        if args.svd_sizes:
            bk["svd_size"] = [int(v) for v in args.svd_sizes.split(",")]
        tlr.tlr_ctx_set_buckets(ctx, bk)
    stream = torch.cuda.current_stream()
    xy_h, xy, z = make_inputs(tlr, ctx, torch, dev, rank)
    thetas = synth.theta_walk(THETA0, args.warmup + args.steps, seed=7, scale=0.05)
    L = tlr.TlrMatrix(ctx, N_POINTS, NB)
    xyo = torch.empty_like(xy)
    perm = torch.empty(N_POINTS, dtype=torch.int64, device=dev)
    zo = torch.empty_like(z)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    precisions = {"mixed": tlr.TLR_PREC_MIXED, "fp64": tlr.TLR_PREC_FP64, "tensor": tlr.TLR_PREC_TENSOR}

    def step(theta, opts):
        tlr.tlr_order(ctx, xy, ORDER, perm=perm, xy_out=xyo)
        tlr.tlr_gather(ctx, perm, z, dst=zo)
        return tlr.tlr_loglik(L, xyo, zo, theta, opts)

    def timed(prec: str) -> dict:
        """W untimed warm-up steps, then K steps each bracketed by CUDA events on
        the launching stream; the L2 is flushed (256 MB write) between steps,
        outside the events."""
        opts = tlr.Options(nb=NB, eps=EPS, precision=precisions[prec])
        for k in range(args.warmup):
            step(thetas[k], opts)
        torch.cuda.synchronize()
        tlr.tlr_profile(ctx, True)
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
        out = {"results": [], "gemm_ms": 0.0, "gemm_flops": 0.0, "panel_launches": 0,
               "stage_ms": {k: 0.0 for k in tlr.STAGES}, "comp_ms": {k: 0.0 for k in tlr.COMPRESS_STEPS},
               "detail_ms": {k: 0.0 for k in tlr.DETAILS},
               "k16": {"jacobi16_ms": 0.0, "jacobi16_flops": 0.0, "jacobi16_launches": 0, "jacobi16_clusters": 0},
               "comp_stats": {k: 0 for k in tlr.COMPRESS_STATS}}
        clocks = ClockSampler(local)
        if world > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()
        launches0 = tlr.tlr_launch_count()
        clocks.start()
        for k in range(args.steps):
            flush.zero_()
            ev[k][0].record(stream)
            r = step(thetas[args.warmup + k], opts)
            ev[k][1].record(stream)
            prof = tlr.tlr_profile(ctx, True)
            out["gemm_ms"] += prof["gemm_ms"]
            out["gemm_flops"] += prof["gemm_flops"]
            out["panel_launches"] += prof["panel_launches"]
            for name, v in tlr.tlr_stage_times(ctx).items():
                out["stage_ms"][name] += v / args.steps
            for name, v in tlr.tlr_compress_times(ctx).items():
                out["comp_ms"][name] += v / args.steps
            for name, v in tlr.tlr_detail_times(ctx).items():
                out["detail_ms"][name] += v / args.steps
            for name, v in tlr.tlr_kernel_stats(ctx).items():
                out["k16"][name] += v
            for name, v in tlr.tlr_compress_stats(ctx).items():
                cs = out["comp_stats"]
                cs[name] = max(cs[name], v) if name == "max_sweeps" else cs[name] + v
            out["results"].append(r)
        torch.cuda.synchronize()
        out["clocks"] = clocks.stop()
        out["launches"] = tlr.tlr_launch_count() - launches0
        out["times"] = [a.elapsed_time(b) for a, b in ev]
        out["ranks"] = tlr.tlr_mat_ranks(L)  # the last step's factor
        out["value"], out["total_ms"] = aggregate(sum(out["times"]), args.steps, world, device=dev)
        if world > 1:
            torch.distributed.barrier()
        tlr.tlr_profile(ctx, False)
        return out

    want = ("fp64", "mixed", "tensor") if args.paths in ("all", "both") else (args.paths,)
    runs = {name: timed(name) for name in want}
    fp64, mixed, tensor = runs.get("fp64"), runs.get("mixed"), runs.get("tensor")
    rel = {}
    if fp64 is not None:
        for name in ("mixed", "tensor"):
            if runs.get(name) is not None:
                rel[name] = max(abs(a["loglik"] - b["loglik"]) / abs(b["loglik"])
                                for a, b in zip(runs[name]["results"], fp64["results"]))
        # the headline: the fastest mixed path that keeps |dl|/|l| <= 1e-6 against
        # the FP64 path at every step, else the FP64 path
        ok = [name for name, r in rel.items() if r <= 1e-6]
        head_name = max(ok, key=lambda nm: runs[nm]["value"]) if ok else "fp64"
    else:
        head_name = want[0]  # one path only (profiling runs)
    rel_dl = rel.get(head_name) if head_name != "fp64" else (max(rel.values()) if rel else None)
    head = runs[head_name]
    head_opts = tlr.Options(nb=NB, eps=EPS, precision=precisions[head_name])

    # end to end through the C ABI with HOST buffers (tlr_loglik_host): the
    # pinned host inputs are copied to the device inside every call, ordered,
    # permuted and evaluated; the result comes back on the host
    xy_pin = torch.from_numpy(xy_h).pin_memory()
    z_pin = z.cpu().pin_memory()
    e2e_steps = max(1, min(args.steps, 10))
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for k in range(e2e_steps):
        tlr.tlr_loglik_host(L, xy_pin, z_pin, thetas[args.warmup + k], head_opts, order=ORDER)
    torch.cuda.synchronize()
    e2e_s = time.perf_counter() - t0
    e2e_value = world * e2e_steps / e2e_s

    clk = head["clocks"]
    sm_mhz = clk.get("sm_mhz") or peaks()[0].get("sm_max_mhz", 2070.0)
    n_sms = torch.cuda.get_device_properties(dev).multi_processor_count
    fp64_peak = n_sms * 4 * sm_mhz * 1e6 / 1e12  # 2 DFMA per clock per SM
    # paired-FP32 product: 12 FP32 instructions per emulated multiply-add on
    # 128 FP32 lanes per SM per clock
    df_peak = n_sms * 128 * 2 / 12 * sm_mhz * 1e6 / 1e12
    # tensor path: 15 BF16 slice-pair products per FP64-equivalent product,
    # against the measured sustained BF16 rate
    pk, pk_src = peaks()
    tc_peak = pk["bf16_tflops_sustained"] / 15.0

    def roof_panel(o):
        launches = max(o["panel_launches"], 1)
        avg = o["gemm_ms"] / launches
        fl = o["gemm_flops"] / launches
        achieved = fl / (avg / 1000.0) / 1e12 if avg > 0 else 0.0
        if o is tensor:
            name = ("k_gemm_tc<5,2,TcEpiLinear> (panel update: FP64 covariance panel by k_generate_panel, operand "
                    "splits, then T -= P Q' as tcgen05 products of 5 BF16 slices, 15 slice pairs; the time covers "
                    "all three)")
            peak, src = tc_peak, ("bf16_tflops_sustained %.1f of MEASURED_PEAKS.json (%s) / 15 slice-pair "
                                  "products per FP64-equivalent product" % (pk["bf16_tflops_sustained"], pk_src))
        elif o is mixed:
            name = "k_gemm_df<64,64,N,T,EpiMatern> (panel update + Matern generation, paired-FP32 products)"
            peak, src = df_peak, ("FP32 pipe for paired-FP32 products: %d SMs x 128 lanes x 2 flop / 12 instr "
                                  "per emulated FMA x %.0f MHz (sampled SM clock)" % (n_sms, sm_mhz))
        else:
            name = "k_gemm_f64<64,64,N,T,EpiMatern> (panel update + Matern generation)"
            peak, src = fp64_peak, "FP64 DFMA pipe: %d SMs x 4 flop/clk x %.0f MHz (sampled SM clock)" % (n_sms, sm_mhz)
        return {"bound": "alu", "kernel": name, "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                "frac": achieved / peak if peak else None, "traffic": None, "peak_source": src,
                "launch_ms_avg": avg, "launches": o["panel_launches"], "flops_per_launch": fl,
                "total_ms": o["gemm_ms"]}

    def roof_jacobi(o):
        k = o["k16"]
        launches = max(k["jacobi16_launches"], 1)
        avg = k["jacobi16_ms"] / launches
        fl = k["jacobi16_flops"] / launches
        achieved = fl / (avg / 1000.0) / 1e12 if avg > 0 else 0.0
        clusters = k["jacobi16_clusters"] / launches
        occupied = min(n_sms, 16 * clusters) * 4 * sm_mhz * 1e6 / 1e12
        return {"bound": "alu", "kernel": "k_jacobi_sm<16> (cluster Jacobi SVD of the high-rank tiles)",
                "achieved": achieved, "peak": fp64_peak, "unit": "TFLOP/s",
                "frac": achieved / fp64_peak if fp64_peak else None, "traffic": None,
                "peak_source": "FP64 DFMA pipe: %d SMs x 4 flop/clk x %.0f MHz (sampled SM clock)" % (n_sms, sm_mhz),
                "frac_of_occupied_sms": achieved / occupied if occupied else None,
                "clusters_per_launch": clusters, "launch_ms_avg": avg, "launches": k["jacobi16_launches"],
                "flops_per_launch": fl, "total_ms": k["jacobi16_ms"],
                "flops_counted": "FP64 work as executed: M J (2 s^3), norms per sweep (2 s^2), "
                                 "2 s per pair checked, 6 s per pair rotated"}

    def roof_potrf(o):
        # one launch per tile column on the side stream: L = chol(T_jj) (the
        # algorithmic m^3/3 FP64 flops) and L^-1 (another m^3/3, executed work
        # that replaces the TRSM); its in-step time from the events around it
        # on that stream
        nt = (N_POINTS + NB - 1) // NB
        ms_step = o["detail_ms"]["potrf"]
        avg = ms_step / nt
        ms = [min(NB, N_POINTS - t * NB) for t in range(nt)]
        fl = sum(m ** 3 / 3.0 for m in ms) / nt
        achieved = fl / (avg / 1000.0) / 1e12 if avg > 0 else 0.0
        occupied = 16 * 4 * sm_mhz * 1e6 / 1e12
        traffic = NCU_TRAFFIC.get(("k_potrf_inv<16, 1>", NB))
        return {"bound": "alu", "kernel": "k_potrf_inv<16, 1> (diagonal tile: Cholesky in FP64, its inverse in "
                                          "float-float pairs on the paired paths; one 16-CTA cluster)",
                "achieved": achieved, "peak": fp64_peak, "unit": "TFLOP/s",
                "frac": achieved / fp64_peak if fp64_peak else None,
                "traffic": traffic[0] if traffic else None,
                "traffic_source": traffic[1] if traffic else None,
                "peak_source": "FP64 DFMA pipe: %d SMs x 4 flop/clk x %.0f MHz (sampled SM clock)" % (n_sms, sm_mhz),
                "frac_of_occupied_sms": achieved / occupied if occupied else None,
                "launch_ms_avg": avg, "launches": nt * args.steps, "flops_per_launch": fl,
                "flops_counted": "algorithmic: m^3/3 (Cholesky of the diagonal tile)",
                "executed_flops_per_launch": 2.0 * fl,
                "executed_tflops": 2.0 * achieved,
                "executed_note": "the launch also forms L^-1 (another m^3/3), used in place of a TRSM",
                "total_ms": ms_step * args.steps}

    # the dominant kernel of the headline path: the largest device time per step
    cand = [roof_panel(head), roof_jacobi(head), roof_potrf(head)]
    roofline = max(cand, key=lambda r: r["total_ms"])
    other = [r for r in cand if r is not roofline]

    def eval_roofline(o, name):
        """Whole evaluation: the algorithmic flops of its rank map (Sec. 2 terms,
        algorithmic_flops) over the measured time per evaluation, against the FP64
        pipe and, on the mixed path, the pipe that runs its off-diagonal products."""
        alg = algorithmic_flops(o["ranks"], N_POINTS, NB)
        ms = o["total_ms"] / args.steps
        achieved = alg["total"] / (ms / 1000.0) / 1e12
        r = {"bound": "alu", "flops_algorithmic": alg["total"], "flops_by_term": alg,
             "flops_executed": float(o["results"][-1]["flops"]), "ms_per_eval": ms, "achieved": achieved,
             "unit": "TFLOP/s", "peak_fp64": fp64_peak, "frac_fp64": achieved / fp64_peak,
             "counted_from": "rank map of the last timed evaluation"}
        if name == "mixed":
            r["peak_products"] = df_peak
            r["frac_products"] = achieved / df_peak
            r["peak_products_source"] = "paired-FP32 products on the FP32 pipe (see roofline_other)"
        elif name == "tensor":
            r["peak_products"] = tc_peak
            r["frac_products"] = achieved / tc_peak
            r["peak_products_source"] = "BF16 tensor rate (sustained, measured) / 15 slice-pair products"
        return r

    def summary(o):
        res = o["results"]
        cs = o["comp_stats"]
        return {"evals_per_s": o["value"], "ms_per_step": o["total_ms"] / args.steps,
                "p50_ms": float(np.percentile(o["times"], 50)), "p99_ms": float(np.percentile(o["times"], 99)),
                "stage_ms_per_step": o["stage_ms"], "compress_ms_per_step": o["comp_ms"],
                "detail_ms_per_step": o["detail_ms"],
                "compress_per_step": {"tiles": cs["tiles"] / args.steps, "rounds": cs["rounds"] / args.steps,
                                      "mean_sweeps": cs["sweeps"] / max(cs["tiles"], 1),
                                      "max_sweeps": cs["max_sweeps"],
                                      "mean_sweeps_fp32": cs["sweeps32"] / max(cs["tiles"], 1)},
                "panel_tflops": roof_panel(o)["achieved"], "jacobi16": o["k16"], "gpu_launches": int(o["launches"]),
                "eval_roofline": eval_roofline(o, "tensor" if o is tensor else ("mixed" if o is mixed else "fp64")),
                "loglik_last": res[-1]["loglik"], "max_rank_last": res[-1]["max_rank"],
                "mean_rank_last": res[-1]["mean_rank"], "offdiag_mb_last": res[-1]["offdiag_bytes"] / 1e6}

    # latency over many evaluations: the head path, theta continuing along the
    # walk, each evaluation timed by CUDA events on the launching stream (L2
    # flushed before each, outside the events)
    lat = []
    if args.latency_evals > 0:
        lthetas = synth.theta_walk(THETA0, args.warmup + args.steps + args.latency_evals, seed=7, scale=0.05)
        lev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
               for _ in range(args.latency_evals)]
        for k in range(args.latency_evals):
            flush.zero_()
            lev[k][0].record(stream)
            step(lthetas[args.warmup + args.steps + k], head_opts)
            lev[k][1].record(stream)
        torch.cuda.synchronize()
        lat = [a.elapsed_time(b) for a, b in lev]
    lat_src = lat if lat else head["times"]

    line = {
        "metric": METRIC,
        "value": head["value"],
        "unit": UNIT,
        "n_gpus": world,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": head["total_ms"] / args.steps,
        "p50_ms": float(np.percentile(lat_src, 50)),
        "p99_ms": float(np.percentile(lat_src, 99)),
        "latency": {"evals": len(lat_src), "p50_ms": float(np.percentile(lat_src, 50)),
                    "p90_ms": float(np.percentile(lat_src, 90)), "p99_ms": float(np.percentile(lat_src, 99)),
                    "max_ms": float(max(lat_src)), "path": head_name,
                    "how": "separate loop after the timed steps, theta continuing along the walk, CUDA events "
                           "per evaluation, L2 flushed before each"},
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": {"mixed": "f64 storage, paired-f32 products", "tensor": "f64 storage, bf16x5 tensor products",
                  "fp64": "f64"}[head_name],
        "data": "synthetic",
        "config": {"workload": "TLR Matern log-likelihood, n=%d (perturbed grid), Matern sigma2=%g beta=%g nu=%g "
                               "walk start, %s, tile %d, eps %g, %s path" % ((N_POINTS,) + tuple(THETA0) +
                                                                            (ORDER, NB, EPS, head_name)),
                   "n": N_POINTS, "nb": NB, "eps": EPS, "ordering": ORDER, "theta0": list(THETA0),
                   "precision": head_name,
                   "theta_walk": "log-space, scale 0.05/step, seed 7",
                   "l2": "flushed between timed steps (256 MB write outside the events)",
                   "parallelism": "replicas" if world > 1 else "single GPU",
                   "rank_buckets": tlr.tlr_ctx_get_buckets(ctx)},
        "rel_dl_vs_fp64": rel_dl,
        "fp64_path": summary(fp64) if fp64 is not None else None,
        "mixed_path": summary(mixed) if mixed is not None else None,
        "tensor_path": summary(tensor) if tensor is not None else None,
        "rel_dl_vs_fp64_by_path": rel,
        "clocks": clk,
        "e2e": {"value": e2e_value, "unit": UNIT, "steps": e2e_steps,
                "how": "tlr_loglik_host: host buffers in, copies, ordering and evaluation inside the call, "
                       "host clock around the calls",
                "h2d_bytes_per_step": int(xy_pin.numel() * 8 + z_pin.numel() * 8),
                "d2h_bytes_per_step": 8 * 3},
        "gpu_launches": int(head["launches"]),
        "roofline": roofline,
        "roofline_other": other,
    }
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline_sample()
    # compact summary last, so that a truncated log tail still shows both paths
    er = line[head_name + "_path"]["eval_roofline"] if line.get(head_name + "_path") else None
    line["summary"] = {
        "mixed_evals_per_s": mixed["value"] if mixed else None,
        "fp64_evals_per_s": fp64["value"] if fp64 else None,
        "mixed_ms": mixed["total_ms"] / args.steps if mixed else None,
        "tensor_evals_per_s": tensor["value"] if tensor else None,
        "tensor_ms": tensor["total_ms"] / args.steps if tensor else None,
        "fp64_ms": fp64["total_ms"] / args.steps if fp64 else None,
        "rel_dl_vs_fp64": rel_dl, "head": head_name,
        "p50_ms": line["p50_ms"], "p99_ms": line["p99_ms"], "latency_evals": len(lat_src),
        "e2e_evals_per_s": e2e_value,
        "roofline": "%s %.4f of %s" % (roofline["kernel"].split(" ")[0], roofline["frac"] or 0.0, roofline["unit"]),
        "eval_frac_fp64": er["frac_fp64"] if er else None,
        "eval_tflops": er["achieved"] if er else None,
        "loglik_last": head["results"][-1]["loglik"]}
    if rank == 0:
        print(json.dumps(line), flush=True)
    L.close()
    ctx.close()
    if world > 1:
        torch.distributed.destroy_process_group()


def cpu_baseline_sample(n_sample: int = 12800, theta=THETA0, single_thread_c1: bool = True):
    """The oracle (dense FP64 Cholesky likelihood) on a bounded sample, scaled to n = 40,000.

    Sample: n = 12,800 (the first n points of a perturbed 114 x 114 grid), about
    10 s on 16 host cores.  The covariance fill is scaled by (40000/n)^2, the
    Cholesky + solve by (40000/n)^3.  Also times the small workload (n = 1,600,
    40 x 40 grid) on one thread in a child process.
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
    del S
    f = N_POINTS / n_sample
    est = (t1 - t0) * f ** 2 + (t2 - t1) * f ** 3
    side = math.ceil(math.sqrt(n_sample))
    out = {"value": 1.0 / est, "unit": UNIT, "cores": os.cpu_count(), "kind": "oracle",
           "sample": "dense FP64 oracle at n=%d (perturbed %dx%d grid, first n points): Matern fill %.2fs x "
                     "(%d/%d)^2, Cholesky+solve %.2fs x (%d/%d)^3 -> %.1fs per n=%d evaluation"
                     % (n_sample, side, side, t1 - t0, N_POINTS, n_sample, t2 - t1, N_POINTS, n_sample, est,
                        N_POINTS),
           "cpu_model": cpu_model(),
           # the sample's own time, and the share of one full-size evaluation
           # it stands for under the scaling rule above
           "sample_s": t2 - t0, "evals_equiv": (t2 - t0) / est}
    if single_thread_c1:
        out["single_thread_n1600"] = oracle_single_thread(1600)
    return out


def cpu_model() -> str:
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.strip().lower().startswith("model name") and ":" in line:
                return line.split(":", 1)[1].strip()
    except Exception:
        pass
    import platform
    return platform.processor() or platform.machine()


def oracle_single_thread(n: int) -> dict:
    """One dense oracle evaluation (fill + Cholesky + solve) on one thread, in a
    child process whose OpenMP and BLAS pools are pinned to one thread."""
    code = ("import sys, time, json; sys.path.insert(0, %r); import oracle, synth; "
            "xy = synth.jittered_grid(%d, seed=1); z = synth.standard_normal(%d, seed=2); "
            "oracle.loglik_dense(xy, z, %r); t = time.perf_counter(); "
            "r = oracle.loglik_dense(xy, z, %r); print(json.dumps({'s': time.perf_counter() - t, "
            "'loglik': r['loglik']}))" % (ROOT, n, n, tuple(THETA0), tuple(THETA0)))
    env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1")
    try:
        p = subprocess.run([sys.executable, "-c", code], env=env, capture_output=True, text=True, timeout=300)
        r = json.loads(p.stdout.strip().splitlines()[-1])
        return {"n": n, "seconds": r["s"], "evals_per_s": 1.0 / r["s"], "threads": 1}
    except Exception as e:  # reported, never fatal
        return {"n": n, "error": str(e)[:200]}


def run_oracle_fullsize(args):
    """One real dense oracle evaluation at the full size (n = 40,000) on all
    host cores, after no warm-up (one run of about 200 s; not part of the
    default bench).  Prints one JSON line."""
    import oracle
    import synth
    xy = synth.jittered_grid(N_POINTS, seed=1)
    z = synth.standard_normal(N_POINTS, seed=2)
    t0 = time.perf_counter()
    S = oracle.cov_matrix(xy, THETA0)
    t1 = time.perf_counter()
    r = oracle.loglik_from_cov(S, z)
    t2 = time.perf_counter()
    print(json.dumps({"workload": "oracle-fullsize", "n": N_POINTS, "theta": list(THETA0),
                      "fill_s": t1 - t0, "cholesky_solve_s": t2 - t1, "total_s": t2 - t0,
                      "evals_per_s": 1.0 / (t2 - t0), "loglik": r["loglik"], "cores": os.cpu_count(),
                      "cpu_model": cpu_model(),
                      "threads": {k: os.environ.get(k) for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS")}}),
          flush=True)


def run_reference(args):
    """Reference arm: the CPU oracle as it stands, on bounded samples of the same workload."""
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    for _ in range(args.warmup):
        cpu_baseline_sample(n_sample=3200, single_thread_c1=False)
    vals = []
    t0 = time.perf_counter()
    for _ in range(args.steps):
        vals.append(cpu_baseline_sample(n_sample=3200, single_thread_c1=False))
    wall = time.perf_counter() - t0
    # a step is one n = 3,200 sample; it does the share of one n = 40,000
    # evaluation that the fill's n^2 and the factorisation's n^3 give it, so
    # the rate is those shares over the measured time of the steps
    busy = sum(x["sample_s"] for x in vals)
    evals = sum(x["evals_equiv"] for x in vals)
    v = evals / busy
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000.0 * busy / args.steps,
            "evals_per_step": evals / args.steps,
            "step": "one dense FP64 oracle evaluation at n=3200 (fill + Cholesky + solve), counted as "
                    "(3200/40000)^2 of the fill and (3200/40000)^3 of the factorisation of one n=40000 "
                    "evaluation; ms_per_step is its measured time",
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": "Matern log-likelihood, n=%d (perturbed grid), sigma2=%g beta=%g nu=%g: dense "
                                   "FP64 oracle on n=3200 samples scaled to n=%d" % ((N_POINTS,) + tuple(THETA0) +
                                                                                      (N_POINTS,)),
                       "n": N_POINTS, "theta0": list(THETA0)},
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": os.cpu_count(), "kind": "oracle",
                             "sample": vals[-1]["sample"]},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
            "wall_s": wall}
    print(json.dumps(line), flush=True)


# ---- ordering study (Table 1, Sec. 5.2-5.3) ----------------------------------

STUDY_ORDERS = ("random", "morton", "hilbert", "kdtree", "maxmin")
STUDY_NU = (0.5, 1.0)
STUDY_BETA = (0.03, 0.1, 0.3)
STUDY_EPS = (1e-9, 1e-7, 1e-5)
TABLE1_N = (10000, 20000, 30000, 40000)
TABLE1_ORDERS = {"none": "random", "morton": "morton", "hilbert": "hilbert", "kdtree": "kdtree"}


def table1_golden():
    """Table 1's MB per (n, ordering, correlation) from tests/golden/table1_memory.txt."""
    out = {}
    with open(os.path.join(ROOT, "tests", "golden", "table1_memory.txt")) as f:
        for line in f:
            if not line[:1].isdigit():
                continue
            n, order, *vals = line.split()
            out[(int(n), order)] = [None if v == "NA" else float(v) for v in vals]
    return out


def run_ordering_study(args):
    """The ordering study: every ordering x nu in {0.5, 1} x beta in {0.03, 0.1,
    0.3} x eps in {1e-9, 1e-7, 1e-5} at n = 40,000, tile 800, FP64 path.  Per
    point: time per evaluation (CUDA events, after one warm-up that sets the
    rank map), l and its two terms, the factor's rank map (max / mean rank,
    off-diagonal MB) and |dl| against the exact dense l where the oracle has it
    (theta = (1, 0.1, 0.5) with the golden Z = L w), else against the same
    ordering at eps = 1e-9.  Then Table 1's memory of the compressed covariance
    (tile 1000, nu = 0.5, eps 1e-7) for n = 10k..40k beside the paper's values.
    Z per theta: the golden Z where it exists, else Z = L w with L the
    library's TLR factor at eps 1e-9 (Hilbert, maxrank nb), w seed 2.
    A point whose tiles need more than maxrank = nb/2 is "NA" (Table 1's NA)."""
    import numpy as np
    import torch
    import paper_2402_09356_gb300 as tlr
    import synth
    dev = torch.device("cuda", 0)
    ctx = tlr.Context(0)
    stream = torch.cuda.current_stream()
    n, nb = N_POINTS, NB
    xy_h = synth.jittered_grid(n, seed=1)
    w_h = synth.standard_normal(n, seed=2)
    xy = torch.from_numpy(xy_h).to(dev)
    w = torch.from_numpy(w_h).to(dev)
    gold = None
    gpath = os.path.join(ROOT, "tests", "golden", "fullsize_loglik_n%d.json" % n)
    zpath = os.path.join(ROOT, "tests", "golden", "fullsize_z_n%d.npy" % n)
    if os.path.exists(gpath) and os.path.exists(zpath):
        gold = json.load(open(gpath))
        gold["z_arr"] = np.load(zpath)
    orders = [o for o in (args.study_orders.split(",") if args.study_orders else STUDY_ORDERS)]
    rows, rank_maps = [], {}
    t_all = time.perf_counter()

    def draw_z(theta):
        if gold is not None and tuple(gold["theta"]) == tuple(theta):
            return torch.from_numpy(gold["z_arr"]).to(dev), gold
        xyo = torch.empty_like(xy)
        perm = tlr.tlr_order(ctx, xy, "hilbert", xy_out=xyo)
        L = tlr.TlrMatrix(ctx, n, nb, maxrank=nb)
        try:
            tlr.tlr_loglik(L, xyo, torch.zeros(n, dtype=torch.float64, device=dev), theta,
                           tlr.Options(nb=nb, eps=1e-9, maxrank=nb))
            zo = tlr.tlr_lmul(L, tlr.tlr_gather(ctx, perm, w))
            z = torch.empty_like(zo)
            z[perm] = zo
            return z, None
        finally:
            L.close()

    for nu in STUDY_NU:
        for beta in STUDY_BETA:
            theta = (1.0, beta, nu)
            try:
                z, g = draw_z(theta)
            except tlr.TlrError as e:
                rows.append({"theta": list(theta), "error": "Z draw: " + str(e)[:120]})
                continue
            for order in orders:
                xyo = torch.empty_like(xy)
                perm = tlr.tlr_order(ctx, xy, order, xy_out=xyo)
                zo = tlr.tlr_gather(ctx, perm, z)
                ref9 = None
                for eps in STUDY_EPS:
                    row = {"order": order, "nu": nu, "beta": beta, "eps": eps}
                    L = tlr.TlrMatrix(ctx, n, nb)
                    opts = tlr.Options(nb=nb, eps=eps, precision=tlr.TLR_PREC_FP64)
                    try:
                        tlr.tlr_loglik(L, xyo, zo, theta, opts)  # warm-up: rank map
                        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
                              for _ in range(args.study_steps)]
                        for a, b in ev:
                            a.record(stream)
                            r = tlr.tlr_loglik(L, xyo, zo, theta, opts)
                            b.record(stream)
                        torch.cuda.synchronize()
                        ms = [a.elapsed_time(b) for a, b in ev]
                        rk = tlr.tlr_mat_ranks(L)
                        off = rk[np.tril_indices(rk.shape[0], -1)]
                        row.update({"ms_per_eval": float(np.mean(ms)), "loglik": r["loglik"],
                                    "logdet": r["logdet"], "quad": r["quad"], "max_rank": int(off.max()),
                                    "mean_rank": float(off.mean()), "offdiag_mb": r["offdiag_bytes"] / 1e6,
                                    "flops_algorithmic": algorithmic_flops(rk, n, nb)["total"]})
                        rank_maps["%s nu=%g beta=%g eps=%g" % (order, nu, beta, eps)] = rk.tolist()
                        if g is not None:
                            row["dl_vs_exact"] = abs(r["loglik"] - g["loglik"])
                            row["rel_dl_vs_exact"] = row["dl_vs_exact"] / abs(g["loglik"])
                            row["dlogdet_vs_exact"] = abs(r["logdet"] - g["logdet"])
                            row["dquad_vs_exact"] = abs(r["quad"] - g["quad"])
                        if eps == STUDY_EPS[0]:
                            ref9 = r["loglik"]
                        elif ref9 is not None:
                            row["dl_vs_eps1e-9"] = abs(r["loglik"] - ref9)
                    except tlr.TlrError as e:
                        row["status"] = "NA" if e.code == tlr.TLR_ERR_RANK else "error %d" % e.code
                        row["error"] = str(e)[:120]
                        torch.cuda.synchronize()
                    finally:
                        L.close()
                    rows.append(row)
    study_s = time.perf_counter() - t_all

    # Table 1: memory of the compressed covariance, tile 1000, nu 0.5, eps 1e-7
    paper = table1_golden()
    t1 = []
    t_tab = time.perf_counter()
    for nn in (TABLE1_N if args.table1 else ()):
        xy1 = torch.from_numpy(synth.jittered_grid(nn, seed=1)).to(dev)
        for label, order in TABLE1_ORDERS.items():
            xyo = torch.empty_like(xy1)
            tlr.tlr_order(ctx, xy1, order, xy_out=xyo)
            for c, beta in enumerate(STUDY_BETA):
                theta = (1.0, beta, 0.5)
                ent = {"n": nn, "ordering": label, "beta": beta,
                       "paper_mb": paper.get((nn, label), [None] * 3)[c]}
                M = tlr.TlrMatrix(ctx, nn, 1000)
                try:
                    tiles = tlr.tlr_generate(ctx, xyo, 1000, theta)
                    tlr.tlr_compress(M, tiles, 1e-7 * theta[0])
                    del tiles
                    rk = tlr.tlr_mat_ranks(M)
                    m = [min(1000, nn - t * 1000) for t in range(rk.shape[0])]
                    mb = sum((m[i] + m[j]) * int(rk[i, j]) * 8 for i in range(len(m)) for j in range(i)) / 1e6
                    ent["mb"] = mb
                    if ent["paper_mb"]:
                        ent["ratio_to_paper"] = mb / ent["paper_mb"]
                except tlr.TlrError as e:
                    ent["mb"] = "NA" if e.code == tlr.TLR_ERR_RANK else "error %d" % e.code
                    torch.cuda.synchronize()
                finally:
                    M.close()
                t1.append(ent)
    table_s = time.perf_counter() - t_tab
    out_dir = args.out_dir
    os.makedirs(out_dir, exist_ok=True)
    with open(os.path.join(out_dir, "ordering_study.json"), "w") as f:
        json.dump({"rows": rows, "table1": t1, "rank_maps": rank_maps}, f)
    ok = [r for r in rows if "ms_per_eval" in r]
    line = {"workload": "ordering-study", "n": n, "nb": nb, "orders": orders, "points": len(rows),
            "measured": len(ok), "na": sum(1 for r in rows if r.get("status") == "NA"),
            "study_s": study_s, "table1_s": table_s, "rows_file": os.path.join(out_dir, "ordering_study.json"),
            "rows": [{k: (round(v, 6) if isinstance(v, float) else v) for k, v in r.items()
                      if k in ("order", "nu", "beta", "eps", "ms_per_eval", "max_rank", "mean_rank", "offdiag_mb",
                               "rel_dl_vs_exact", "dl_vs_eps1e-9", "status")} for r in rows],
            "table1": t1}
    print(json.dumps(line), flush=True)
    ctx.close()


# ---- many datasets: batched evaluation (256 datasets) and serving -----------

BATCH_BUCKETS = ((2000, 5000), (5000, 10000), (10000, 20001))
BATCH_TILE_CANDIDATES = (384, 512, 800, 1024)
# rank buckets of the compression (tlr_buckets): the default (latency: large
# clusters for large samples) and a throughput map (half the CTAs per tile)
BUCKETS_DEFAULT = {"qr_edge": [64, 128, 2 ** 31 - 1, 2 ** 31 - 1], "qr_size": [4, 8, 16, 16],
                   "svd_edge": [48, 96, 160, 2 ** 31 - 1], "svd_size": [1, 4, 8, 16]}
BUCKETS_THROUGHPUT = {"qr_edge": [64, 128, 2 ** 31 - 1, 2 ** 31 - 1], "qr_size": [2, 4, 8, 8],
                      "svd_edge": [48, 96, 160, 2 ** 31 - 1], "svd_size": [1, 2, 4, 8]}
# (group size, buckets) candidates of the batched workload's autotuner
BATCH_CANDIDATES = ((1, "default"), (2, "default"), (4, "default"), (8, "default"), (16, "default"),
                    (1, "throughput"), (8, "throughput"))
BUCKET_MAPS = {"default": BUCKETS_DEFAULT, "throughput": BUCKETS_THROUGHPUT}


def batched_datasets(count: int, seed: int = 2024):
    """Sizes n ~ U[2000, 20000] and starting thetas sigma2 ~ U[0.5, 2], beta ~
    U[0.02, 0.3], nu ~ U[0.5, 2.5] of the batched workload (seeded)."""
    import numpy as np
    rng = np.random.default_rng(seed)
    sizes = rng.integers(2000, 20001, count)
    thetas = np.stack([rng.uniform(0.5, 2.0, count), rng.uniform(0.02, 0.3, count),
                       rng.uniform(0.5, 2.5, count)], axis=1)
    return sizes, thetas


def run_batched(args):
    """Batched workload: `--datasets` independent datasets (jittered grids,
    first n points of a ceil(sqrt n)^2 grid, Z = L(theta_i) w_i drawn from each
    dataset's own model with w_i ~ N(0, I) seeded), Morton order,
    eps 1e-7.  Tile size per n bucket picked by the pool's autotuner on one
    dataset of the bucket.  One step = every dataset evaluated once (one
    tlr_pool_loglik call), thetas moving along a per-dataset log-space walk."""
    import numpy as np
    import torch
    import paper_2402_09356_gb300 as tlr
    import synth
    # under torchrun every rank takes the datasets the footprint placement
    # gives it (independent units, no collective on the data path) and the
    # job's throughput is the sum of evaluations over the slowest rank's time
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    all_sizes, all_th0 = batched_datasets(args.datasets)
    place, _ = shard_batched(all_sizes, world, args.maxrank)
    mine = [i for i in range(args.datasets) if place[i] == rank]
    sizes, th0 = all_sizes[mine], all_th0[mine]
    count = len(mine)
    t_setup = time.perf_counter()
    bucket_of = [next(b for b, (lo, hi) in enumerate(BATCH_BUCKETS) if lo <= n < hi) for n in sizes]
    tuned = {}
    tune_pool = tlr.Pool(local, workers=args.workers, nb=512, maxrank=args.maxrank)
    for b, (lo, hi) in enumerate(BATCH_BUCKETS):
        members = [i for i in range(count) if bucket_of[i] == b]
        if not members:
            continue
        if args.batch_nb > 0:  # a fixed tile size instead of the tuner's choice
            tuned[b] = {"best_nb": args.batch_nb, "ms": {}}
            continue
        mid = (lo + hi) / 2
        rep = min(members, key=lambda i: abs(sizes[i] - mid))
        n = int(sizes[rep])
        rid = tlr.tlr_pool_add(tune_pool, synth.jittered_grid(n, seed=10 + mine[rep]),
                               synth.standard_normal(n, seed=5000 + mine[rep]), "morton")
        best, ms = tlr.tlr_pool_tune(tune_pool, rid, tuple(th0[rep]), list(BATCH_TILE_CANDIDATES), eps=EPS,
                                     precision=tlr.TLR_PREC_MIXED)
        tuned[b] = {"n": n, "best_nb": best, "ms": ms}
    tune_pool.close()

    # every dataset's data drawn from its own model, Z = L(theta_i) w_i
    zctx = tlr.Context(local)
    zs, z_white = [], 0
    for i in range(count):
        z, ok = draw_z_lw(tlr, zctx, synth.jittered_grid(int(sizes[i]), seed=10 + mine[i]),
                          synth.standard_normal(int(sizes[i]), seed=5000 + mine[i]), th0[i], "morton", 512)
        zs.append(z)
        z_white += 0 if ok else 1
    zctx.close()

    def new_pool(cfg):
        # every path gets a pool of its own, so that each dataset's rank-map
        # history (the compression's sample sizes) comes from that path alone
        pool = tlr.Pool(local, workers=args.workers, nb=512, maxrank=args.maxrank)
        tlr.tlr_pool_configure(pool, cfg[0], BUCKET_MAPS[cfg[1]])
        ids = [tlr.tlr_pool_add(pool, synth.jittered_grid(int(sizes[i]), seed=10 + mine[i]), zs[i], "morton",
                                nb=tuned[bucket_of[i]]["best_nb"]) for i in range(count)]
        return pool, ids

    # group size and rank buckets: the pool's throughput autotuner on every
    # fourth dataset (mixed path; each candidate evaluates the subset twice)
    pool, ids = new_pool((1, "default"))
    sub_ids = ids[::4]
    best, rates = tlr.tlr_pool_autotune(pool, sub_ids, [tuple(th0[i]) for i in range(0, count, 4)],
                                        [(g, BUCKET_MAPS[b]) for g, b in BATCH_CANDIDATES], eps=EPS,
                                        precision=tlr.TLR_PREC_MIXED, rounds=2)
    pool.close()
    cfg_tuned = BATCH_CANDIDATES[best]
    autotune = {"subset": len(sub_ids), "rounds": 2, "precision": "mixed", "chosen": list(cfg_tuned),
                "evals_per_s": {"group %d, %s buckets" % c: r for c, r in zip(BATCH_CANDIDATES, rates)},
                "buckets": BUCKET_MAPS}
    setup_s = time.perf_counter() - t_setup
    walks = [synth.theta_walk(tuple(th0[i]), args.warmup + args.steps, seed=900 + mine[i], scale=0.05)
             for i in range(count)]
    out = {}
    clocks_all = {}
    # every path with the tuned configuration, and the mixed path once more
    # with the untuned one (group 1, default buckets) for comparison
    paths = (("fp64", tlr.TLR_PREC_FP64, cfg_tuned), ("mixed", tlr.TLR_PREC_MIXED, cfg_tuned),
             ("tensor", tlr.TLR_PREC_TENSOR, cfg_tuned), ("auto", tlr.TLR_PREC_AUTO, cfg_tuned),
             ("mixed_untuned", tlr.TLR_PREC_MIXED, (1, "default")))
    pool_stats = {}
    for name, prec, cfg in paths:
        pool, ids = new_pool(cfg)
        for k in range(args.warmup):
            tlr.tlr_pool_loglik(pool, ids, [tuple(w[k]) for w in walks], eps=EPS, precision=prec)
        clocks = ClockSampler(local)
        torch.cuda.synchronize()
        launches0 = tlr.tlr_launch_count()
        clocks.start()
        times, results, fails, used64, statuses = [], [], 0, 0, []
        for k in range(args.steps):
            t0 = time.perf_counter()
            res, st = tlr.tlr_pool_loglik(pool, ids, [tuple(w[args.warmup + k]) for w in walks], eps=EPS,
                                          precision=prec)
            times.append(time.perf_counter() - t0)
            fails += sum(1 for x in st if x != 0)
            used64 += sum(1 for r, x in zip(res, st) if x == 0 and r["precision_used"] == tlr.TLR_PREC_FP64)
            results.append([(r["loglik"], r["min_pivot2"], r["logdet"]) if x == 0 else None
                            for r, x in zip(res, st)])
            statuses.append([(int(x), int(r["precision_used"]) if x == 0 else None) for r, x in zip(res, st)])
        torch.cuda.synchronize()
        clocks_all[name] = clocks.stop()
        total = sum(times)
        if world > 1:
            torch.distributed.barrier()
        rate, units, total = aggregate_units(count * args.steps, total, world, torch.device("cuda", local))
        out[name] = {"evals_per_s": rate, "s_per_step": total / args.steps,
                     "failed": fails, "fp64_results": used64,
                     "gpu_launches": int(tlr.tlr_launch_count() - launches0), "results": results,
                     "statuses": statuses}
        pool_stats[name] = tlr.tlr_pool_stats(pool)
        pool.close()

    def compare(name):
        rel, pairs, absd, dlogdet = [], [], [], []
        for k, (ra, rb) in enumerate(zip(out[name]["results"], out["fp64"]["results"])):
            for i, (a, b) in enumerate(zip(ra, rb)):
                if a is not None and b is not None:
                    rel.append(abs(a[0] - b[0]) / abs(b[0]))
                    absd.append(abs(a[0] - b[0]))
                    dlogdet.append(abs(a[2] - b[2]) / abs(b[2]))
                    th = walks[i][args.warmup + k]
                    pairs.append((rel[-1], a[1] / th[0], int(sizes[i]), [round(float(v), 4) for v in th]))
        compare.extra[name] = {"abs_dl_max": max(absd, default=None),
                               "abs_dl_median": float(np.median(absd)) if absd else None,
                               "rel_dlogdet_max": max(dlogdet, default=None)}
        return rel, pairs
    compare.extra = {}

    def by_theta_region():
        # failures, AUTO's FP64 redos and the mixed path's worst |dl| / |l|
        # per region of the evaluated theta (range beta, smoothness nu)
        def region(th):
            b = "beta<0.1" if th[1] < 0.1 else ("beta<0.2" if th[1] < 0.2 else "beta>=0.2")
            return b + (", nu<1.5" if th[2] < 1.5 else ", nu>=1.5")
        reg = {}
        for k in range(args.steps):
            for i in range(count):
                th = walks[i][args.warmup + k]
                e = reg.setdefault(region(th), {"evals": 0, "failed": {nm: 0 for nm in ("fp64", "mixed", "tensor",
                                                                                        "auto")},
                                                "auto_fp64_results": 0, "mixed_rel_dl_max": 0.0})
                e["evals"] += 1
                for nm in e["failed"]:
                    e["failed"][nm] += out[nm]["statuses"][k][i][0] != 0
                e["auto_fp64_results"] += out["auto"]["statuses"][k][i][1] == tlr.TLR_PREC_FP64
                a, b = out["mixed"]["results"][k][i], out["fp64"]["results"][k][i]
                if a is not None and b is not None:
                    e["mixed_rel_dl_max"] = max(e["mixed_rel_dl_max"], abs(a[0] - b[0]) / abs(b[0]))
        return dict(sorted(reg.items()))

    theta_regions = by_theta_region()
    rel, pairs = compare("mixed")
    rel_auto, _ = compare("auto")
    rel_tensor, _ = compare("tensor")
    # the tuned and untuned mixed pools compute the same results up to the
    # buckets' rounding (group size alone changes nothing)
    same_untuned = [a == b for ra, rb in zip(out["mixed"]["results"], out["mixed_untuned"]["results"])
                    for a, b in zip(ra, rb)]
    # calibration of the auto rule: worst mixed-vs-FP64 difference among the
    # evaluations whose smallest squared pivot (/ sigma2) is at least t
    calib = {("%g" % t): {"kept": sum(1 for p in pairs if p[1] >= t),
                          "max_rel": max([p[0] for p in pairs if p[1] >= t], default=None)}
             for t in (1e-8, 1e-7, 1e-6, 1e-5, 1e-4, 1e-3)}
    pairs.sort(reverse=True)
    accuracy = {"pairs": len(rel), "within_1e-6": int(sum(1 for r in rel if r <= 1e-6)),
                "median": float(np.median(rel)) if rel else None,
                "worst": [{"rel": r, "min_pivot2": pv, "n": n, "theta": th} for r, pv, n, th in pairs[:6]],
                "by_min_pivot2": calib, **compare.extra["mixed"]}
    accuracy_auto = {"pairs": len(rel_auto), "within_1e-6": int(sum(1 for r in rel_auto if r <= 1e-6)),
                     "max": max(rel_auto) if rel_auto else None, **compare.extra["auto"]}
    accuracy_tensor = {"pairs": len(rel_tensor), "within_1e-6": int(sum(1 for r in rel_tensor if r <= 1e-6)),
                       "max": max(rel_tensor) if rel_tensor else None, **compare.extra["tensor"]}
    st = pool_stats
    # the fastest path whose every evaluated pair is within 1e-6 of the FP64 path
    ok = [nm for nm, r in (("mixed", rel), ("tensor", rel_tensor), ("auto", rel_auto)) if r and max(r) <= 1e-6]
    head = max(ok, key=lambda nm: out[nm]["evals_per_s"]) if ok else "fp64"
    line = {"metric": "batched TLR l(theta) evals/s, %d datasets n~U[2000,20000]" % args.datasets,
            "value": out[head]["evals_per_s"], "unit": "evals/s", "n_gpus": 1, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1000.0 * out[head]["s_per_step"], "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None,
            "dtype": {"fp64": "f64", "tensor": "f64 storage, bf16-slice tensor-core panel products"}.get(
                head, "f64 storage, paired-f32 products"), "data": "synthetic",
            "config": {"workload": "batched: %d datasets, n ~ U[2000, 20000] jittered grids, theta ~ U(sigma2 "
                                   "[0.5,2], beta [0.02,0.3], nu [0.5,2.5]), Z = L(theta) w, Morton, eps %g, "
                                   "%d workers, group %d, %s buckets" % (args.datasets, EPS, args.workers, cfg_tuned[0],
                                                                         cfg_tuned[1]),
                       "z": "Z = L(theta_i) w_i from the library's TLR factor at eps 1e-9 (tile 512); "
                            "%d datasets too ill-conditioned for it kept Z = w" % z_white,
                       "precision": head, "workers": args.workers, "maxrank": args.maxrank,
                       "tile_autotune": {str(BATCH_BUCKETS[b]): v for b, v in tuned.items()},
                       "group_bucket_autotune": autotune,
                       "timing": "host wall clock around each blocking tlr_pool_loglik (all datasets)",
                       "l2": "inputs (all datasets' factors) larger than L2"},
            "fp64_path": {k: v for k, v in out["fp64"].items() if k not in ("results", "statuses")},
            "mixed_path": {k: v for k, v in out["mixed"].items() if k not in ("results", "statuses")},
            "auto_path": {k: v for k, v in out["auto"].items() if k not in ("results", "statuses")},
            "tensor_path": {k: v for k, v in out["tensor"].items() if k not in ("results", "statuses")},
            "mixed_untuned_path": {k: v for k, v in out["mixed_untuned"].items() if k not in ("results", "statuses")},
            "tuned_over_untuned": out["mixed"]["evals_per_s"] / out["mixed_untuned"]["evals_per_s"],
            "mixed_tuned_equal_untuned": "%d of %d results bit for bit" % (sum(same_untuned), len(same_untuned)),
            "rel_dl_mixed_vs_fp64_max": max(rel) if rel else None,
            "mixed_vs_fp64": accuracy,
            "auto_vs_fp64": accuracy_auto,
            "tensor_vs_fp64": accuracy_tensor,
            "by_theta_region": theta_regions,
            "pool": st, "setup_s": setup_s, "clocks": clocks_all[head],
            "gpu_launches": out[head]["gpu_launches"]}
    if world > 1:
        line["config"]["sharding"] = {"ranks": world, "datasets_per_rank": [int((place == r).sum())
                                                                             for r in range(world)],
                                      "placement": "largest footprint first onto the least-loaded rank",
                                      "accuracy_and_autotune": "rank 0's datasets"}
        line["n_gpus"] = world
        line["scaling"] = "strong"
        torch.distributed.barrier()
        torch.distributed.destroy_process_group()
    if rank == 0:
        print(json.dumps(line), flush=True)


SERVE_SIZES = (5000, 10000, 20000, 40000, 80000)


def run_serving(args):
    """Serving workload: 32 resident datasets with n cycling through 5k, 10k,
    20k, 40k, 80k (jittered grids, Z = L w drawn from the model at the walk's
    start theta = (1, 0.1, 1.0), w ~ N(0, I) seeded, Hilbert order, tile
    800), a Poisson stream of `--requests` l(theta) requests at `--rate` per
    second on uniformly drawn datasets, theta following each dataset's own
    simplex-like walk in log(sigma2, beta, nu) around (1, 0.1, 1.0), and two
    MLE jobs (n = 5k and 10k) submitted beside the stream.  Latency = host
    time from submission to completion."""
    import threading
    import numpy as np
    import torch
    import paper_2402_09356_gb300 as tlr
    import synth
    nd = 32
    sizes = [SERVE_SIZES[i % len(SERVE_SIZES)] for i in range(nd)]
    pool = tlr.Pool(0, workers=args.workers, nb=NB, maxrank=args.maxrank)
    tlr.tlr_pool_configure(pool, args.group)
    t_setup = time.perf_counter()
    zctx = tlr.Context(0)
    zs = [draw_z_lw(tlr, zctx, synth.jittered_grid(n, seed=300 + i), synth.standard_normal(n, seed=600 + i),
                    (1.0, 0.1, 1.0), "hilbert", NB) for i, n in enumerate(sizes)]
    zctx.close()
    z_white = sum(1 for _, ok in zs if not ok)
    ids = [tlr.tlr_pool_add(pool, synth.jittered_grid(n, seed=300 + i), zs[i][0], "hilbert")
           for i, n in enumerate(sizes)]
    setup_s = time.perf_counter() - t_setup
    rng = np.random.default_rng(77)
    R = args.requests
    arrivals = np.cumsum(rng.exponential(1.0 / args.rate, R))
    targets = rng.integers(0, nd, R)
    steps_of = [0] * nd
    per_data = np.bincount(targets, minlength=nd)
    walks = [synth.theta_walk((1.0, 0.1, 1.0), int(per_data[d]) + 1, seed=1200 + d, scale=0.15) for d in range(nd)]
    mle_ids = [ids[0], ids[1]]
    out = {}
    for name, prec in (("fp64", tlr.TLR_PREC_FP64), ("mixed", tlr.TLR_PREC_MIXED)):
        # warm-up: one request per dataset size
        for i in range(len(SERVE_SIZES)):
            tlr.tlr_pool_wait(pool, tlr.tlr_pool_submit(pool, ids[i], (1.0, 0.1, 1.0), EPS, prec))
        steps_of = [0] * nd
        tickets = [None] * R
        mle_out = {}

        def mle(j, did):
            t0 = time.perf_counter()
            th, ll, it = tlr.tlr_pool_mle(pool, did, (0.8, 0.08, 1.2), (0.05, 0.005, 0.2), (5.0, 1.0, 3.0),
                                          eps=EPS, precision=prec, tol=1e-6, max_iter=args.mle_iters)
            mle_out[j] = {"n": sizes[mle_ids.index(did)], "theta": th, "loglik": ll, "evals": it,
                          "wall_s": time.perf_counter() - t0}

        clocks = ClockSampler(0)
        torch.cuda.synchronize()
        launches0 = tlr.tlr_launch_count()
        clocks.start()
        t_start = time.perf_counter()
        mle_threads = [threading.Thread(target=mle, args=(j, d)) for j, d in enumerate(mle_ids)]
        for t in mle_threads:
            t.start()
        for q in range(R):
            delay = t_start + arrivals[q] - time.perf_counter()
            if delay > 0:
                time.sleep(delay)
            d = int(targets[q])
            th = tuple(walks[d][steps_of[d]])
            steps_of[d] += 1
            tickets[q] = tlr.tlr_pool_submit(pool, ids[d], th, EPS, prec)
        lat, queue, run, fails = [], [], [], 0
        lls = [None] * R
        by_n = {n: [] for n in SERVE_SIZES}
        for q in range(R):
            try:
                res, tm = tlr.tlr_pool_wait(pool, tickets[q])
            except tlr.TlrError:
                fails += 1
                continue
            lls[q] = res["loglik"]
            lat.append(tm["latency_ms"])
            queue.append(tm["queue_ms"])
            run.append(tm["run_ms"])
            by_n[sizes[int(targets[q])]].append(tm["latency_ms"])
        t_stream = time.perf_counter() - t_start
        for t in mle_threads:
            t.join()
        t_all = time.perf_counter() - t_start
        torch.cuda.synchronize()
        clk = clocks.stop()
        mle_evals = sum(v["evals"] for v in mle_out.values())
        pct = lambda a, p: float(np.percentile(a, p)) if a else None
        out[name] = {"evals_per_s": (R - fails + mle_evals) / t_all, "stream_evals_per_s": (R - fails) / t_stream,
                     "p50_ms": pct(lat, 50), "p99_ms": pct(lat, 99), "queue_p50_ms": pct(queue, 50),
                     "run_p50_ms": pct(run, 50), "failed": fails, "wall_s": t_all,
                     "by_n": {str(n): {"count": len(v), "p50_ms": pct(v, 50), "p99_ms": pct(v, 99)}
                              for n, v in by_n.items()},
                     "mle": mle_out, "clocks": clk, "gpu_launches": int(tlr.tlr_launch_count() - launches0),
                     "pool": tlr.tlr_pool_stats(pool), "lls": lls}
    rel = [abs(a - b) / abs(b) for a, b in zip(out["mixed"]["lls"], out["fp64"]["lls"]) if a is not None and b is not None]
    for name in out:
        out[name].pop("lls")
    line = {"metric": "served TLR l(theta) evals/s and p50/p99 latency, 32 resident datasets",
            "value": out["mixed"]["evals_per_s"], "unit": "evals/s", "n_gpus": 1, "steps": R, "warmup": 5,
            "ms_per_step": 1000.0 / out["mixed"]["evals_per_s"], "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64 storage, paired-f32 products", "data": "synthetic",
            "p50_ms": out["mixed"]["p50_ms"], "p99_ms": out["mixed"]["p99_ms"],
            "config": {"workload": "serving: 32 resident datasets n in {5k,10k,20k,40k,80k}, nu=1.0 walk start, "
                                   "Hilbert, tile %d, eps %g, Poisson %g req/s x %d requests + 2 MLE jobs, "
                                   "%d workers" % (NB, EPS, args.rate, R, args.workers),
                       "workers": args.workers, "group": args.group, "maxrank": args.maxrank, "rate": args.rate,
                       "requests": R,
                       "latency": "host clock, submission to completion",
                       "z": "Z = L(1, 0.1, 1.0) w from the library's TLR factor at eps 1e-9; %d kept Z = w"
                            % z_white},
            "fp64_path": out["fp64"], "mixed_path": out["mixed"], "setup_s": setup_s,
            "mixed_vs_fp64": {"pairs": len(rel), "max": max(rel) if rel else None,
                              "within_1e-6": int(sum(1 for r in rel if r <= 1e-6))},
            "clocks": out["mixed"]["clocks"], "gpu_launches": out["mixed"]["gpu_launches"]}
    print(json.dumps(line), flush=True)
    pool.close()


def main():
    global N_POINTS, NB, EPS, ORDER, THETA0
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--latency-evals", type=int, default=100,
                    help="evaluations of the separate latency loop (p50/p99); 0 = use the timed steps")
    ap.add_argument("--n", type=int, default=N_POINTS, help="locations (profiling of smaller cases)")
    ap.add_argument("--nb", type=int, default=NB)
    ap.add_argument("--eps", type=float, default=EPS)
    ap.add_argument("--order", default=ORDER)
    ap.add_argument("--theta", default=None, help="walk start sigma2,beta,nu (default 1,0.1,0.5)")
    ap.add_argument("--paths", default="all", choices=["all", "both", "mixed", "fp64", "tensor"],
                    help="precision paths to time (all for the headline; one for profiling runs)")
    ap.add_argument("--study-steps", type=int, default=2, help="timed evaluations per ordering-study point")
    ap.add_argument("--study-orders", default="", help="comma-separated orderings of the study (default: all five)")
    ap.add_argument("--no-table1", dest="table1", action="store_false", help="skip the Table 1 memory comparison")
    ap.add_argument("--out-dir", default=os.path.join(ROOT, "study_out"), help="where the study writes its tables")
    ap.add_argument("--workload", default="headline",
                    choices=["headline", "batched", "serving", "ordering-study", "oracle-fullsize"],
                    help="headline: one n = 40,000 evaluation per step; batched: many datasets per step; "
                         "serving: a Poisson request stream over resident datasets")
    ap.add_argument("--workers", type=int, default=8, help="pool workers (batched / serving)")
    ap.add_argument("--group", type=int, default=1, help="serving: requests a worker evaluates together")
    ap.add_argument("--datasets", type=int, default=256, help="datasets of the batched workload")
    ap.add_argument("--batch-nb", type=int, default=0, help="fixed tile size for the batched workload (0: tuned)")
    ap.add_argument("--maxrank", type=int, default=0, help="rank slots per tile (batched / serving; 0 = nb/2)")
    ap.add_argument("--qr-sizes", default="", help="headline: cluster sizes of the QR rank buckets, e.g. 4,8,16,16")
    ap.add_argument("--svd-sizes", default="", help="headline: cluster sizes of the SVD rank buckets, e.g. 1,4,8,16")
    ap.add_argument("--requests", type=int, default=96, help="requests of the serving stream")
    ap.add_argument("--rate", type=float, default=500.0, help="arrival rate of the serving stream (1/s)")
    ap.add_argument("--mle-iters", type=int, default=30, help="evaluations per MLE job (serving)")
    args = ap.parse_args()
    N_POINTS, NB, EPS, ORDER = args.n, args.nb, args.eps, args.order
    if args.theta:
        THETA0 = tuple(float(v) for v in args.theta.split(","))
    if args.impl == "reference":
        run_reference(args)
        return
    if args.workload == "oracle-fullsize":
        run_oracle_fullsize(args)
        return
    from paper_2402_09356_gb300 import build as lib_build
    lib_build.build()
    if args.workload == "batched":
        run_batched(args)
    elif args.workload == "serving":
        run_serving(args)
    elif args.workload == "ordering-study":
        run_ordering_study(args)
    else:
        run_gpu(args)


if __name__ == "__main__":
    main()
