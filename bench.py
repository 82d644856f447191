#!/usr/bin/env python3
"""Benchmark of the Zeus hot path on one GB300 (or N, one process per GPU).

The default step is the batched form on its full workload: 4096
independent problems (d log-uniform in [2, 128]; Rosenbrock chain,
Rastrigin and Ackley mixed; 256 particles each, 10 PSO updates, BFGS cap
500, ||g|| < 1e-8), FP64, solved by one CUDA-graph replay of
zeus_batch_solve per step (PSO, BFGS from every particle, best-of-swarm
reduction of every problem).  The metric is start-iterations per second
(sum over starts of completed BFGS iterations divided by device time).
Prints one JSON line.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl zeus|reference]
                  [--workload mixed4096_n256|rastrigin10d_n16384|rosenbrock256d_n8192|...]

At one GPU the default line also carries, each measured here with its own
roofline: the single-problem workloads (10-D Rastrigin, the d = 256
Rosenbrock chain in FP32 with FP64 guards and in FP64, the d = 1024
Rosenbrock chain and Ackley with the adjoint and the forward-mode
gradient) under "extras"; the forms' time to 1e-6 of the global minimum at
their success rates over 20 seeds, whole batch included, under "forms";
the FP32 form's per-start error against the FP64 method under
"fp32_error"; the early-stop study's PSO-update sweep under "study"; the
clustering of the final points; and the oracle on all host cores and on
one core.  --workload <single problem> makes that workload the timed step;
--study runs the whole early-stop study instead.

--impl reference times the FP64 CPU oracle (the only reference: the paper
ships no code) on the host cores for the same workload, a bounded sample of
starts or problems per step.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_2603_28770_gb300 import workloads  # noqa: E402

BATCH_WORKLOAD = "mixed4096_n256"
DEFAULT_WORKLOAD = BATCH_WORKLOAD
METRIC = "start-iters/s"


def _args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="zeus", choices=["zeus", "reference"])
    ap.add_argument("--workload", default=DEFAULT_WORKLOAD)
    ap.add_argument("--grad-mode", default="forward", choices=["forward", "adjoint"])
    ap.add_argument("--lanes", type=int, default=0, help="threads per start (0 = automatic)")
    ap.add_argument("--layout", type=int, default=-1,
                    help="batched workload: threads per start of every problem instead of the "
                         "autotuner's choice (profiling cases)")
    ap.add_argument("--precision", default="fp64", choices=["fp64", "fp32_guarded"])
    ap.add_argument("--study", action="store_true",
                    help="the early-stop study instead of the benchmark: PSO updates vs time and "
                         "correct solutions (5-D Rastrigin, Rosenbrock), correct solutions vs d")
    ap.add_argument("--study-runs", type=int, default=10)
    ap.add_argument("--lbfgs-m", type=int, default=0,
                    help="L-BFGS with this many pairs instead of the dense inverse Hessian")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extras", action="store_true",
                    help="only the main line (no extras, forms, error, study, clustering)")
    ap.add_argument("--form-seeds", type=int, default=20)
    ap.add_argument("--e2e-steps", type=int, default=3,
                    help="end-to-end repetitions (host buffers, copies in the timed region)")
    ap.add_argument("--starts", type=int, default=0,
                    help="override the workload's number of starts (smaller profiling cases)")
    ap.add_argument("--problems", type=int, default=0,
                    help="batched workload: only its first N problems (smaller profiling cases)")
    ap.add_argument("--iters", type=int, default=0,
                    help="override the workload's BFGS iteration cap (smaller profiling cases)")
    return ap.parse_args()


# ----------------------------------------------------------------- clocks

class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons during a region."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "20"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except OSError:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self) -> dict:
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                mx.append(float(parts[1]))
            except ValueError:
                continue
            for name, val in zip(names, parts[4:8]):
                if val.lower() == "active":
                    reasons.add(name)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# --------------------------------------------------------- roofline model
#
# Algorithmic FP64 operations, counted from the operations the method needs
# as implemented (FMA = 2, every other FP64 add, multiply, rounding or
# conversion = 1, division and square root = 1):
#   sin(2 pi x) and cos(2 pi x) together: argument reduction 7, two Horner
#     chains of 8 FMA each 32, final product 1 -> 40; cos(2 pi x) alone: one
#     chain -> 26; e^x: reduction 6, 13 FMA 26 -> 32.
#   gradient (Alg. 5, one dual pass per coordinate; the passes skip the
#   terms whose tangent is an exact zero where the tangent does not depend
#   on the sums):
#     Rastrigin  per coordinate sin/cos 40 + tangent 4              ->  44 d
#     Rosenbrock per coordinate two dual terms of 18                 ->  36 d
#     Ackley     per pass the two sums over all d terms (x^2 1, cos 26,
#                two adds) 29 d, the sine of x_i 40, the exponentials,
#                divisions, square root and tangents of the finish 88 -> d (29 d + 128)
#     quadratic  per coordinate 5                                     ->   5 d
#   adjoint (one forward and one reverse sweep): Rastrigin 44 d, Rosenbrock
#     10 d, Ackley the two sums 29 d + 75 and per coordinate sin/cos and 5
#     -> 74 d + 75, quadratic 5 d
#   value at a trial point (trial coordinates x + a p included):
#     Rastrigin 32 d + 2, Rosenbrock 12 d, Ackley 31 d + 75, quadratic 7 d
#   user objectives: Griewank d passes x d coordinates x (dual square 4,
#     sum 2, scaled argument 2, dual cosine 42, product 4) and a value sweep
#     of 28 d; Himmelblau 2 passes x 20 and 14.

def objective_flops(objective, d: int, grad_mode: str = "forward"):
    """(gradient, value at a trial point) FP64 operations, model above."""
    if objective == "griewank":
        return 54.0 * d * d, 28.0 * d
    if objective == "himmelblau":
        return 40.0, 14.0
    adj = grad_mode == "adjoint"
    if objective == "ackley":
        return (74.0 * d + 75.0 if adj else d * (29.0 * d + 128.0)), 31.0 * d + 75.0
    if objective == "rosenbrock":
        return (10.0 * d if adj else 36.0 * d), 12.0 * d
    if objective == "quadratic":
        return 5.0 * d, 7.0 * d
    return 44.0 * d, 32.0 * d + 2.0  # rastrigin


def fp64_flops(d: int, iters: int, fevals: int, objective="rastrigin", grad_mode="forward") -> float:
    """Algorithmic FP64 operations of a BFGS phase:
      per start-iteration  the gradient (objective_flops),
                           ||g|| 2d + 1, p = -H g 2d^2 + d, g'p 2d, x_new 2d,
                           s, y, y's, |s|^2, |y|^2 8d, curvature test 5,
                           H y 2d^2, y'Hy 2d, rho and its factor 4,
                           rank-two update: two FMAs (4) per element of
                           the upper triangle of the symmetric H, d(d+1)/2
                           -> 6 d^2 + 23 d + 10 + gradient
      per line-search evaluation  the value at the trial point + Armijo test 3"""
    grad, val = objective_flops(objective, d, grad_mode)
    return iters * (6.0 * d * d + 23.0 * d + 10.0 + grad) + fevals * (val + 3.0)


FP64_PEAK_TFLOPS = 1.25  # FP64 FMA throughput measured on GB300 (= nominal)
FP32_PEAK_TFLOPS = 80.5  # nominal: 152 SMs x 128 lanes x 2 x 2.07 GHz


def _peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        return json.load(open(path))
    except OSError:
        return {}


def hbm_peak():
    """(GB/s, source) of the HBM roofline."""
    p = _peaks()
    for k in ("hbm_gbs", "hbm_copy_gbs"):
        if k in p:
            return float(p[k]), "measured HBM copy bandwidth (MEASURED_PEAKS.json)"
    return 6794.1, "HBM copy bandwidth measured on this pool's GB300 (6794.1 GB/s)"


def aggregate(total_ms: float, iters: int, world: int, device=None):
    """Whole-job figures over the ranks of the process group: the slowest
    rank's timed milliseconds and the sum of the ranks' start-iterations
    (weak scaling: every rank solves its own independent problem)."""
    if world <= 1:
        return float(total_ms), float(iters)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(total_ms)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    n = torch.tensor([float(iters)], dtype=torch.float64, device=device)
    dist.all_reduce(n, op=dist.ReduceOp.SUM)
    return float(t.item()), float(n.item())


def rank_seed(seed: int, rank: int, stride: int = 1) -> int:
    """Seed of rank `rank`'s independent problem (rank 0 keeps the base seed)."""
    return int(seed) + stride * int(rank)


def clopper_pearson(k: int, n: int, level: float = 0.95):
    """Exact two-sided binomial interval for k successes in n trials."""
    from scipy.stats import beta
    a = (1.0 - level) / 2.0
    lo = 0.0 if k == 0 else float(beta.ppf(a, k, n - k + 1))
    hi = 1.0 if k == n else float(beta.ppf(1.0 - a, k + 1, n - k))
    return [round(lo, 4), round(hi, 4)]


# ------------------------------------------------------ single problem

def _problem(z, fields):
    return z.Problem(**{k: v for k, v in fields.items() if k in z.Problem.__dataclass_fields__})


# DRAM traffic of the streamed-H kernel per algorithmic byte of its H
# passes, from one ncu capture (dram__bytes_read.sum + dram__bytes_write.sum
# over the launch) of the current build on a small case of each workload:
# Rosenbrock chain d = 256 FP32, forward, 8192 starts, K = 50: 102.90 GB for
# 104.56 GB of triangle passes (the 86 MB of tiles partly stay in L2);
# d = 1024 FP32, adjoint, 608 starts, K = 40: 100.69 GB for 97.47 GB (the
# tiles on the diagonal carry their lower elements too).  Traffic grows
# with the passes, so a full launch's traffic is its algorithmic bytes
# times the ratio.  Keyed by (objective, d, precision, gradient mode);
# other cases report null.
STREAM_TRAFFIC_RATIO = {("rosenbrock", 256, "fp32_guarded", "forward"): 102.90 / 104.56,
                        ("rosenbrock", 1024, "fp32_guarded", "adjoint"): 100.69 / 97.47}


def single_roofline(z, pc, d, iters, fevals, summary, bfgs_s, fields, lbfgs_m, precision):
    """Roofline of the BFGS phase (the dominant launch sequence), timed by the
    events around zeus_solve_from on its stream."""
    plan = z.zeus_plan_info(pc)
    grad_mode = fields.get("grad_mode", "forward")
    if plan["lbfgs"]:
        # L-BFGS: per start-iteration the two loops over the m pairs (a dot
        # product and an update of length d each, FMA = 2: 8 m d) plus the
        # O(d) work of the dense model's linear terms; no H traffic
        m = lbfgs_m
        flops = iters * (8.0 * m * d + 65.0 * d + 10.0) + fevals * (30.0 * d + 3.0)
        f32 = precision == "fp32_guarded"
        peak = FP32_PEAK_TFLOPS if f32 else FP64_PEAK_TFLOPS
        achieved = flops / bfgs_s / 1e12
        return {"kernel": "bfgs_stream_kernel, L-BFGS variant (+ argmin)", "bound": "alu",
                "achieved": round(achieved, 5), "peak": peak, "unit": "TFLOP/s",
                "frac": round(achieved / peak, 5), "traffic": None,
                "peak_source": ("FP32: nominal 152 SMs x 128 lanes x 2 x 2.07 GHz" if f32
                                else "FP64 FMA rate measured on this GB300"),
                "flops_per_launch": flops, "launch_ms": round(bfgs_s * 1e3, 3)}
    if plan["stream"]:
        # H streamed from HBM, per pass that read or wrote it (the kernel
        # counts them; at most 2 per start-iteration, none while H = I): FP64
        # H moves the full matrix, d^2 x 8 bytes; FP32 H is held as the tiles
        # of its upper triangle, and its algorithmic bytes are the
        # triangle's, d (d + 1) / 2 x 4 (the tiles on the diagonal carry a
        # few more: plan h_bytes)
        reads, writes = summary["h_reads"], summary["h_writes"]
        b = 4 if precision == "fp32_guarded" else 8
        tiled = b == 4 and plan["h_bytes"] < d * d * 4  # past d ~ 3200 FP32 H streams whole
        per_pass = d * (d + 1) // 2 * 4 if tiled else d * d * b
        nbytes = float(per_pass) * (reads + writes)
        achieved = nbytes / bfgs_s / 1e9
        peak, src = hbm_peak()
        ratio = STREAM_TRAFFIC_RATIO.get((fields["objective"], d, precision, grad_mode))
        roof = {"kernel": "bfgs_stream_kernel (+ argmin)", "bound": "hbm",
                "achieved": round(achieved, 1), "peak": peak, "unit": "GB/s",
                "frac": round(achieved / peak, 4),
                "traffic": round(nbytes * ratio) if ratio else None, "peak_source": src,
                "bytes_per_launch": nbytes, "launch_ms": round(bfgs_s * 1e3, 3),
                "h_passes": {"reads": reads, "writes": writes, "bytes_per_pass": per_pass,
                             "stored_bytes_per_pass": plan["h_bytes"]}}
        if precision == "fp64":
            # FP64 H: every pass takes d^2 FMAs for H g and 2 d^2 more when
            # it applies an update; against the FP64 pipe this is the bound
            pass_flops = 2.0 * d * d * max(reads, writes) + 4.0 * d * d * writes
            tf = pass_flops / bfgs_s / 1e12
            if tf / FP64_PEAK_TFLOPS > roof["frac"]:
                roof = dict(roof, bound="alu", achieved=round(tf, 4), peak=FP64_PEAK_TFLOPS,
                            unit="TFLOP/s", frac=round(tf / FP64_PEAK_TFLOPS, 4),
                            peak_source="FP64 FMA rate measured on this GB300",
                            flops_per_launch=pass_flops,
                            hbm={"achieved_gbs": round(achieved, 1), "frac": round(achieved / peak, 4)})
        return roof
    flops = fp64_flops(d, iters, fevals, fields["objective"], grad_mode)
    achieved = flops / bfgs_s / 1e12
    kname = ("bfgs_fused_kernel (lane tiles and hand-over service in one cooperative launch)"
             if plan["handover"] else ("bfgs_narrow_kernel" if plan["narrow"] else "bfgs_wide_kernel"))
    return {"kernel": kname + " (+ argmin)", "bound": "alu", "achieved": round(achieved, 5),
            "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s", "frac": round(achieved / FP64_PEAK_TFLOPS, 5),
            "traffic": None,
            "peak_source": "FP64 FMA rate measured on this GB300 (1.25 TFLOP/s, equal to the "
                           "part's nominal FP64 rate)",
            "flops_per_launch": flops, "launch_ms": round(bfgs_s * 1e3, 3)}


def measure_single(z, dev, fields, steps, warmup, world=1, rank=0, e2e_steps=3, lbfgs_m=0):
    """One step = the whole path on one problem: zeus_pso (PSO phase) then
    zeus_solve_from (BFGS from the final positions, argmin), inputs resident
    on the device, L2 flushed between steps outside the events.  Returns
    the measured figures (whole-job over the ranks) and the objects the
    caller may reuse."""
    import torch
    p = _problem(z, fields)
    pc = p.to_c()
    n, d = p.n_starts, p.dim
    ws = z.new_workspace(pc, dev)
    x = torch.empty(n, d, dtype=torch.float64, device=dev)
    f = torch.empty(n, dtype=torch.float64, device=dev)
    gn = torch.empty(n, dtype=torch.float64, device=dev)
    st = torch.empty(n, dtype=torch.int32, device=dev)
    it = torch.empty(n, dtype=torch.int32, device=dev)
    v = torch.empty(n, d, dtype=torch.float64, device=dev)
    px = torch.empty(n, d, dtype=torch.float64, device=dev)
    pf = torch.empty(n, dtype=torch.float64, device=dev)
    gx = torch.empty(d, dtype=torch.float64, device=dev)
    res = z.new_result(dev)
    ws_pso = z.new_workspace(pc, dev)
    flush = torch.empty(256 * 1024 * 1024, dtype=torch.uint8, device=dev)  # > 129 MB L2
    stream = torch.cuda.current_stream(dev)

    def step(ev=None):
        if ev:
            ev[0].record(stream)
        z.zeus_pso(pc, ws_pso, x, v, px, pf, gx, None, stream)
        if ev:
            ev[1].record(stream)
        z.zeus_solve_from(pc, x, ws, x, f, gn, st, it, res, stream)
        if ev:
            ev[2].record(stream)

    for _ in range(warmup):
        step()
    torch.cuda.synchronize(dev)
    summary = z.decode_result(res)
    iters_per_step = int(summary["total_iters"])
    feval_per_step = int(summary["total_feval"])
    events = [[torch.cuda.Event(enable_timing=True) for _ in range(3)] for _ in range(steps)]
    if world > 1:
        import torch.distributed as dist
        dist.barrier()
    torch.cuda.synchronize(dev)
    t_wall = time.perf_counter()
    with ClockSampler(dev.index or 0) as clk:
        for k in range(steps):
            flush.fill_(k & 0xFF)  # evict L2 between timed steps (outside the events)
            step(events[k])
        torch.cuda.synchronize(dev)
    t_wall = time.perf_counter() - t_wall
    if world > 1:
        dist.barrier()
    step_ms = [e[0].elapsed_time(e[2]) for e in events]
    bfgs_ms = [e[1].elapsed_time(e[2]) for e in events]
    summary = z.decode_result(res)
    assert int(summary["total_iters"]) == iters_per_step, "non-deterministic iteration count"
    total_ms, iters_all = aggregate(sum(step_ms), iters_per_step, world, dev)
    value = iters_all * steps / (total_ms / 1e3)

    # end to end through the host-buffer C entry point: the problem struct
    # in, every per-start output copied back to pinned host memory
    ctx = z.Context()
    hx = torch.empty(n, d, dtype=torch.float64).pin_memory()
    hf = torch.empty(n, dtype=torch.float64).pin_memory()
    hg = torch.empty(n, dtype=torch.float64).pin_memory()
    hs = torch.empty(n, dtype=torch.int32).pin_memory()
    hi = torch.empty(n, dtype=torch.int32).pin_memory()
    ctx.zeus_solve_host(pc, hx, hf, hg, hs, hi, stream)  # warm-up (allocates)
    e2e_ms = []
    for k in range(max(1, e2e_steps)):
        flush.fill_(k & 0xFF)
        torch.cuda.synchronize(dev)
        t0 = time.perf_counter()
        r = ctx.zeus_solve_host(pc, hx, hf, hg, hs, hi, stream)  # synchronizes the stream
        e2e_ms.append((time.perf_counter() - t0) * 1e3)
    ctx.close()
    assert int(r["total_iters"]) == iters_per_step
    e2e_value = iters_per_step * len(e2e_ms) / (sum(e2e_ms) / 1e3)
    d2h = n * d * 8 + n * 8 * 2 + n * 4 * 2 + 128

    bfgs_s = statistics.mean(bfgs_ms) / 1e3
    roof = single_roofline(z, pc, d, iters_per_step, feval_per_step, summary, bfgs_s, fields,
                           lbfgs_m, fields.get("precision", "fp64"))
    out = {"value": round(value, 1), "unit": METRIC, "ms_per_step": round(total_ms / steps, 3),
           "steps": steps, "warmup": warmup,
           "config": {"objective": p.objective, "dim": d, "n_starts": n, "pso_iters": p.pso_iters,
                      "bfgs_max_iters": p.bfgs_max_iters, "grad_mode": p.grad_mode,
                      "precision": p.precision, "lbfgs_m": lbfgs_m,
                      "start_iters_per_step": iters_per_step, "feval_per_step": feval_per_step},
           "e2e": {"value": round(e2e_value, 1), "unit": METRIC, "h2d_bytes_per_step": 128,
                   "d2h_bytes_per_step": d2h,
                   "api": "zeus_solve_host (problem struct in, host outputs back, stream synchronized)"},
           "gpu_launches": steps * (p.pso_iters + 3),
           "roofline": roof, "best_f": summary["best_f"], "n_converged": summary["n_converged"],
           "status_counts": {str(k): int(c) for k, c in
                             zip(*np.unique(st.cpu().numpy(), return_counts=True))},
           "wall_s_timed": round(t_wall, 3), "clocks": clk.summary()}
    return out, dict(x=x, f=f, st=st, stream=stream, n=n, d=d)


def cluster_figures(z, dev, keep) -> dict:
    """Solution clustering of a step's final points (Section VI proposes
    it), timed apart from the step: converged starts by coordinates, tol
    1e-4, the first 256 regions."""
    import torch
    n, d, x, f, st, stream = keep["n"], keep["d"], keep["x"], keep["f"], keep["st"], keep["stream"]
    cp = z._capi.zeus_cluster_params(1, 256, 1, 0, 1e-4)
    lab = torch.empty(n, dtype=torch.int32, device=dev)
    lead = torch.empty(256, dtype=torch.int32, device=dev)
    cnt = torch.empty(256, dtype=torch.int32, device=dev)
    cres = torch.empty(64, dtype=torch.uint8, device=dev)
    cws = torch.empty(z.zeus_cluster_workspace_size(256), dtype=torch.uint8, device=dev)
    for _ in range(3):
        z.zeus_cluster(cp, n, d, x, f, st, lab, lead, cnt, cres, cws, stream)
    c0, c1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    c0.record(stream)
    for _ in range(5):
        z.zeus_cluster(cp, n, d, x, f, st, lab, lead, cnt, cres, cws, stream)
    c1.record(stream)
    torch.cuda.synchronize(dev)
    cs = z._capi.zeus_cluster_result.from_buffer_copy(bytes(cres.cpu().numpy().tobytes()))
    return {"kernel": "cluster_kernel (cooperative grid, one barrier per region)",
            "method": "x", "tol": 1e-4, "max_clusters": 256, "only_converged": True,
            "ms": round(c0.elapsed_time(c1) / 5, 4), "n_candidates": cs.n_candidates,
            "n_clusters": cs.n_clusters, "n_left": cs.n_left, "best_count": cs.best_count,
            "best_f": cs.best_f}


def single_fields(a, name=None, **over):
    fields = workloads.workload(name or a.workload, grad_mode=a.grad_mode,
                                threads_per_start=a.lanes, precision=a.precision)
    if a.lbfgs_m:
        fields["lbfgs_m"] = a.lbfgs_m
    if a.starts:
        fields["n_starts"] = a.starts
    if a.iters:
        fields["bfgs_max_iters"] = a.iters
    fields.update(over)
    return fields


def run_single_main(a, z, dev, world, rank):
    """--workload <single problem>: that workload is the timed step."""
    fields = single_fields(a)
    # weak scaling: every rank solves its own independent multistart problem
    fields["seed"] = rank_seed(fields["seed"], rank)
    line, keep = measure_single(z, dev, fields, a.steps, a.warmup, world, rank, a.e2e_steps,
                                a.lbfgs_m)
    cfg = dict(line["config"], workload=a.workload,
               l2="flushed between timed steps (256 MB write outside the events)",
               parallelism=f"replicas x{world}")
    out = {"metric": METRIC, "value": line["value"], "unit": METRIC, "n_gpus": world,
           "steps": a.steps, "warmup": a.warmup, "ms_per_step": line["ms_per_step"],
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
           "dtype": "f32" if a.precision == "fp32_guarded" else "f64",
           "data": "synthetic (seeded Philox draws of the method itself; no dataset)",
           "config": cfg}
    for k in ("e2e", "gpu_launches", "roofline", "best_f", "n_converged", "status_counts",
              "wall_s_timed", "clocks"):
        out[k] = line[k]
    if rank == 0 and world == 1 and not a.lbfgs_m and not a.no_extras:
        out["cluster"] = cluster_figures(z, dev, keep)
    if rank == 0 and not a.no_cpu_baseline:
        out["cpu_baseline"] = cpu_baseline(fields, budget_s=12.0)
    if rank == 0:
        print(json.dumps(out), flush=True)


# ------------------------------------------------------------ batched form

def _tuner():
    """The layout autotuner with its cache in the user's cache directory."""
    from paper_2603_28770_gb300.autotune import Autotuner
    return Autotuner()


def _tuned_summary(b) -> dict:
    counts = {}
    for p in b.problems:
        counts[str(int(p.threads_per_start))] = counts.get(str(int(p.threads_per_start)), 0) + 1
    return {"threads_per_start_counts": counts}


def _obj_name(p):
    o = p.objective
    if isinstance(o, str):
        return o
    names = {0: "rosenbrock", 1: "rastrigin", 2: "ackley", 3: "goldstein_price", 100: "quadratic"}
    return names.get(int(o), "user")


def batch_flops(b) -> float:
    """FP64-model operations of one batched solve (per-problem counters)."""
    gm = {0: "forward", 1: "adjoint"}
    return float(sum(fp64_flops(p.dim, s["total_iters"], s["total_feval"], _obj_name(p),
                                gm.get(int(p.grad_mode), p.grad_mode) if not isinstance(p.grad_mode, str)
                                else p.grad_mode)
                     for p, s in zip(b.problems, b.summaries())))


def batch_fields(a, n_problems=None, **over):
    return workloads.batch_problems(BATCH_WORKLOAD, n_problems, precision=a.precision,
                                    grad_mode=a.grad_mode, **over)


def run_batch_main(a, z, dev, world, rank):
    """Default step: one solve of the whole batch (4096 problems, 2^20
    starts), replayed from a CUDA graph."""
    import torch
    fields = batch_fields(a, a.problems or None)
    # weak scaling: each rank solves its own batch (seeds shifted by rank);
    # threads per start chosen by the autotuner (measured once, then cached)
    t0 = time.perf_counter()
    if a.layout >= 0:
        fields = [dict(f, threads_per_start=a.layout) for f in fields]
    b = z.Batch([z.Problem(**dict(f, seed=rank_seed(f["seed"], rank, 4096))) for f in fields],
                device=dev, autotuner=None if a.layout >= 0 else _tuner())
    tune_s = time.perf_counter() - t0
    flush = torch.empty(256 * 1024 * 1024, dtype=torch.uint8, device=dev)
    b.solve()
    torch.cuda.synchronize(dev)
    b.capture()
    for _ in range(max(0, a.warmup - 1)):
        b.replay()
    torch.cuda.synchronize(dev)
    iters = int(b.iters.sum().item())
    flops = batch_flops(b)
    events = [[torch.cuda.Event(enable_timing=True) for _ in range(2)] for _ in range(a.steps)]
    if world > 1:
        import torch.distributed as dist
        dist.barrier()
    torch.cuda.synchronize(dev)
    t_wall = time.perf_counter()
    with ClockSampler(dev.index or 0) as clk:
        for k in range(a.steps):
            flush.fill_(k & 0xFF)
            events[k][0].record()
            b.replay()
            events[k][1].record()
        torch.cuda.synchronize(dev)
    t_wall = time.perf_counter() - t_wall
    if world > 1:
        dist.barrier()
    step_ms = [e[0].elapsed_time(e[1]) for e in events]
    assert int(b.iters.sum().item()) == iters, "non-deterministic iteration count"
    total_ms, iters_all = aggregate(sum(step_ms), iters, world, dev)
    value = iters_all * a.steps / (total_ms / 1e3)

    # end to end: the problem tables go up (zeus_batch_prepare), the graph
    # runs, every per-start output and the per-problem summaries come back
    pl = b.plan
    host = {k: torch.empty(getattr(b, k).shape, dtype=getattr(b, k).dtype).pin_memory()
            for k in ("x", "f", "gnorm", "status", "iters", "results")}
    e2e_ms = []
    for k in range(max(1, a.e2e_steps)):
        flush.fill_(k & 0xFF)
        torch.cuda.synchronize(dev)
        t0 = time.perf_counter()
        z.zeus_batch_prepare(b.problems, pl, b.workspace)
        b.replay()
        for name, h in host.items():
            h.copy_(getattr(b, name), non_blocking=True)
        torch.cuda.synchronize(dev)
        e2e_ms.append((time.perf_counter() - t0) * 1e3)
    assert int(host["iters"].sum().item()) == iters
    e2e_value = iters * len(e2e_ms) / (sum(e2e_ms) / 1e3)
    d2h = sum(h.numel() * h.element_size() for h in host.values())

    step_s = statistics.mean(step_ms) / 1e3
    achieved = flops / step_s / 1e12
    roof = {"kernel": "batch_bfgs_kernel (all classes + hand-over) + batch PSO + argmin",
            "bound": "alu", "achieved": round(achieved, 5), "peak": FP64_PEAK_TFLOPS,
            "unit": "TFLOP/s", "frac": round(achieved / FP64_PEAK_TFLOPS, 5), "traffic": None,
            "peak_source": "FP64 FMA rate measured on this GB300 (1.25 TFLOP/s, equal to the "
                           "part's nominal FP64 rate)",
            "model": "bench.py fp64_flops per problem (Alg. 5 passes as implemented)",
            "flops_per_launch": flops, "launch_ms": round(step_s * 1e3, 3)}
    st = b.status.cpu().numpy()
    out = {
        "metric": METRIC, "value": round(value, 1), "unit": METRIC, "n_gpus": world,
        "steps": a.steps, "warmup": a.warmup, "ms_per_step": round(total_ms / a.steps, 3),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32" if a.precision == "fp32_guarded" else "f64",
        "data": "synthetic (seeded mixed problem list; Philox draws of the method itself)",
        "config": {"workload": BATCH_WORKLOAD if not a.problems
                   else f"first {pl.n_problems} problems of {BATCH_WORKLOAD}",
                   "problems": pl.n_problems,
                   "starts": int(pl.total_starts), "pso_iters": 10, "bfgs_max_iters": 500,
                   "grad_mode": a.grad_mode, "precision": a.precision,
                   "start_iters_per_step": iters, "bfgs_classes": int(pl.n_classes),
                   "autotune": dict(_tuned_summary(b), setup_s=round(tune_s, 2)),
                   "l2": "flushed between timed steps (256 MB write outside the events)",
                   "step": "one CUDA graph replay of zeus_batch_solve",
                   "parallelism": f"replicas x{world}"},
        "e2e": {"value": round(e2e_value, 1), "unit": METRIC,
                "h2d_bytes_per_step": int(pl.table_bytes), "d2h_bytes_per_step": d2h,
                "api": "zeus_batch_prepare (tables up, synchronizes) + graph replay + all outputs back"},
        "gpu_launches": a.steps * b.launches,
        "roofline": roof,
        "status_counts": {str(k): int(c) for k, c in zip(*np.unique(st, return_counts=True))},
        "problems_at_1e-6": int(sum(s["best_f"] <= 1e-6 for s in b.summaries())),
        "wall_s_timed": round(t_wall, 3),
        "clocks": clk.summary(),
    }
    extras_on = rank == 0 and world == 1 and not a.no_extras
    if extras_on:
        out["cluster"] = batch_cluster_figures(b, dev)
    del b
    torch.cuda.empty_cache()
    if extras_on:
        out["extras"] = run_extras(z, dev, a)
        stream = torch.cuda.current_stream(dev)
        out["forms"] = run_forms(z, dev, stream, seeds=a.form_seeds)
        out["fp32_error"] = run_fp32_error(z, dev)
        out["study"] = run_study_sweep(z, dev)
    if rank == 0 and not a.no_cpu_baseline:
        out["cpu_baseline"] = cpu_baseline_batch(budget_s=12.0)
    if rank == 0:
        print(json.dumps(out), flush=True)


def batch_cluster_figures(b, dev) -> dict:
    """Every problem's final points clustered in one launch (converged
    starts by coordinates, tol 1e-4, the first 64 regions of each)."""
    import torch
    b.cluster(method="x", tol=1e-4, max_clusters=64)
    c0, c1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    stream = torch.cuda.current_stream(dev)
    c0.record(stream)
    cl = None
    for _ in range(3):
        cl = b.cluster(method="x", tol=1e-4, max_clusters=64)
    c1.record(stream)
    torch.cuda.synchronize(dev)
    sums = cl["summaries"]
    return {"kernel": "batch_cluster_kernel (one block per problem)", "method": "x",
            "tol": 1e-4, "max_clusters": 64, "only_converged": True,
            "ms": round(c0.elapsed_time(c1) / 3, 3),
            "note": "ms includes copying the summaries back",
            "regions_total": int(sum(s["n_clusters"] for s in sums)),
            "problems_with_best_count_ge_2": int(sum(s["best_count"] >= 2 for s in sums))}


# ---------------------------------------------------------------- extras

EXTRA_LINES = [
    # (name, workload, overrides, steps, warmup)
    ("rastrigin10d_n16384", "rastrigin10d_n16384", {}, 10, 3),
    ("rosenbrock256d_n8192/fp32_guarded", "rosenbrock256d_n8192", {"precision": "fp32_guarded"}, 3, 2),
    ("rosenbrock256d_n8192/fp64", "rosenbrock256d_n8192", {"precision": "fp64"}, 2, 1),
    ("rosenbrock1024d_n2048/fp32_guarded/adjoint", "rosenbrock1024d_n2048",
     {"precision": "fp32_guarded", "grad_mode": "adjoint"}, 2, 1),
    ("rosenbrock1024d_n2048/fp32_guarded/forward", "rosenbrock1024d_n2048",
     {"precision": "fp32_guarded", "grad_mode": "forward"}, 2, 1),
    ("ackley1024d_n2048/fp32_guarded/adjoint", "ackley1024d_n2048",
     {"precision": "fp32_guarded", "grad_mode": "adjoint"}, 2, 1),
    ("ackley1024d_n2048/fp32_guarded/forward", "ackley1024d_n2048",
     {"precision": "fp32_guarded", "grad_mode": "forward"}, 2, 1),
]


def run_extras(z, dev, a) -> dict:
    """The single-problem workloads, each one line with its own roofline
    (steps and warm-up as listed; L2 flushed between steps)."""
    import torch
    out = {}
    for name, wl, over, steps, warm in EXTRA_LINES:
        fields = dict(workloads.workload(wl), **over)
        line, keep = measure_single(z, dev, fields, steps, warm, e2e_steps=1)
        if wl == "rastrigin10d_n16384":
            line["cluster"] = cluster_figures(z, dev, keep)
        del keep
        torch.cuda.empty_cache()
        out[name] = line
    return out


# ------------------------------------------------------------------ forms

FORM_WORKLOADS = ("rosenbrock2d_n128", "rastrigin5d_n16384", "rastrigin10d_n16384")
FORMS = (("fp64", "forward"), ("fp64", "adjoint"), ("fp32_guarded", "forward"),
         ("fp32_guarded", "adjoint"))


def run_forms(z, dev, stream, seeds=20):
    """Time to 1e-6 of the global minimum (f* = 0) of the whole path (PSO +
    BFGS + reduction) with the stop-on-target flag, per workload and form,
    over `seeds` seeds: median time, success (best f <= 1e-6) with its 95 %
    Clopper-Pearson interval, and the start-iterations made.  Forms: the
    plain FP64 method (forward-mode duals), the FP64 adjoint, the FP32 form
    with FP64 guards (forward and adjoint).  A run that never reaches the
    target ends when every start has ended; its time is the time to finish.
    Then the batched form: 16 independent 5-D Rastrigin problems, and the
    whole 4096-problem batch, FP64 against the FP32 form."""
    out = {}
    for w in FORM_WORKLOADS:
        out[w] = _forms_on(z, workloads.workload(w), dev, stream, seeds)
    out["batched_rastrigin5d_x16"] = _batched_to_target(z, dev, stream)
    out["batched_" + BATCH_WORKLOAD] = _whole_batch_to_target(z, dev)
    return out


def _forms_on(z, fields, dev, stream, seeds):
    import torch
    out = {}
    for prec, grad in FORMS:
        times, ok, iters = [], 0, []
        for r in range(seeds + 1):  # the first run warms up
            f = dict(fields, precision=prec, grad_mode=grad, target_f=1e-6, seed=1000 + r)
            p = _problem(z, f)
            pc = p.to_c()
            ws = z.new_workspace(pc, dev)
            xo = torch.empty(p.n_starts, p.dim, dtype=torch.float64, device=dev)
            fo = torch.empty(p.n_starts, dtype=torch.float64, device=dev)
            res = z.new_result(dev)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize(dev)
            e0.record(stream)
            z.zeus_solve(pc, ws, xo, fo, None, None, None, res, stream)
            e1.record(stream)
            torch.cuda.synchronize(dev)
            if r == 0:
                continue
            s = z.decode_result(res)
            times.append(e0.elapsed_time(e1))
            ok += int(s["best_f"] <= 1e-6)
            iters.append(int(s["total_iters"]))
        out[f"{prec}/{grad}"] = {"time_to_target_ms": round(statistics.median(times), 3),
                                 "time_q25_q75_ms": [round(float(np.percentile(times, 25)), 3),
                                                     round(float(np.percentile(times, 75)), 3)],
                                 "success": f"{ok}/{seeds}", "success_ci95": clopper_pearson(ok, seeds),
                                 "start_iters_median": int(statistics.median(iters))}
    return out


def _batched_to_target(z, dev, stream, n_problems=16):
    """Time to 1e-6 of the global minimum for 16 independent 5-D Rastrigin
    problems (16384 particles each, seeds 2000..2015): the plain FP64 method
    one problem after another, against one batch (FP64, and FP32 with FP64
    guards) replayed from a CUDA graph.  Success = problems whose best f
    reached 1e-6."""
    import torch
    base = dict(workloads.workload("rastrigin5d_n16384"), target_f=1e-6)
    fields = [dict(base, seed=2000 + i) for i in range(n_problems)]
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    res = {}
    singles = []
    for f in fields:
        pc = _problem(z, f).to_c()
        singles.append((pc, z.new_workspace(pc, dev),
                        torch.empty(pc.n_starts * pc.dim, dtype=torch.float64, device=dev),
                        torch.empty(pc.n_starts, dtype=torch.float64, device=dev), z.new_result(dev)))
    for rep in range(2):  # the first pass warms up
        torch.cuda.synchronize(dev)
        e0.record(stream)
        for pc, ws, x, fo, r in singles:
            z.zeus_solve(pc, ws, x, fo, None, None, None, r, stream)
        e1.record(stream)
        torch.cuda.synchronize(dev)
    ok = sum(int(z.decode_result(r)["best_f"] <= 1e-6) for *_, r in singles)
    res["fp64/forward one by one"] = {"time_to_target_ms": round(e0.elapsed_time(e1), 3),
                                     "success": f"{ok}/{n_problems}",
                                     "success_ci95": clopper_pearson(ok, n_problems)}
    for prec in ("fp64", "fp32_guarded"):
        b = z.Batch([_problem(z, dict(f, precision=prec)) for f in fields], device=dev)
        b.solve()
        torch.cuda.synchronize(dev)
        b.capture()
        times = []
        for rep in range(3):
            e0.record()
            b.replay()
            e1.record()
            torch.cuda.synchronize(dev)
            times.append(e0.elapsed_time(e1))
        ok = sum(int(s["best_f"] <= 1e-6) for s in b.summaries())
        res[f"{prec}/forward batched"] = {"time_to_target_ms": round(statistics.median(times), 3),
                                         "success": f"{ok}/{n_problems}",
                                         "success_ci95": clopper_pearson(ok, n_problems)}
    return res


def _whole_batch_to_target(z, dev) -> dict:
    """The whole 4096-problem batch with the stop-on-target flag of every
    problem at 1e-6 (f* = 0 for all three objectives): one graph replay per
    form (median of three), problems whose best f reached 1e-6 with their
    95 % interval, and the start-iterations made.  Layouts autotuned."""
    import torch
    out = {}
    flush = torch.empty(256 * 1024 * 1024, dtype=torch.uint8, device=dev)
    tuner = _tuner()
    for prec in ("fp64", "fp32_guarded"):
        fields = workloads.batch_problems(BATCH_WORKLOAD, None, precision=prec, target_f=1e-6)
        t0 = time.perf_counter()
        b = z.Batch([z.Problem(**f) for f in fields], device=dev, autotuner=tuner)
        tune_s = time.perf_counter() - t0
        b.solve()
        torch.cuda.synchronize(dev)
        b.capture()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        times = []
        for rep in range(3):
            flush.fill_(rep)
            e0.record()
            b.replay()
            e1.record()
            torch.cuda.synchronize(dev)
            times.append(e0.elapsed_time(e1))
        sums = b.summaries()
        ok = sum(int(s["best_f"] <= 1e-6) for s in sums)
        n = len(sums)
        st = b.status.cpu().numpy()
        out[f"{prec}/forward"] = {"time_to_target_ms": round(statistics.median(times), 2),
                                  "problems_at_target": f"{ok}/{n}",
                                  "success_ci95": clopper_pearson(ok, n),
                                  "start_iters": int(b.iters.sum().item()),
                                  "status_counts": {str(k): int(c) for k, c in
                                                    zip(*np.unique(st, return_counts=True))},
                                  "autotune_setup_s": round(tune_s, 2)}
        del b
        torch.cuda.empty_cache()
    return out


# ------------------------------------------------------- FP32 form error

def run_fp32_error(z, dev) -> dict:
    """The FP32 form's error start by start against the FP64 method from the
    same start points (the PSO phase's final positions; precision_error):
    |f32 - f64| quantiles and the share within 1e-6, on the 10-D Rastrigin
    workload (all 16384 starts) and on 512 starts of the d = 256 Rosenbrock
    chain workload.  The FP64 method is itself checked against the FP64
    oracle per start in the GPU tests."""
    out = {}
    for name, n_sample in (("rastrigin10d_n16384", None), ("rosenbrock256d_n8192", 512)):
        fields = workloads.workload(name)
        p = _problem(z, fields)
        sw = z.pso(p, device=dev)
        x0 = sw["x"]
        if n_sample:
            idx = np.random.default_rng(7).choice(p.n_starts, n_sample, replace=False)
            x0 = x0[idx].contiguous()
            p = p.replace(n_starts=n_sample)
        r = z.precision_error(p, x0, device=dev)
        s = r["summary"]
        out[name] = dict({k: (round(v, 12) if isinstance(v, float) else v) for k, v in s.items()},
                         status_fp32={str(k): int(c) for k, c in
                                      zip(*np.unique(r["status_fp32"], return_counts=True))})
    return out


# -------------------------------------------------- early-stop study sweep

def _study_run(z, fields, dev, xstar):
    """One early-stopped solve: (ms, correct starts).  Correct: the start
    converged (||g|| < tol) within Euclidean distance 0.5 of the global
    minimiser, the paper's N_correct (Section V)."""
    import torch
    p = _problem(z, fields)
    pc = p.to_c()
    ws = z.new_workspace(pc, dev)
    x = torch.empty(p.n_starts, p.dim, dtype=torch.float64, device=dev)
    st = torch.empty(p.n_starts, dtype=torch.int32, device=dev)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    z.zeus_solve(pc, ws, x, None, None, st, None, None)
    e1.record()
    torch.cuda.synchronize(dev)
    dist = torch.linalg.norm(x - torch.tensor(xstar, dtype=torch.float64, device=dev), dim=1)
    correct = int(((st == 1) & (dist < 0.5)).sum().item())
    return e0.elapsed_time(e1), correct


def _quart(v):
    q = np.percentile(np.asarray(v, dtype=np.float64), [25, 50, 75])
    return [round(float(t), 3) for t in q]


def study_pso_sweep(z, dev, runs, Ts=(0, 1, 2, 5, 10, 20)) -> dict:
    """The early-stop study's PSO-update sweep (the shapes of the paper's
    PSO-iteration experiments, Section V): 5-D Rastrigin and Rosenbrock,
    16384 particles, every run stopped once 100 starts have converged
    (required_c, Alg. 10); time and N_correct quartiles over the runs."""
    out = {}
    for obj, box, xs in (("rastrigin", (-5.12, 5.12), 0.0), ("rosenbrock", (-5.0, 5.0), 1.0)):
        rows = []
        for T in Ts:
            ts, nc = [], []
            for r in range(runs + 1):  # the first run warms up
                f = dict(objective=obj, dim=5, lower=box[0], upper=box[1], n_starts=16384,
                         pso_iters=T, bfgs_max_iters=1000, required_converged=100, seed=500 + r)
                ms, c = _study_run(z, f, dev, [xs] * 5)
                if r:
                    ts.append(ms)
                    nc.append(c)
            rows.append({"T": T, "time_ms_q": _quart(ts), "n_correct_q": _quart(nc)})
        out[f"{obj}5d_n16384"] = rows
    return out


def run_study_sweep(z, dev) -> dict:
    return {"study": "early stop at 100 converged starts", "runs": 5,
            "pso_iters": study_pso_sweep(z, dev, runs=5, Ts=(0, 2, 5, 10, 20))}


def run_study(a):
    """The whole early-stop study: the PSO-update sweep and N_correct
    against d (Rastrigin, 10^5 particles, T = 5).  Prints one JSON line of
    medians and quartiles over the runs."""
    import torch
    import paper_2603_28770_gb300 as z
    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    runs = a.study_runs
    out = {"study": "early stop at 100 converged starts", "runs": runs,
           "pso_iters": study_pso_sweep(z, dev, runs), "dims": {}}
    rows = []
    for d in range(1, 11):
        nc = []
        for r in range(runs):
            f = dict(objective="rastrigin", dim=d, lower=-5.12, upper=5.12, n_starts=100000,
                     pso_iters=5, bfgs_max_iters=1000, required_converged=100, seed=900 + r)
            nc.append(_study_run(z, f, dev, [0.0] * d)[1])
        rows.append({"d": d, "n_correct_q": _quart(nc)})
    out["dims"]["rastrigin_n100000_T5"] = rows
    print(json.dumps(out), flush=True)


# ------------------------------------------------------------ oracle arm

def _oracle_sample(fields, n_sample, threads):
    import oracle
    op = oracle.Problem(**{k: v for k, v in fields.items() if k in oracle.Problem.__dataclass_fields__})
    op.n_threads = threads
    t0 = time.perf_counter()
    sw = oracle.pso(op)
    x0 = sw["x"][:n_sample]
    r = oracle.bfgs_many(op, x0)
    dt = time.perf_counter() - t0
    return int(r["iters"].sum()), dt


def _cpu_single(fields, budget_s, threads) -> dict:
    n_sample = 16
    iters, dt = _oracle_sample(fields, n_sample, threads)
    while dt < budget_s / 4 and n_sample < fields["n_starts"]:
        n_sample = min(fields["n_starts"], n_sample * 4)
        iters, dt = _oracle_sample(fields, n_sample, threads)
    return {"value": round(iters / dt, 1), "unit": METRIC, "cores": threads, "kind": "oracle",
            "sample": f"PSO over all {fields['n_starts']} particles + BFGS from the first "
                      f"{n_sample} of them ({iters} start-iterations in {dt:.2f} s, OpenMP)"}


def cpu_baseline(fields, budget_s=12.0) -> dict:
    """The FP64 oracle as it stands on the host cores: the full PSO phase
    plus BFGS from the first M particles, M grown until ~budget_s; the same
    on one core beside it."""
    import oracle
    oracle.build()
    threads = os.cpu_count() or 1
    out = _cpu_single(fields, budget_s, threads)
    out["single_core"] = _cpu_single(fields, budget_s / 2, 1)
    return out


def _oracle_batch_sample(budget_s, threads):
    """Whole-method oracle solves of the batch's problems in order until
    budget_s has passed: (start-iterations, seconds, problems)."""
    import oracle
    fields = workloads.batch_problems(BATCH_WORKLOAD, None)
    iters, t0, n = 0, time.perf_counter(), 0
    for f in fields:
        op = oracle.Problem(**{k: v for k, v in f.items() if k in oracle.Problem.__dataclass_fields__})
        op.n_threads = threads
        iters += int(oracle.solve(op)["iters"].sum())
        n += 1
        if time.perf_counter() - t0 > budget_s:
            break
    return iters, time.perf_counter() - t0, n


def cpu_baseline_batch(budget_s=12.0) -> dict:
    import oracle
    oracle.build()
    out = {}
    for key, threads, b in (("all", os.cpu_count() or 1, budget_s), ("single_core", 1, budget_s / 2)):
        iters, dt, n = _oracle_batch_sample(b, threads)
        out[key] = {"value": round(iters / dt, 1), "unit": METRIC, "cores": threads, "kind": "oracle",
                    "sample": f"the first {n} problems of {BATCH_WORKLOAD}, whole method, FP64 "
                              f"({iters} start-iterations in {dt:.2f} s, OpenMP)"}
    res = dict(out["all"])
    res["single_core"] = out["single_core"]
    return res


def run_reference(a):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    import oracle
    oracle.build()
    threads = os.cpu_count() or 1
    if a.workload in workloads.BATCH_WORKLOADS:
        for _ in range(a.warmup):
            _oracle_batch_sample(0.0, threads)
        times, iters, probs = [], [], 0
        for _ in range(a.steps):
            it, dt, n = _oracle_batch_sample(5.0, threads)
            times.append(dt)
            iters.append(it)
            probs = n
        value = sum(iters) / sum(times)
        sample = f"per step: whole-method oracle solves of the first {probs} problems"
    else:
        fields = workloads.workload(a.workload)
        # BFGS from as many of the swarm's particles as fit about half a
        # second per step, so that the full PSO phase does not weigh on a
        # small BFGS sample
        n_sample = 64
        _, dt = _oracle_sample(fields, n_sample, threads)
        while dt < 0.5 and n_sample < fields["n_starts"]:
            n_sample = min(fields["n_starts"], n_sample * 4)
            _, dt = _oracle_sample(fields, n_sample, threads)
        for _ in range(a.warmup):
            _oracle_sample(fields, n_sample, threads)
        times, iters = [], []
        for _ in range(a.steps):
            it, dt = _oracle_sample(fields, n_sample, threads)
            times.append(dt)
            iters.append(it)
        value = sum(iters) / sum(times)
        sample = (f"per step: PSO over all {fields['n_starts']} particles + BFGS from the first "
                  f"{n_sample}")
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": round(value, 1), "unit": METRIC,
        "n_gpus": world, "steps": a.steps, "warmup": a.warmup,
        "ms_per_step": round(1e3 * sum(times) / a.steps, 3), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": a.workload, "sample": sample},
        "cpu_baseline": {"value": round(value, 1), "unit": METRIC, "cores": threads,
                         "kind": "oracle", "sample": sample},
        "e2e": {"value": round(value, 1), "unit": METRIC, "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }), flush=True)


# ------------------------------------------------------------------ main

def run_zeus(a):
    import torch
    import torch.distributed as dist

    import paper_2603_28770_gb300 as z

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if a.workload in workloads.BATCH_WORKLOADS:
        run_batch_main(a, z, dev, world, rank)
    else:
        run_single_main(a, z, dev, world, rank)
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    args = _args()
    if args.study:
        run_study(args)
        sys.exit(0)
    if args.impl == "reference":
        run_reference(args)
    else:
        run_zeus(args)
