#!/usr/bin/env python
"""Benchmark of the PonD D2Q16 time step on GB300.

Headline (one JSON line on rank 0): node-updates/s of the plain FP64 step on
the 2048 x 2048 supersonic workload (uniform u = (1.5, 0.5), rho and T with
8 seeded sinusoidal perturbations), inputs resident in HBM.  Extra keys
report the mixed FP32/FP64 form on the same field and on the 4096^2
temperature-ratio-4 field, the batched ensemble (256 uneven grids, one
graph-replayed persistent launch per step), the moment error of the mixed
form against the FP64 run, the roofline of the dominant kernel, the FP64 CPU
oracle on a bounded sample, and the end-to-end rate through host buffers.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

Under torchrun (N > 1) every rank advances its own replica of the workload
(weak scaling, no collective on the data path).
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "PonD D2Q16 node-updates/s (FP32 vs FP64 @ moment err); adjoint/forward time"
UNIT = "node-updates/s"
WORKLOAD = "supersonic-2048-fp64"

# Algorithmic FP work per predictor-corrector pass of one node (D2Q16,
# 4 x 4 stencil): 256 (population, source) pairs x 56 fused multiply-adds
# (3 gauge differences, 8 xi offsets, 24 Lagrange-Taylor terms, 20
# contraction, 1 weighted accumulate) = 28672 flops, plus 16 departures with
# their cubic weights (20 flops each) and the moments / gauge update (128).
FLOP_PER_PASS = 256 * 112 + 16 * 20 + 128
# Algorithmic HBM bytes per node update: read and write 16 populations and
# 3 FP64 gauge values (FP64: 2 x 152 B; mixed: 2 x (64 + 24) B).
BYTES_FP64 = 2 * (16 * 8 + 3 * 8)
BYTES_MIXED = 2 * (16 * 4 + 3 * 8)
# The same on D2Q9 (9 populations, quadratic 1D maps): 144 pairs x 34 FMAs
# (3 gauge differences, 6 xi offsets, 12 Lagrange-Taylor terms, 12
# contraction, 1 accumulate), 9 departures, moments 9 x 8.
FLOP_PER_PASS_Q9 = 144 * 68 + 9 * 20 + 72
BYTES_FP64_Q9 = 2 * (9 * 8 + 3 * 8)
BYTES_MIXED_Q9 = 2 * (9 * 4 + 3 * 8)
# The reference-gauge staged kernel (the default) does less arithmetic per
# pass: the sources are re-expressed once per step in the tile's reference
# gauge, and each pass, for every x-speed index k, sweeps the rows of the
# union of the n1 y-stencils.  FP64 form: per row, 4 sources x n1 x n1 FMAs
# (the x-interpolation with the x-map folded into its weights, formed once
# per k: 4 n1 products), and each population (k, l) takes its four rows once
# (4 x n1 FMAs).  Mixed form (every_row=True): per row the x-interpolation
# (4 n1^2), the x-map (n1^2) and the row added to the n1 populations (n1^2,
# zero weights outside a stencil).  The rows per sweep are
# 4 + (c_max - c_min) sqrt(theta) on average (the spread of the y-departures
# plus the stencil).  Per (node, k) add the x-map's Taylor entries (5 n1
# ops), the departure and cubic weights (20), the y-map applied after the
# sweep (mixed: n1 x 6 n1 FMAs with its entries; FP64: n1 x n1 FMAs, the
# entries computed once per pass, 4 n1^2 FMAs) and the moments (8 n1); per
# pass the y-departures (20 n1) and the gauge update (40).  The once-per-step staging (~500 flops
# per staged source) is left out: the count is the per-pass work alone, so
# the fraction is a lower bound.
def staged_flops_per_pass(n1: int, st_mean: float, every_row: bool = False) -> float:
    spread = 2 * 2.3344142183389773 if n1 == 4 else 2.0
    rows = 4.0 + spread * st_mean
    if every_row:
        sweep = 2 * (4 * n1 * n1 + n1 * n1 + n1 * n1) * rows
        ymap_k, ymap_pass = n1 * 2 * 6 * n1, 0
    else:
        sweep = 2 * (4 * n1 * n1) * rows + 4 * n1 + 2 * 4 * n1 * n1
        # the y-map entries once per pass (a table), one FMA each per (k, l, b)
        ymap_k, ymap_pass = 2 * n1 * n1, 2 * 4 * n1 * n1
    per_k = sweep + 2 * 5 * n1 + 20 + ymap_k + 8 * n1
    return n1 * per_k + 20 * n1 + 40 + ymap_pass


# Nominal peaks of the arithmetic pipes at the 2070 MHz maximum SM clock
# (FP64 1.25 TFLOP/s; FP32 152 SMs x 128 lanes x 2 flops x 2.07 GHz).  The
# roofline uses the rates the FMA-chain probe (pond_measure_peak) measures
# at the start of every run instead; these are the fallback if it fails.
PEAK_FP64_TFLOPS = 1.25
PEAK_FP32_TFLOPS = 152 * 128 * 2 * 2.07e9 / 1e12
# DRAM bytes per FP64 step launch at 2048^2 of the staged kernel: the ncu
# capture of the same kernel (k_step_staged<StagedFP64, 32, 8, 4>) at 1024^2
# read 161.5 MB and wrote 125.6 MB; traffic grows with the node count (4x).
K_STAGED64_TRAFFIC_2048 = 4 * (161.49e6 + 125.57e6)
K_STAGED64_TRAFFIC_SOURCE = ("ncu dram__bytes_read.sum + dram__bytes_write.sum of one "
                             "k_step_staged<StagedFP64, 32, 8, 4> launch at 1024^2 (287.1 MB), "
                             "scaled x4 by nodes to the 2048^2 launch")


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="pond", choices=["pond", "reference"])
    ap.add_argument("--no-forms", action="store_true", help="headline only")
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU oracle sample")
    ap.add_argument("--cpu-seconds", type=float, default=12.0)
    ap.add_argument("--precision-steps", type=int, default=1000,
                    help="steps of the mixed-vs-FP64 moment-error leg")
    ap.add_argument("--precision-quick", action="store_true",
                    help="run that leg at 2048^2 instead of the full 4096^2 field "
                         "(whose FP64 reference takes ~6 min)")
    ap.add_argument("--precision-full", action="store_true",
                    help="the full 4096^2 field (the default; kept for older command lines)")
    return ap.parse_args()


def measured_peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        return {}


# ------------------------------------------------------------------ clocks

class ClockSampler:
    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.FIELDS,
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None
        time.sleep(0.3)
        return self

    def __exit__(self, *a):
        self.out = ""
        if self.proc:
            time.sleep(0.25)
            self.proc.terminate()
            try:
                self.out, _ = self.proc.communicate(timeout=5)
            except Exception:
                self.proc.kill()
                self.out = ""

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in (self.out or "").splitlines():
            p = [x.strip() for x in line.split(",")]
            if len(p) < 8:
                continue
            try:
                sm.append(float(p[0]))
                mx.append(float(p[1]))
            except ValueError:
                continue
            for n, v in zip(names, p[4:8]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": max(mx),
                "reasons": sorted(reasons), "samples": len(sm)}


# ------------------------------------------------------------------ helpers

def dist_setup():
    import torch
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        if torch.cuda.is_available():
            torch.cuda.set_device(local)
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    return world, rank, local


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(world, value: float) -> float:
    if world == 1:
        return value
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([value], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def oracle_rows_for(st, ny: int, seconds: float, params=None) -> int:
    """Rows R of the workload whose oracle step takes about `seconds`.  The
    first step call pays a large one-off cost (the output state's first
    touch), and every call a fixed one, so the per-row time comes from the
    difference of two timed probes after an untimed warm-up call."""
    import oracle
    oracle.step(st, params, rows=(0, 1))
    lo, hi = min(2, ny), min(6, ny)
    t0 = time.perf_counter()
    oracle.step(st, params, rows=(0, lo))
    t_lo = time.perf_counter() - t0
    if hi == lo:
        return ny
    t0 = time.perf_counter()
    oracle.step(st, params, rows=(0, hi))
    t_hi = time.perf_counter() - t0
    per_row = max((t_hi - t_lo) / (hi - lo), 1e-4)
    fixed = max(t_lo - lo * per_row, 0.0)
    return int(max(1, min(ny, (seconds - fixed) / per_row)))


def oracle_sample(fields, seconds: float, params=None):
    """Time the FP64 CPU oracle on a bounded sample: one step of the first R
    rows of the workload, R sized for about `seconds` of CPU time."""
    import oracle
    st = oracle.init_equilibrium(fields.rho, fields.ux, fields.uy, fields.T)
    ny, nx = fields.shape
    rows = oracle_rows_for(st, ny, seconds, params)
    t0 = time.perf_counter()
    oracle.step(st, params, rows=(0, rows))
    dt = time.perf_counter() - t0
    cores = oracle.num_threads()
    out = {"value": rows * nx / dt, "unit": UNIT, "cores": cores, "kind": "oracle",
           "sample": "one FP64 oracle step of rows 0..%d (%d nodes) of the %dx%d field, %.1f s"
                     % (rows - 1, rows * nx, nx, ny, dt)}
    # the same oracle on one core, on a sample a few times smaller
    rows1 = max(1, rows // max(2, 2 * cores))
    oracle.set_num_threads(1)
    try:
        t0 = time.perf_counter()
        oracle.step(st, params, rows=(0, rows1))
        dt1 = time.perf_counter() - t0
    finally:
        oracle.set_num_threads(cores)
    out["single_thread"] = {"value": rows1 * nx / dt1, "cores": 1,
                            "sample": "rows 0..%d (%d nodes), %.1f s" % (rows1 - 1, rows1 * nx, dt1)}
    return out


def measure_peaks(local):
    """FP64 and FP32 FMA rates of this GPU, measured now by the library's
    FMA-chain probe (pond_measure_peak; best of three launches of about
    0.1 s each), with the clocks seen meanwhile.  The FP32 figure is the
    packed fma.rn.f32x2 form, which reaches the pipe's rate with half the
    issue slots; the scalar form is reported beside it."""
    import torch
    from paper_1806_05089_gb300 import pond
    sink = torch.zeros(16, dtype=torch.float64, device="cuda")
    out = {}
    with ClockSampler(local) as clk:
        for name, pipe, iters in (("fp64", pond.POND_PIPE_FP64, 2000),
                                  ("fp32_scalar", pond.POND_PIPE_FP32, 100000),
                                  ("fp32", pond.POND_PIPE_FP32X2, 50000)):
            try:
                out[name] = max(pond.pond_measure_peak(pipe, iters, sink)[0] for _ in range(3))
            except Exception as e:  # keep the bench running on the nominal figure
                out[name + "_error"] = str(e)
    out["clocks"] = clk.summary()
    out["how"] = ("pond_measure_peak: 8 independent FMA chains per thread, grid = SMs x resident "
                  "CTAs of 256 threads, one launch of ~0.1 s timed with CUDA events after a "
                  "warm-up launch, best of 3")
    return out


def time_steps(sim, stream, steps):
    """Time `steps` PonD steps on `stream` with CUDA events; returns (seconds,
    stats)."""
    import torch
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    stats = sim.step(steps)
    e1.record(stream)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / 1e3, stats


def form_line(name, nodes, steps, secs, stats, precision_peak_tflops, bytes_per_update,
              flop_per_pass=FLOP_PER_PASS, direct_flop_per_pass=FLOP_PER_PASS):
    """One form's throughput and roofline; flop_per_pass is the count of the
    kernel that ran (staged_flops_per_pass for the staged kernel, the
    per-pair count FLOP_PER_PASS for the direct ones).  The per-pair count
    of the lattice (direct_flop_per_pass) gives the direct-equivalent rate
    beside it: the same throughput counted as the per-pair form's work."""
    passes = stats["passes"] / max(stats["node_updates"], 1)
    achieved = flop_per_pass * stats["passes"] / secs / 1e12
    direct_eq = direct_flop_per_pass * stats["passes"] / secs / 1e12
    return {
        "workload": name,
        "value": nodes * steps / secs,
        "unit": UNIT,
        "steps": steps,
        "ms_per_step": secs / steps * 1e3,
        "mean_passes": passes,
        "max_passes": stats["max_passes"],
        "nonconverged": stats["nonconverged"],
        "halo_fallback": stats.get("halo_fallback", 0),
        "tile": [32, stats.get("tile_rows", 0)],
        "alu_tflops": achieved,
        "alu_frac": achieved / precision_peak_tflops,
        "flop_per_pass": flop_per_pass,
        "direct_equivalent_frac": direct_eq / precision_peak_tflops,
        "hbm_gbs_algorithmic": nodes * steps * bytes_per_update / secs / 1e9,
    }


# ------------------------------------------------------------------ arms

def run_reference(args, world, rank):
    from paper_1806_05089_gb300 import workloads
    if rank != 0:
        return
    import oracle
    fields = workloads.supersonic(2048)
    st = oracle.init_equilibrium(fields.rho, fields.ux, fields.uy, fields.T)
    ny, nx = fields.shape
    budget = min(args.cpu_seconds, max(0.05, 150.0 / max(args.steps + args.warmup, 1)))
    rows = oracle_rows_for(st, ny, budget)
    for _ in range(args.warmup):
        oracle.step(st, None, rows=(0, 1))
    times = []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        oracle.step(st, None, rows=(0, rows))
        times.append(time.perf_counter() - t0)
    secs = float(np.sum(times))
    value = rows * nx * args.steps / secs
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "impl": "reference",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": secs / args.steps * 1e3, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "nx": nx, "ny": ny,
                   "sample_rows_per_step": rows},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": oracle.num_threads(),
                         "kind": "oracle",
                         "sample": "each step: one FP64 oracle step of rows 0..%d of the %dx%d field"
                                   % (rows - 1, nx, ny)},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def run_pond(args, world, rank, local):
    import torch
    from paper_1806_05089_gb300 import pond, workloads

    if not torch.cuda.is_available():
        raise SystemExit("bench.py needs a CUDA GPU (the library has no CPU path)")
    torch.cuda.set_device(local)
    pond.load()
    peaks = measured_peaks()
    stream = torch.cuda.Stream()
    fields = workloads.supersonic(2048)
    ny, nx = fields.shape
    nodes = nx * ny
    probe = measure_peaks(local)
    peak64 = probe.get("fp64", PEAK_FP64_TFLOPS)
    peak32 = probe.get("fp32", PEAK_FP32_TFLOPS)
    peak_src = ("measured in this run by the FMA-chain probe" if "fp64" in probe
                else "nominal FP64 rate at 2070 MHz (probe failed)")

    # ---- headline: FP64 step (the staged kernel, tile shape autotuned during
    # the warm-up), state resident in HBM (1.2 GB > L2)
    sim = pond.Sim(nx, ny, pond.POND_FP64, stream=stream.cuda_stream, autotune=1)
    sim.set_state(fields.rho, fields.ux, fields.uy, fields.T)
    torch.cuda.synchronize()
    sim.step(args.warmup)
    st_mean = float(np.sqrt(fields.T).mean())
    flop_pass = staged_flops_per_pass(4, st_mean)
    barrier(world)
    with ClockSampler(local) as clk:
        secs, stats = time_steps(sim, stream, args.steps)
    barrier(world)
    secs_max = max_over_ranks(world, secs)
    clocks = clk.summary()
    rho64, ux64, uy64, T64 = sim.moments()
    mean_passes = stats["passes"] / stats["node_updates"]
    kernel_s = secs / args.steps
    achieved = flop_pass * (stats["passes"] / args.steps) / kernel_s / 1e12
    line = {
        "metric": METRIC,
        "value": world * nodes * args.steps / secs_max,
        "unit": UNIT,
        "n_gpus": world,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": secs_max / args.steps * 1e3,
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": WORKLOAD, "nx": nx, "ny": ny, "lattice": "D2Q16",
                   "u": [1.5, 0.5], "perturbation": "8 sinusoids, 0.1/8 each, k 1..8",
                   "nu": 0.01, "eps": [1e-12, 1e-10], "parallelism": "replica per GPU",
                   "l2": "no flush: the state read and written per step (1.27 GB) exceeds L2"},
        "mean_passes": mean_passes,
        "max_passes": stats["max_passes"],
        "nonconverged": stats["nonconverged"],
        "gpu_launches": args.steps,
        "roofline": {"bound": "alu", "pipe": "fp64", "achieved": achieved,
                     "peak": peak64, "unit": "TFLOP/s",
                     "frac": achieved / peak64,
                     "traffic": K_STAGED64_TRAFFIC_2048,
                     "traffic_source": K_STAGED64_TRAFFIC_SOURCE,
                     "peak_source": peak_src,
                     "peak_nominal": PEAK_FP64_TFLOPS,
                     "flop_per_pass": flop_pass,
                     "flop_count": "staged kernel, per-pass sweep only (staging excluded)",
                     "direct_equivalent_tflops": FLOP_PER_PASS * (stats["passes"] / args.steps)
                                                 / kernel_s / 1e12,
                     "tile": [32, stats.get("tile_rows", 0)],
                     "kernel": "k_step_staged<StagedFP64>", "kernel_ms": kernel_s * 1e3,
                     "hbm_gbs_algorithmic": nodes * BYTES_FP64 / kernel_s / 1e9,
                     "hbm_peak_gbs": peaks.get("hbm_gbs")},
        "clocks": clocks,
        "peaks_measured": probe,
    }

    # ---- end to end through the public API with host buffers
    pin = {k: torch.from_numpy(np.ascontiguousarray(getattr(fields, k))).pin_memory()
           for k in ("rho", "ux", "uy", "T")}
    rho_out = torch.empty((ny, nx), dtype=torch.float64).pin_memory()
    e2e_steps = max(2, min(args.steps, 5))
    for it in range(e2e_steps + 1):
        if it == 1:
            torch.cuda.synchronize()
            t0 = time.perf_counter()
        pond.pond_set_state(sim.ctx, 0, pin["rho"], pin["ux"], pin["uy"], pin["T"])
        pond.pond_step(sim.ctx, 1, want_stats=False)
        pond.pond_moments(sim.ctx, 0, rho_out)
    e2e_s = time.perf_counter() - t0
    e2e_max = max_over_ranks(world, e2e_s)
    line["e2e"] = {"value": world * nodes * e2e_steps / e2e_max, "unit": UNIT,
                   "h2d_bytes_per_step": 4 * 8 * nodes, "d2h_bytes_per_step": 8 * nodes,
                   "steps": e2e_steps,
                   "call": "pond_set_state(host rho,u,T) + pond_step(1) + pond_moments(host rho)"}
    sim.close()

    # ---- other forms (not part of the headline's timed region)
    if not args.no_forms:
        forms = {}
        k2 = max(args.steps, 10)
        msim = pond.Sim(nx, ny, pond.POND_FP32_MIXED, stream=stream.cuda_stream, use_graph=1,
                        autotune=1)
        msim.set_state(fields.rho, fields.ux, fields.uy, fields.T)
        msim.step(args.warmup)
        msecs, mstats = time_steps(msim, stream, args.steps)
        rho32, ux32, uy32, T32 = msim.moments()
        forms["fp32_mixed_2048"] = form_line("supersonic-2048-mixed", nodes, args.steps, msecs,
                                             mstats, peak32, BYTES_MIXED,
                                             staged_flops_per_pass(4, st_mean, every_row=True))
        forms["fp32_mixed_2048"]["moment_err_vs_fp64"] = {
            "after_steps": args.warmup + args.steps,
            "rho": float(np.max(np.abs(rho32 - rho64)) / np.max(np.abs(rho64))),
            "u": float(max(np.max(np.abs(ux32 - ux64)), np.max(np.abs(uy32 - uy64)))
                       / np.max(np.hypot(ux64, uy64))),
            "T": float(np.max(np.abs(T32 - T64)) / np.max(np.abs(T64)))}
        forms["fp32_mixed_2048"]["speedup_vs_fp64"] = (nodes * args.steps / msecs) / (
            nodes * args.steps / secs)
        msim.close()

        # the direct per-pair kernels on the same field, for comparison
        for key, prec, peak, nb, kw in (
                ("fp64_direct_2048", pond.POND_FP64, peak64, BYTES_FP64, {}),
                ("fp32_mixed_direct_2048", pond.POND_FP32_MIXED, peak32, BYTES_MIXED,
                 {"use_graph": 1, "autotune": 1})):
            with pond.Sim(nx, ny, prec, stream=stream.cuda_stream, kernel=pond.POND_KERNEL_DIRECT,
                          **kw) as dsim:
                dsim.set_state(fields.rho, fields.ux, fields.uy, fields.T)
                dsim.step(2)
                dsteps = 4 if prec == pond.POND_FP64 else args.steps
                dsecs, dstats = time_steps(dsim, stream, dsteps)
            forms[key] = form_line(key.replace("_", "-"), nodes, dsteps, dsecs, dstats, peak, nb)

        pf = workloads.precision(4096)
        psim = pond.Sim(4096, 4096, pond.POND_FP32_MIXED, stream=stream.cuda_stream, use_graph=1,
                        autotune=1)
        psim.set_state(pf.rho, pf.ux, pf.uy, pf.T)
        psim.step(args.warmup)
        psecs, pstats = time_steps(psim, stream, k2)
        forms["fp32_mixed_4096"] = form_line("precision-4096-mixed", 4096 * 4096, k2, psecs,
                                             pstats, peak32, BYTES_MIXED,
                                             staged_flops_per_pass(4, float(np.sqrt(pf.T).mean()), every_row=True))
        psim.close()
        del pf

        # the ensemble: whole grids sharded over the ranks (largest first to
        # the least loaded rank), each rank's share as one batched context
        from paper_1806_05089_gb300 import decomp
        nxs_all, nys_all = workloads.ensemble_sizes(256)
        mine = decomp.ensemble_shards(nxs_all, nys_all, world)[rank]
        members = workloads.ensemble(256)
        nxs = [nxs_all[i] for i in mine]
        nys = [nys_all[i] for i in mine]
        bsim = pond.Sim(nxs, nys, pond.POND_FP32_MIXED, stream=stream.cuda_stream, use_graph=1,
                        autotune=1)
        for j, i in enumerate(mine):
            m = members[i]
            bsim.set_state(m.rho, m.ux, m.uy, m.T, grid=j)
        bnodes = int(sum(a * b for a, b in zip(nxs, nys)))
        st_b = float(np.average([np.sqrt(members[i].T).mean() for i in mine],
                                weights=[nxs_all[i] * nys_all[i] for i in mine]))
        bsim.step(args.warmup)
        barrier(world)
        bsecs, bstats = time_steps(bsim, stream, k2)
        barrier(world)
        bsecs_max = max_over_ranks(world, bsecs)
        forms["batched_256"] = form_line("ensemble-256-mixed", bnodes, k2, bsecs, bstats,
                                         peak32, BYTES_MIXED,
                                         staged_flops_per_pass(4, st_b, every_row=True))
        forms["batched_256"]["grids_on_this_rank"] = len(mine)
        # share of the persistent launches' CTA slots left idle (start skew
        # and the tail after the work list ran dry), from the kernel's own
        # globaltimer stamps
        if bstats.get("slot_ns", 0) > 0:
            forms["batched_256"]["idle_slot_frac"] = 1.0 - bstats["busy_ns"] / bstats["slot_ns"]
        forms["batched_256"]["all_ranks_value"] = (int(sum(a * b for a, b in zip(nxs_all, nys_all)))
                                                   * k2 / bsecs_max)
        bsim.close()

        # the paper's own D2Q9 lattice on the same supersonic flow, rescaled to
        # T_L = 1/3 (T / 3, u / sqrt 3: the same Mach numbers)
        q9 = workloads.supersonic(2048)
        q9.T, q9.ux, q9.uy = q9.T / 3.0, q9.ux / np.sqrt(3.0), q9.uy / np.sqrt(3.0)
        q9_out = {}
        for key, prec, peak, nbytes in (("fp64_d2q9_2048", pond.POND_FP64, peak64,
                                         BYTES_FP64_Q9),
                                        ("fp32_mixed_d2q9_2048", pond.POND_FP32_MIXED,
                                         peak32, BYTES_MIXED_Q9)):
            extra = {"use_graph": 1, "autotune": 1}
            qsim = pond.Sim(nx, ny, prec, stream=stream.cuda_stream, lattice=pond.POND_D2Q9,
                            T_ref=1.0 / 3.0, **extra)
            qsim.set_state(q9.rho, q9.ux, q9.uy, q9.T)
            qsim.step(args.warmup)
            qsecs, qstats = time_steps(qsim, stream, args.steps)
            forms[key] = form_line("supersonic-2048-d2q9-" + ("fp64" if prec == pond.POND_FP64
                                                              else "mixed"),
                                   nodes, args.steps, qsecs, qstats, peak, nbytes,
                                   staged_flops_per_pass(3, float(np.sqrt(q9.T * 3.0).mean()),
                                                         every_row=prec != pond.POND_FP64),
                                   FLOP_PER_PASS_Q9)
            q9_out[key] = qsim.moments()
            qsim.close()
        r64, u64x, u64y, t64 = q9_out["fp64_d2q9_2048"]
        r32, u32x, u32y, t32 = q9_out["fp32_mixed_d2q9_2048"]
        forms["fp32_mixed_d2q9_2048"]["moment_err_vs_fp64"] = {
            "after_steps": args.warmup + args.steps,
            "rho": float(np.max(np.abs(r32 - r64)) / np.max(np.abs(r64))),
            "u": float(max(np.max(np.abs(u32x - u64x)), np.max(np.abs(u32y - u64y)))
                       / np.max(np.hypot(u64x, u64y))),
            "T": float(np.max(np.abs(t32 - t64)) / np.max(np.abs(t64)))}
        del q9, q9_out

        # the paper's hardest flow: an isentropic vortex advected through the
        # periodic box, over a small (Ma_a, Ma_v) sweep, mixed form (staged
        # kernel), with the pass counts of its iteration map
        vortex = {}
        for ma, mv in ((0.0, 0.5), (1.0, 0.5), (3.0, 0.5), (1.0, 0.8)):
            vf = workloads.vortex(1024, 64.0, mv, ma, angle=0.6)
            with pond.Sim(1024, 1024, pond.POND_FP32_MIXED, stream=stream.cuda_stream,
                          use_graph=1, autotune=1) as vsim:
                vsim.set_state(vf.rho, vf.ux, vf.uy, vf.T)
                vsim.step(args.warmup)
                vsecs, vstats = time_steps(vsim, stream, k2)
            line_v = form_line("vortex-1024-mixed", 1024 * 1024, k2, vsecs, vstats, peak32,
                               BYTES_MIXED,
                               staged_flops_per_pass(4, float(np.sqrt(vf.T).mean()), every_row=True))
            vortex["Ma_a=%g,Ma_v=%g" % (ma, mv)] = {
                k: line_v[k] for k in ("value", "ms_per_step", "mean_passes", "max_passes",
                                       "nonconverged", "halo_fallback", "alu_frac", "tile")}
        forms["vortex_mixed_1024"] = {"workload": "vortex-1024-mixed", "unit": UNIT,
                                      "radius": 64.0, "steps": k2, "sweep": vortex}

        # adjoint / forward time on the 512^2 Taylor-Green + pulse workload.
        # One short rollout with its backward runs first, untimed, so that
        # one-time costs (first launches of the adjoint kernels and of
        # torch's own loss kernels, first allocations) stay out of both
        # legs.  The forward leg is the rollout call alone; the backward leg
        # is the loss and its backward (segment recompute + adjoint steps).
        from paper_1806_05089_gb300.autograd import pond_rollout
        af, target = workloads.adjoint(512)
        dev = torch.device("cuda", local)
        gauge = [torch.tensor(a, device=dev) for a in (af.ux, af.uy, af.T)]
        tgt = torch.tensor(target, device=dev)

        def rollout_times(precision):
            for steps, timed in ((4, False), (200, True)):
                r = torch.tensor(af.rho, device=dev, requires_grad=True)
                n = torch.tensor(0.01, dtype=torch.float64, device=dev, requires_grad=True)
                torch.cuda.synchronize()
                t0 = time.perf_counter()
                rho = pond_rollout(r, n, *gauge, steps, 20 if timed else 2, precision=precision)
                torch.cuda.synchronize()
                t1 = time.perf_counter()
                loss = 0.5 * ((rho - tgt) ** 2).sum()
                loss.backward()
                torch.cuda.synchronize()
                t2 = time.perf_counter()
            return r, n, loss, t1 - t0, t2 - t1

        r, n, loss, fwd, bwd = rollout_times(pond.POND_FP64)
        forms["adjoint_512"] = {"workload": "adjoint-512-fp64", "steps": 200, "ckpt_every": 20,
                                "forward_s": fwd, "backward_s": bwd,
                                "adjoint_over_forward": bwd / fwd,
                                "nu_grad": float(n.grad), "loss": float(loss.detach())}
        g64 = r.grad.detach().clone()
        nu64 = float(n.grad)
        r32, n32, loss32, fwd32, bwd32 = rollout_times(pond.POND_FP32_MIXED)
        forms["adjoint_512_mixed"] = {
            "workload": "adjoint-512-mixed", "steps": 200, "ckpt_every": 20,
            "forward_s": fwd32, "backward_s": bwd32,
            "adjoint_over_forward": bwd32 / fwd32,
            "grad_rel_err_vs_fp64": float((r32.grad - g64).abs().max() / g64.abs().max()),
            "grad_max_abs": [float(g64.abs().max()), float(r32.grad.abs().max())],
            "nu_grad_rel_err_vs_fp64": abs(float(n32.grad) - nu64) / abs(nu64),
            "backward_speedup_vs_fp64": bwd / bwd32}

        # moment error of the mixed form against the FP64 step after 1000
        # steps on the temperature-ratio-4 precision field at 4096^2 (the
        # FP64 reference takes ~6 min); --precision-quick runs the same
        # field recipe at 2048^2 (steeper gradients per cell, so no easier).
        pn = 2048 if args.precision_quick else 4096
        pstate = workloads.precision(pn)
        res = {}
        for prec in (pond.POND_FP64, pond.POND_FP32_MIXED):
            extra = {"use_graph": 1, "autotune": 1}
            with pond.Sim(pn, pn, prec, stream=stream.cuda_stream, **extra) as ps:
                ps.set_state(pstate.rho, pstate.ux, pstate.uy, pstate.T)
                ev = time_steps(ps, stream, args.precision_steps)
                res[prec] = (ps.moments(), ev)
        (r64_, x64_, y64_, t64_), (s64, st64) = res[pond.POND_FP64]
        (r32_, x32_, y32_, t32_), (s32, st32) = res[pond.POND_FP32_MIXED]
        forms["precision_%d_%dsteps" % (pn, args.precision_steps)] = {
            "workload": "precision-%d" % pn, "steps": args.precision_steps,
            "rho": float(np.max(np.abs(r32_ - r64_) / r64_)),
            "u": float(max(np.abs(x32_ - x64_).max(), np.abs(y32_ - y64_).max())
                       / np.hypot(x64_, y64_).max()),
            "T": float(np.max(np.abs(t32_ - t64_) / t64_)),
            "bound": 1e-5,
            "fp64_s": s64, "mixed_s": s32,
            "speedup_mixed_vs_fp64": s64 / s32,
            "mean_passes": [st64["passes"] / st64["node_updates"],
                            st32["passes"] / st32["node_updates"]],
            "nonconverged": [st64["nonconverged"], st32["nonconverged"]],
            "error_definition": "max over nodes: |d rho|/rho, |d u|/max|u_fp64|, |d T|/T"}
        pkey = "precision_%d_%dsteps" % (pn, args.precision_steps)
        forms["fp32_mixed_4096"]["moment_err_vs_fp64"] = {
            "after_steps": args.precision_steps, "grid": "%dx%d" % (pn, pn),
            "rho": forms[pkey]["rho"], "u": forms[pkey]["u"], "T": forms[pkey]["T"],
            "see": pkey}
        del pstate, res
        line["forms"] = forms

    # ---- CPU oracle on a bounded sample (rank 0, N = 1)
    if rank == 0 and world == 1 and not args.no_cpu:
        line["cpu_baseline"] = oracle_sample(fields, args.cpu_seconds)
    if rank == 0:
        print(json.dumps(line), flush=True)


def main():
    args = parse()
    world, rank, local = dist_setup()
    if args.impl == "reference":
        run_reference(args, world, rank)
    else:
        run_pond(args, world, rank, local)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
