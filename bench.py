#!/usr/bin/env python
"""Throughput of the radial-line 3D NUFFT projector (forward + adjoint).

Metric: nonuniform points per second, P / (t_forward + t_adjoint), on the
256^3 workload (K = 512, J = 6, 360 x 256 umbrella lines of 512 samples:
P = 47,185,920 points) with a seeded ellipsoid phantom plus N(0, 0.01^2)
noise.  A step is one forward projection of the volume followed by the
adjoint of the resulting lines.  The min-max coefficients are the exact ones
at every point (--coeffs exact, the default; the oracle's per-point solve is
its reference) or linearly interpolated from the L = 1024 table
(--coeffs table).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Multi-GPU (torchrun, one rank per GPU): every rank runs an independent replica
of the workload (the projector does not shard across GPUs here); the value is
the points of all ranks over the slowest rank's time ("scaling": "weak").
The reference arm times the FP64 CPU oracle on the host cores on a bounded
sample of the same workload (rank 0 only).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "nonuniform pts/s fwd+adj NUFFT at 256^3 FP32"
UNIT = "pts/s"
FP32_LANES_PER_SM = 128   # FP32 FMA lanes per SM (nominal; the peak itself is measured)
SMEM_BYTES_PER_CLK = 128  # shared-memory data path per SM and clock


def parse_args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=50)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="full256")
    ap.add_argument("--grid-dtype", default="c64")
    ap.add_argument("--gather-variant", type=int, default=-1)
    ap.add_argument("--spread-variant", type=int, default=-1)
    ap.add_argument("--points-per-subproblem", type=int, default=0)
    ap.add_argument("--tile-edge", type=int, default=0)
    ap.add_argument("--keep-duplicates", action="store_true")
    ap.add_argument("--coeffs", default="exact", choices=["table", "exact"],
                    help="min-max coefficients from the L = 1024 table, or exact per point (fitted polynomials)")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-fft-compare", action="store_true", help="skip the cuFFT comparison")
    ap.add_argument("--no-extras", action="store_true",
                    help="skip the reduced-precision, keep-duplicates and batch24 measurements beside the headline")
    ap.add_argument("--cpu-sample-lines", type=int, default=0,
                    help="lines of the CPU oracle sample (0: sized for about 20 s of CPU work)")
    return ap.parse_args()


# ----------------------------------------------------------------------------
# clocks
# ----------------------------------------------------------------------------
CLOCK_QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
               "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
               "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")


class ClockSampler:
    def __init__(self, device_index: int):
        self.dev = device_index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.dev), f"--query-gpu={CLOCK_QUERY}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=self.fh, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["clock sampling unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.fh.close()
        with open(self.path) as fh:
            out = parse_clocks(fh.readlines())
        os.unlink(self.path)
        return out


def parse_clocks(lines):
    """Median SM clock, max clock and active throttle reasons from nvidia-smi
    CSV lines (noheader, nounits) of the CLOCK_QUERY fields."""
    sm, smax, reasons = [], [], set()
    names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
    for line in lines:
        parts = [p.strip() for p in line.split(",")]
        if len(parts) < 9:
            continue
        try:
            sm.append(float(parts[1]))
            smax.append(float(parts[2]))
        except ValueError:
            continue
        for name, v in zip(names, parts[5:9]):
            if v.lower().startswith("active"):
                reasons.add(name)
    return {"sm_mhz": statistics.median(sm) if sm else None,
            "sm_max_mhz": max(smax) if smax else None,
            "reasons": sorted(reasons), "samples": len(sm)}


# ----------------------------------------------------------------------------
# roofline bookkeeping: algorithmic work per stage
# ----------------------------------------------------------------------------
def stage_work(n, k, j, m, d, p_eval=None, spread_tap_bytes=16):
    """Algorithmic bytes and flops per launch of each stage: every stage moves
    its input and output arrays once; the interpolation does 8 (J^3 + J^2 + J)
    flops per evaluated point (coincident samples are evaluated once) and reads
    the touched part of the grid (the ball |k| <= K/2 + J/2).  Shared-memory
    bytes per tap: 8 for the gather's read, 16 for the FP32 spread's
    read-modify-write, 8 for the fixed-point spread's two 4-byte reductions."""
    P = d * m
    Pe = P if p_eval is None else p_eval
    c8 = 8
    ball = min(1.0, 4.0 / 3.0 * 3.141592653589793 * (0.5 + (j / 2) / k) ** 3)
    interp_flops = 8 * (j ** 3 + j ** 2 + j) * Pe
    return {
        "forward": {
            "x_pass": {"bytes": 4 * n ** 3 + c8 * n * n * k},
            "y_pass": {"bytes": c8 * n * n * k + c8 * n * k * k},
            "z_pass": {"bytes": c8 * n * k * k + c8 * k ** 3},
            "gather": {"bytes": ball * c8 * k ** 3 + c8 * P + 8 * Pe, "flops": interp_flops,
                       "smem_bytes": j ** 3 * 8 * Pe},
            "line_dft": {"bytes": 2 * c8 * P},
        },
        "adjoint": {
            "line_dft": {"bytes": 2 * c8 * P},
            "grid_clear": {"bytes": c8 * k ** 3},
            "spread": {"bytes": 2 * ball * c8 * k ** 3 + c8 * P + 8 * Pe, "flops": interp_flops,
                       "smem_bytes": j ** 3 * spread_tap_bytes * Pe},
            "z_pass": {"bytes": c8 * k ** 3 + c8 * n * k * k},
            "y_pass": {"bytes": c8 * n * k * k + c8 * n * n * k},
            "x_pass": {"bytes": c8 * n * n * k + 4 * n ** 3},
        },
    }


def cufft_compare(K: int, D: int, M: int, dev, reps: int = 10):
    """Milliseconds of cuFFT (through torch.fft) on resident complex64 data of
    the workload's shapes, event-timed: the K^3 forward and inverse transforms
    and the batch of D line transforms of length M."""
    import torch

    s = torch.cuda.current_stream(dev)
    out = {}

    def timed(fn, x):
        for _ in range(3):
            fn(x)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(s)
        for _ in range(reps):
            fn(x)
        e1.record(s)
        e1.synchronize()
        return round(e0.elapsed_time(e1) / reps, 4)

    g = torch.randn((K, K, K), dtype=torch.complex64, device=dev)
    out["cufft_fftn_ms"] = timed(torch.fft.fftn, g)
    out["cufft_ifftn_ms"] = timed(torch.fft.ifftn, g)
    del g
    lines = torch.randn((D, M), dtype=torch.complex64, device=dev)
    out["cufft_lines_ifft_ms"] = timed(lambda x: torch.fft.ifft(x, dim=1), lines)
    del lines
    torch.cuda.empty_cache()
    return out


def load_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as fh:
            pk = json.load(fh)
        return {"hbm_gbs": float(pk["hbm_gbs"]), "sm_max_mhz": float(pk.get("sm_max_mhz", 2070.0)),
                "source": "measured"}
    except Exception:
        return {"hbm_gbs": 6800.0, "sm_max_mhz": 2070.0, "source": "fallback"}


INTERP_SOURCES = ("interp_common.cuh", "interp_gather.cu", "interp_spread.cu", "interp_tma.cu", "interp_real.cu",
                  "common.cuh")


def source_hash(files=INTERP_SOURCES) -> str:
    h = hashlib.sha256()
    for fn in files:
        with open(os.path.join(ROOT, "paper_1605_05231_gb300", "csrc", fn), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def ncu_traffic(kernel_stage: str, files=INTERP_SOURCES):
    """DRAM bytes per launch from a committed ncu summary, if the kernel source
    is unchanged since the capture (else None)."""
    path = os.path.join(ROOT, "profiles", "ncu_traffic.json")
    try:
        with open(path) as fh:
            tr = json.load(fh)
        ent = tr.get(kernel_stage)
        if ent and ent.get("source_hash") == source_hash(files):
            return float(ent["dram_bytes_per_launch"])
    except Exception:
        pass
    return None


# ----------------------------------------------------------------------------
# distributed helpers
# ----------------------------------------------------------------------------
def dist_setup(args):
    import torch

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist

        if args.impl == "ours":
            torch.cuda.set_device(local)
            dist.init_process_group("nccl")
        else:
            dist.init_process_group("gloo")
    elif args.impl == "ours":
        torch.cuda.set_device(0)
    return world, rank, local


def barrier(world):
    if world > 1:
        import torch.distributed as dist

        dist.barrier()


def max_over_ranks(world, v: float) -> float:
    """Maximum of v over all ranks (NCCL on the GPU, gloo on the host)."""
    if world == 1:
        return v
    import torch
    import torch.distributed as dist

    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([v], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


# ----------------------------------------------------------------------------
# CPU oracle timing (cpu_baseline and the reference arm)
# ----------------------------------------------------------------------------
def bench_workload(args):
    """The named workload; --coeffs exact selects exact per-point coefficients
    (table_oversamp 0, the oracle's L = 0 variant)."""
    import dataclasses

    from paper_1605_05231_gb300 import inputs as I

    w = I.workload(args.workload)
    return dataclasses.replace(w, table_oversamp=0) if args.coeffs == "exact" else w


def bench_config(w, args, world=1):
    """The workload description shared by both arms (no implementation keys)."""
    return {"workload": w.name, "n": w.n, "k": w.k, "j": w.j, "coefficients": coeff_desc(w),
            "dirs": f"{w.n_az}x{w.n_pol}", "m": w.m, "points": w.n_points, "grid_dtype": args.grid_dtype,
            "parallelism": "replicas" if world > 1 else "single",
            "l2": "working set per step >> L2 (1.07 GB grid, 0.38 GB lines, 0.19 GB point ids)"}


def coeff_desc(w, info=None, oracle=False):
    if w.table_oversamp:
        return f"table, L = {w.table_oversamp}, linear interpolation"
    if oracle:
        return "exact min-max per point (FP64 solve of T c = r at every point)"
    if info:
        return f"exact min-max per point (degree-8 polynomials fitted in FP64, fit error {info['coeff_fit_error']:.1e} of max|c|)"
    return "exact min-max per point"


def oracle_fixed(w, x, dirs):
    """Time the oracle's size-fixed stages at full size: deapodise + pad + K^3
    FFT (forward) and K^3 inverse FFT + crop + deapodise (adjoint)."""
    import numpy as np

    from oracle import nufft3d_oracle as O

    op = O.OraclePlan(w.n, w.k, w.j, w.table_oversamp, dirs, w.m)
    t0 = time.perf_counter()
    Y = O.grid_fft(O.deapodize_pad(x.astype(np.float64), op))
    t1 = time.perf_counter()
    O.crop_deapodize(O.grid_ifft_unnormalised(Y), op)
    t2 = time.perf_counter()
    return op, Y, t2 - t0


def oracle_points(op, Y, lines):
    """Time the oracle's per-point stages (gather + line DFT, line DFT adjoint +
    spread) on the selected lines."""
    from oracle import nufft3d_oracle as O

    t0 = time.perf_counter()
    u = op.point_u(lines).reshape(-1, 3)
    Xh = O.interp_gather(Y, u, op).reshape(len(lines), op.M)
    p = O.radial_idft(Xh, op, lines)
    Yh = O.radial_idft_adjoint(p, op, lines)
    O.interp_spread(Yh.reshape(-1), u, op)
    return time.perf_counter() - t0


def oracle_time(w, x, dirs, sample_lines: int, seed: int = 0, target_s: float = 20.0):
    """Oracle time for the whole workload: the fixed stages at full size plus
    the per-point stages on a sample of lines scaled to all points.  With
    sample_lines = 0 the sample is sized from a 4-line pilot to take about
    target_s seconds."""
    import numpy as np

    t0 = time.perf_counter()
    op, Y, t_fixed = oracle_fixed(w, x, dirs)
    rng = np.random.default_rng(seed)
    if sample_lines <= 0:
        t_pilot = oracle_points(op, Y, np.sort(rng.choice(dirs.shape[0], 4, replace=False)))
        sample_lines = int(min(dirs.shape[0], max(4, 4 * target_s / max(t_pilot, 1e-6))))
    lines = np.sort(rng.choice(dirs.shape[0], sample_lines, replace=False))
    t_pts = oracle_points(op, Y, lines)
    P = dirs.shape[0] * w.m
    Ps = len(lines) * w.m
    return {"t_total": t_fixed + t_pts * P / Ps, "t_fixed": t_fixed, "t_points_sample": t_pts,
            "sample_points": Ps, "sample_lines": len(lines), "wall": time.perf_counter() - t0}


def cpu_cores():
    try:
        return len(os.sched_getaffinity(0))
    except Exception:
        return os.cpu_count()


# ----------------------------------------------------------------------------
# arms
# ----------------------------------------------------------------------------
def run_reference(args):
    """The FP64 oracle on the host cores.  Each step runs the oracle's
    size-fixed stages at full size (deapodise + pad + K^3 FFT, K^3 inverse FFT +
    crop + deapodise) and its per-point stages (gather, line DFTs, spread) on 8
    random lines of the 92,160, all measured; the value projects those measured
    times to the whole workload (fixed stages once, per-point stages for every
    line)."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    import numpy as np

    w = bench_workload(args)
    dirs = w.directions()
    x = w.volume(np.float32)
    per_step_lines = 8
    rng = np.random.default_rng(0)

    def one_step():
        op, Y, tf = oracle_fixed(w, x, dirs)
        tp = oracle_points(op, Y, np.sort(rng.choice(dirs.shape[0], per_step_lines, replace=False)))
        return tf, tp

    for _ in range(args.warmup):
        one_step()
    t_fixed, t_pts = [], []
    t0 = time.perf_counter()
    for _ in range(args.steps):
        tf, tp = one_step()
        t_fixed.append(tf)
        t_pts.append(tp)
    wall = time.perf_counter() - t0
    P = w.n_points
    tf, tp = statistics.mean(t_fixed), statistics.mean(t_pts)
    t_full = tf + tp * dirs.shape[0] / per_step_lines
    value = P / t_full
    sample = (f"each step: the FP64 oracle's K^3 FFT + inverse FFT at full size ({tf:.2f} s) and its gather, "
              f"spread and line DFTs on {per_step_lines} random lines of {dirs.shape[0]} "
              f"({per_step_lines * w.m} points, {tp:.2f} s); value = all {P} points over the fixed stages plus "
              f"the per-point time scaled to every line ({t_full:.0f} s projected)")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * wall / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": bench_config(w, args),
            "measured": {"ms_per_step": 1e3 * wall / args.steps, "fixed_stages_s": tf,
                         "per_point_stages_s": tp, "points_per_step": per_step_lines * w.m,
                         "timed_region_s": wall},
            "projected": {"full_workload_s": t_full, "basis": "fixed stages once + per-point stages x "
                          f"{dirs.shape[0]}/{per_step_lines}"},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cpu_cores(), "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def run_ours(args):
    import numpy as np
    import torch

    from paper_1605_05231_gb300 import Plan
    from paper_1605_05231_gb300 import inputs as I

    world, rank, local = dist_setup(args)
    dev = torch.device("cuda", torch.cuda.current_device())
    w = bench_workload(args)
    dirs = w.directions()
    x = w.volume(np.float32)
    t0 = time.perf_counter()
    plan = Plan(w.n, dirs, m=w.m, k=w.k, j=w.j, table_oversamp=w.table_oversamp or 1024,
                exact_coeffs=w.table_oversamp == 0, grid_dtype=args.grid_dtype,
                keep_duplicates=args.keep_duplicates)
    plan.tune(args.gather_variant, args.spread_variant, args.points_per_subproblem, args.tile_edge)
    torch.cuda.synchronize()
    plan_s = time.perf_counter() - t0
    P = plan.n_points
    xd = torch.from_numpy(x).to(dev)
    lines = torch.empty((plan.n_dirs, plan.m), dtype=torch.complex64, device=dev)
    vout = torch.empty_like(xd)
    stream = torch.cuda.current_stream(dev)

    def step():
        plan.forward(xd, out=lines)
        plan.adjoint(lines, out=vout)

    for _ in range(max(args.warmup, 3)):
        step()
    torch.cuda.synchronize()
    if plan.sync_status() != 0:
        raise RuntimeError("device check failed during warm-up")
    plan.set_timing(args.steps)
    clocks = ClockSampler(dev.index)
    barrier(world)
    torch.cuda.synchronize()
    clocks.start()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    for _ in range(args.steps):
        step()
    ev1.record(stream)
    torch.cuda.synchronize()
    barrier(world)
    clk = clocks.stop()
    ms = ev0.elapsed_time(ev1) / args.steps
    stages = plan.stage_times()
    plan.set_timing(0)
    ms_max = max_over_ranks(world, ms)
    value = world * P / (ms_max * 1e-3)

    # ---- end to end: host buffers through the library's host pipeline ----
    e2e = None
    if not args.no_e2e:
        from paper_1605_05231_gb300 import HostPipeline

        xh = torch.from_numpy(x).pin_memory()
        lh = torch.empty((plan.n_dirs, plan.m), dtype=torch.complex64).pin_memory()
        vh = torch.empty_like(xh).pin_memory()
        pipe = HostPipeline(plan)
        for _ in range(3):
            pipe.run(xh, lh, vh)
        pipe.synchronize()
        if float((lh[:4].abs()).max()) == 0.0:
            raise RuntimeError("host pipeline returned empty lines")
        n_e2e = max(3, min(args.steps, 20))
        barrier(world)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(n_e2e):
            pipe.run(xh, lh, vh)
        pipe.synchronize()
        ms_e2e = max_over_ranks(world, (time.perf_counter() - t0) * 1e3 / n_e2e)
        e2e = {"value": world * P / (ms_e2e * 1e-3), "unit": UNIT,
               "h2d_bytes_per_step": int(xh.numel() * 4),
               "d2h_bytes_per_step": int(lh.numel() * 8 + vh.numel() * 4), "ms_per_step": ms_e2e,
               "copies": ("pinned host buffers through the C ABI (nufft3d_host_forward_adjoint): the library "
                          "copies the volume in and the lines and output volume out on its own streams, "
                          "overlapped with the kernels of the neighbouring calls"),
               "timer": "host wall clock around the enqueue loop and the final nufft3d_host_pipeline_sync"}
        pipe.close()
    if plan.sync_status() != 0:
        raise RuntimeError("device check failed")

    # ---- roofline of the dominant kernel ---------------------------------
    peaks = load_peaks()
    info = plan.info()
    from paper_1605_05231_gb300 import fp32_fma_peak

    fp32_tflops, sms = fp32_fma_peak()
    fixed_point = info["spread_variant"] in (5, 6, 7, 8)
    work = stage_work(w.n, w.k, w.j, w.m, plan.n_dirs, info["evaluated_points"], 8 if fixed_point else 16)
    per_call = {}
    for side in ("forward", "adjoint"):
        calls = max(1, stages[f"{side}_calls"])
        for name, t in stages[side].items():
            per_call[(side, name)] = t / calls
    dom = max(per_call, key=per_call.get)
    t_dom = per_call[dom] * 1e-3
    wk = work[dom[0]][dom[1]]
    f_mhz = peaks["sm_max_mhz"]
    if "flops" in wk:
        nominal = sms * FP32_LANES_PER_SM * 2 * f_mhz * 1e6 / 1e12
        achieved = wk["flops"] / t_dom / 1e12
        roof = {"bound": "alu", "achieved": achieved, "peak": fp32_tflops, "unit": "TFLOP/s",
                "frac": achieved / fp32_tflops, "kernel": f"{dom[0]}.{dom[1]}",
                "peak_source": "measured (FP32 FMA microbenchmark, nufft3d_fp32_fma_peak, this run)",
                "peak_nominal": nominal,
                "peak_nominal_basis": f"{sms} SMs (device attribute) x {FP32_LANES_PER_SM} lanes x 2 x {f_mhz:.0f} MHz",
                "flops_basis": "8 (J^3 + J^2 + J) flops per evaluated point"}
    else:
        achieved = wk["bytes"] / t_dom / 1e9
        roof = {"bound": "hbm", "achieved": achieved, "peak": peaks["hbm_gbs"], "unit": "GB/s",
                "frac": achieved / peaks["hbm_gbs"], "kernel": f"{dom[0]}.{dom[1]}",
                "peak_source": peaks["source"]}
    if "smem_bytes" in wk:
        smem_peak = sms * SMEM_BYTES_PER_CLK * f_mhz * 1e6 / 1e12
        roof["smem_frac"] = wk["smem_bytes"] / t_dom / 1e12 / smem_peak
        roof["smem_basis"] = (f"shared-memory data path (derived, not measured): {sms} SMs x "
                              f"{SMEM_BYTES_PER_CLK} B/clk x {f_mhz:.0f} MHz = {smem_peak:.1f} TB/s; per evaluated "
                              f"point J^3 x 8 B (gather, fixed-point spread) or x 16 B (FP32 spread)")
    # the other interpolation kernel, in the same terms
    other = ("forward", "gather") if dom == ("adjoint", "spread") else ("adjoint", "spread")
    if other in per_call and "flops" in work[other[0]][other[1]]:
        wo = work[other[0]][other[1]]
        to = per_call[other] * 1e-3
        roof["other_interp"] = {"kernel": f"{other[0]}.{other[1]}", "ms": per_call[other],
                                "alu_frac": wo["flops"] / to / 1e12 / fp32_tflops,
                                "smem_frac": wo["smem_bytes"] / to / 1e12 /
                                (sms * SMEM_BYTES_PER_CLK * f_mhz * 1e6 / 1e12),
                                "hbm_frac": wo["bytes"] / to / 1e9 / peaks["hbm_gbs"]}
    roof["algorithmic_bytes"] = wk["bytes"]
    roof["hbm_frac"] = wk["bytes"] / t_dom / 1e9 / peaks["hbm_gbs"]
    roof["traffic"] = ncu_traffic(f"{dom[0]}.{dom[1]}")
    stage_ms = {f"{side}.{name}": round(per_call[(side, name)], 4) for (side, name) in per_call}

    # ---- cuFFT on the same grid, timed only as a comparison --------------
    fft_cmp = None
    if not args.no_fft_compare:
        fft_cmp = cufft_compare(w.k, plan.n_dirs, w.m, dev)
        fft_cmp["ours_forward_ms"] = round(sum(per_call[("forward", s)] for s in ("x_pass", "y_pass", "z_pass")), 4)
        fft_cmp["ours_inverse_ms"] = round(sum(per_call[("adjoint", s)] for s in ("z_pass", "y_pass", "x_pass")), 4)
        fft_cmp["ours_line_dft_ms"] = round(per_call[("forward", "line_dft")], 4)
        fft_cmp["note"] = ("ours: the pruned 3D transform with the zero padding / cropping and the deapodisation "
                           "fused (x, y, z passes), and the centred weighted line DFT; cuFFT: a full "
                           "complex-to-complex K^3 transform of a resident grid and a plain batched line "
                           "transform (torch.fft), nothing fused")

    # ---- CPU oracle baseline (rank 0, N = 1) ----------------------------
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        r = oracle_time(w, x, dirs, args.cpu_sample_lines)
        cpu = {"value": P / r["t_total"], "unit": UNIT, "cores": cpu_cores(), "kind": "oracle",
               "sample": (f"full-size K^3 FFT + inverse FFT of the FP64 oracle, its gather, spread and line DFTs "
                          f"on {r['sample_lines']} of {plan.n_dirs} lines ({r['sample_points']} points), "
                          f"per-point time scaled to all {P} points; {r['wall']:.1f} s of CPU work")}

    plan.close()
    extras = None
    if rank == 0 and world == 1 and not args.no_extras and args.workload == "full256":
        del xd, lines, vout
        torch.cuda.empty_cache()
        extras = run_extras(args, w, dirs, x, dev)

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": ms_max, "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": "f32" if args.grid_dtype == "c64" else f"f32+{args.grid_dtype} grid",
                "data": "synthetic", "config": bench_config(w, args, world),
                "plan": {"coefficients": coeff_desc(w, info), "variants": info, "plan_s": plan_s},
                "gpu_launches": 10 * args.steps, "clocks": clk, "e2e": e2e, "roofline": roof,
                "cpu_baseline": cpu, "stage_ms": stage_ms, "cufft_comparison": fft_cmp,
                "fp32_fma_peak_tflops": fp32_tflops, "sm_count": sms}
        if extras:
            line.update(extras)
        print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist

        dist.destroy_process_group()
    return 0


def time_steps(fn, steps, warmup, stream):
    """Milliseconds per call of fn, CUDA events on `stream` after warm-up."""
    import torch

    for _ in range(warmup):
        fn()
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(steps):
        fn()
    e1.record(stream)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / steps


def batch_one_by_one(b, vols, lines, outs, steps, stream):
    """The batch's items run one after another on one stream through each
    plan's own forward and adjoint calls (same plans and tuned kernels, no
    graph, no overlap between items), all of them and each problem size
    alone: what the one-graph batch is compared with."""
    def run(idx):
        for i in idx:
            b.items[i].forward(vols[i], out=lines[i])
            b.items[i].adjoint(lines[i], out=outs[i])

    every = list(range(len(b.items)))
    ms = time_steps(lambda: run(every), steps, 3, stream)
    by_size = {}
    for n in sorted({p.n for p in b.items}):
        idx = [i for i, p in enumerate(b.items) if p.n == n]
        ms_n = time_steps(lambda: run(idx), steps, 2, stream)
        pts = sum(b.items[i].n_points for i in idx)
        by_size[f"{n}^3"] = {"items": len(idx), "ms_per_step": ms_n, "value": pts / (ms_n * 1e-3)}
    pts = sum(p.n_points for p in b.items)
    return {"value": pts / (ms * 1e-3), "unit": UNIT, "ms_per_step": ms, "by_size": by_size}


def run_extras(args, w, dirs, x, dev, steps=10):
    """The forms reported beside the FP32 headline, on the same 256^3 workload
    and coefficients: the bf16 and fp16 grid storage (throughput, and rel-L2
    of the forward against the FP64 oracle on 64 seeded random lines), every
    sample interpolated separately (keep_duplicates = 1), and the 24-problem
    batch in one CUDA graph (throughput, worst per-item forward rel-L2 against
    the oracle on 8 lines per item)."""
    import numpy as np
    import torch

    from oracle import nufft3d_oracle as O
    from paper_1605_05231_gb300 import Batch, Plan, autotune
    from paper_1605_05231_gb300 import inputs as I

    stream = torch.cuda.current_stream(dev)
    out = {}
    exact = w.table_oversamp == 0
    xd = torch.from_numpy(x).to(dev)
    lines = np.sort(np.random.default_rng(7).choice(dirs.shape[0], 64, replace=False))
    op = O.OraclePlan(w.n, w.k, w.j, w.table_oversamp, dirs, w.m)
    ref = O.nufft_forward(x.astype(np.float64), op, lines=lines)

    def measure(**kw):
        plan = Plan(w.n, dirs, m=w.m, k=w.k, j=w.j, table_oversamp=w.table_oversamp or 1024,
                    exact_coeffs=exact, **kw)
        lb = torch.empty((plan.n_dirs, plan.m), dtype=torch.complex64, device=dev)
        vb = torch.empty_like(xd)

        def step():
            plan.forward(xd, out=lb)
            plan.adjoint(lb, out=vb)

        ms = time_steps(step, steps, 3, stream)
        plan.forward(xd, out=lb)
        if plan.sync_status() != 0:
            raise RuntimeError("device check failed")
        err = O.rel_l2(lb.cpu().numpy()[lines], ref)
        info = plan.info()
        plan.close()
        return {"value": plan.n_points / (ms * 1e-3), "unit": UNIT, "ms_per_step": ms, "steps": steps,
                "fwd_rel_l2_vs_oracle_64_lines": err, "evaluated_points": info["evaluated_points"]}

    rp = {}
    for dt, bar in (("bf16", 1e-4), ("fp16", 1e-4)):
        r = measure(grid_dtype=dt)
        r["bar"] = bar
        r["meets_bar"] = bool(r["fwd_rel_l2_vs_oracle_64_lines"] <= bar)
        rp[dt] = r
    rp["note"] = ("forward grid stored as bf16 / fp16 pairs with a power-of-two scale, FP32 arithmetic; the "
                  "adjoint stays FP32.  bf16 (unit roundoff 2^-8) misses the 1e-4 bar by its storage rounding")
    out["reduced_precision"] = rp
    kd = measure(keep_duplicates=True)
    kd["note"] = ("every one of the 47,185,920 samples interpolated separately (coincident antipodal samples "
                  "not merged); value counts samples per second, as the headline does")
    out["keep_duplicates"] = kd
    del xd
    torch.cuda.empty_cache()

    # 24 mixed problems in one CUDA graph
    works = I.batched_workloads()
    items = [dict(n=v.n, dirs=v.directions(), m=v.m, k=v.k, j=v.j, table_oversamp=v.table_oversamp,
                  exact_coeffs=exact) for v in works]
    t0 = time.perf_counter()
    b = Batch(items)
    tuned = autotune.tune_batch(b, reps=2, cache=None)
    plan_s = time.perf_counter() - t0
    vols = [torch.from_numpy(v.volume(np.float32)).to(dev) for v in works]
    lns = [torch.empty((p.n_dirs, p.m), dtype=torch.complex64, device=dev) for p in b.items]
    outs = [torch.empty_like(v) for v in vols]
    ms = time_steps(lambda: b.forward_adjoint(vols, lns, outs), steps, 3, stream)
    worst = 0.0
    for i, v in enumerate(works):
        if b.items[i].sync_status() != 0:
            raise RuntimeError("device check failed in the batch")
        dv = v.directions()
        sel = np.sort(np.random.default_rng(1000 + i).choice(dv.shape[0], 8, replace=False))
        o = O.OraclePlan(v.n, v.k, v.j, v.table_oversamp if not exact else 0, dv, v.m)
        r = O.nufft_forward(vols[i].cpu().numpy().astype(np.float64), o, lines=sel)
        worst = max(worst, O.rel_l2(lns[i].cpu().numpy()[sel], r))
    Pb = sum(p.n_points for p in b.items)
    out["batch24"] = {"value": Pb / (ms * 1e-3), "unit": UNIT, "ms_per_step": ms, "steps": steps,
                      "points": Pb, "worst_item_fwd_rel_l2_vs_oracle_8_lines": worst, "plan_and_tune_s": plan_s,
                      "items": "8 each at 64^3, 128^3, 192^3, K = M = 2N, azimuths {90,180,360} x polar {64,128}",
                      "autotune": {k: v["best"] for k, v in tuned.items()},
                      "items_one_by_one": batch_one_by_one(b, vols, lns, outs, steps, stream)}
    b.close()
    torch.cuda.empty_cache()
    return out


def run_batch(args):
    """24 mixed problems (8 each at 64^3, 128^3, 192^3) as one CUDA-graph replay
    per step, kernel choices from the autotuner."""
    import numpy as np
    import torch

    from paper_1605_05231_gb300 import Batch, autotune
    from paper_1605_05231_gb300 import inputs as I

    world, rank, local = dist_setup(args)
    dev = torch.device("cuda", torch.cuda.current_device())
    works = I.batched_workloads()
    items = [dict(n=w.n, dirs=w.directions(), m=w.m, k=w.k, j=w.j, table_oversamp=w.table_oversamp,
                  exact_coeffs=args.coeffs == "exact") for w in works]
    t0 = time.perf_counter()
    b = Batch(items)
    tuned = autotune.tune_batch(b, reps=2, cache=None)
    plan_s = time.perf_counter() - t0
    vols = [torch.from_numpy(w.volume(np.float32)).to(dev) for w in works]
    lines = [torch.empty((p.n_dirs, p.m), dtype=torch.complex64, device=dev) for p in b.items]
    outs = [torch.empty_like(v) for v in vols]
    P = sum(p.n_points for p in b.items)
    for _ in range(max(args.warmup, 3)):
        b.forward_adjoint(vols, lines, outs)
    torch.cuda.synchronize()
    stream = torch.cuda.current_stream(dev)
    clocks = ClockSampler(dev.index)
    barrier(world)
    torch.cuda.synchronize()
    clocks.start()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    for _ in range(args.steps):
        b.forward_adjoint(vols, lines, outs)
    ev1.record(stream)
    torch.cuda.synchronize()
    barrier(world)
    clk = clocks.stop()
    ms = max_over_ranks(world, ev0.elapsed_time(ev1) / args.steps)
    for p in b.items:
        if p.sync_status() != 0:
            raise RuntimeError("device check failed")
    seq = batch_one_by_one(b, vols, lines, outs, max(3, min(args.steps, 10)), stream)
    if rank == 0:
        line = {"metric": "nonuniform pts/s fwd+adj NUFFT, 24 mixed problems in one CUDA graph",
                "value": world * P / (ms * 1e-3), "unit": UNIT, "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": "f32", "data": "synthetic",
                "config": {"workload": "batch24", "items": [f"{w.n}^3 {w.n_az}x{w.n_pol}x{w.m}" for w in works],
                           "coefficients": "exact min-max per point" if args.coeffs == "exact" else "table, L = 1024",
                           "points": P, "graph_launches_per_step": 1},
                "clocks": clk, "autotune": {k: v["best"] for k, v in tuned.items()}, "plan_s": plan_s,
                "items_one_by_one": seq}
        print(json.dumps(line), flush=True)
    b.close()
    return 0


RESAMPLE_SHIFT = (0.37, 0.21, 0.43)
RESAMPLE_SOURCES = ("polar_resample.cu",)


def run_resample(args):
    """Direct resampling of the polar Radon grid (Eq. 2.15, J = 3 as in the
    paper's runs): the 360 x 256 x 512 grid of the 256^3 workload's plane
    integrals onto the same grid shifted by (0.37, 0.21, 0.43) cells, so
    47,185,920 targets; the grid holds seeded normal complex values."""
    import numpy as np
    import torch

    from paper_1605_05231_gb300 import binding
    from paper_1605_05231_gb300 import inputs as I

    world, rank, local = dist_setup(args)
    dev = torch.device("cuda", torch.cuda.current_device())
    w = I.workload("full256")
    shape = (w.n_az, w.n_pol, w.m)
    J = 3
    gen = torch.Generator(device=dev)
    gen.manual_seed(11)
    grid = torch.complex(torch.randn(shape, generator=gen, device=dev), torch.randn(shape, generator=gen, device=dev))
    targets = I.shifted_polar_targets(shape, RESAMPLE_SHIFT, device=dev)
    P = targets.shape[0]
    out = torch.empty(P, dtype=torch.complex64, device=dev)
    stream = torch.cuda.current_stream(dev)
    for _ in range(max(args.warmup, 3)):
        binding.polar_resample(grid, targets, J, out=out)
    torch.cuda.synchronize()
    clocks = ClockSampler(dev.index)
    barrier(world)
    torch.cuda.synchronize()
    clocks.start()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    for _ in range(args.steps):
        binding.polar_resample(grid, targets, J, out=out)
    ev1.record(stream)
    torch.cuda.synchronize()
    barrier(world)
    clk = clocks.stop()
    ms = max_over_ranks(world, ev0.elapsed_time(ev1) / args.steps)
    if not bool(torch.isfinite(out[:: 997]).all()):
        raise RuntimeError("non-finite resampled values")
    peaks = load_peaks()
    G = grid.numel()
    nbytes = 8 * G + 12 * P + 8 * P
    achieved = nbytes / (ms * 1e-3) / 1e9
    roof = {"bound": "hbm", "achieved": achieved, "peak": peaks["hbm_gbs"], "unit": "GB/s",
            "frac": achieved / peaks["hbm_gbs"], "kernel": "k_polar_resample<3>", "peak_source": peaks["source"],
            "algorithmic_bytes": nbytes,
            "basis": "grid read once (8 B per cell), targets (12 B) and outputs (8 B) once per point",
            "tap_bytes_through_l1": 8 * J ** 3 * P,
            "traffic": ncu_traffic("resample.polar", RESAMPLE_SOURCES)}
    # end to end: the grid and the targets from pinned host memory, the result back
    e2e = None
    if not args.no_e2e:
        gh = grid.cpu().pin_memory()
        th = targets.cpu().pin_memory()
        oh = torch.empty(P, dtype=torch.complex64).pin_memory()
        gd = torch.empty_like(grid)
        td = torch.empty_like(targets)
        for _ in range(2):
            gd.copy_(gh, non_blocking=True)
            td.copy_(th, non_blocking=True)
            binding.polar_resample(gd, td, J, out=out)
            oh.copy_(out, non_blocking=True)
        torch.cuda.synchronize()
        n_e2e = max(3, min(args.steps, 10))
        t0 = time.perf_counter()
        for _ in range(n_e2e):
            gd.copy_(gh, non_blocking=True)
            td.copy_(th, non_blocking=True)
            binding.polar_resample(gd, td, J, out=out)
            oh.copy_(out, non_blocking=True)
        torch.cuda.synchronize()
        ms_e2e = max_over_ranks(world, (time.perf_counter() - t0) * 1e3 / n_e2e)
        e2e = {"value": world * P / (ms_e2e * 1e-3), "unit": "pts/s", "h2d_bytes_per_step": 8 * G + 12 * P,
               "d2h_bytes_per_step": 8 * P, "ms_per_step": ms_e2e,
               "copies": "pinned host buffers, one stream: grid and targets in, result out, every step"}
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        from oracle import polar_resample as R

        xg = grid.cpu().numpy()
        th = targets.cpu().numpy()
        n0 = 200000
        R.polar_sinc_resample(xg, th[:n0 // 10].astype(np.float64), J)   # warm-up
        t0 = time.perf_counter()
        R.polar_sinc_resample(xg, th[:n0].astype(np.float64), J)
        per = (time.perf_counter() - t0) / n0
        ns = int(min(P, max(n0, 15.0 / max(per, 1e-9))))
        idx = np.linspace(0, P - 1, ns).astype(np.int64)
        t0 = time.perf_counter()
        R.polar_sinc_resample(xg, th[idx].astype(np.float64), J)
        t_s = time.perf_counter() - t0
        cpu = {"value": ns / t_s, "unit": "pts/s", "cores": cpu_cores(), "kind": "oracle",
               "sample": f"{ns} of {P} targets spread over the grid, FP64 NumPy; {t_s:.1f} s of CPU work"}
    if rank == 0:
        line = {"metric": "resampled pts/s, polar Radon grid to shifted polar points (Eq. 2.15, J = 3)",
                "value": world * P / (ms * 1e-3), "unit": "pts/s", "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": "f32", "data": "synthetic",
                "config": {"workload": "resample256", "grid": list(shape), "targets": P, "taps": J,
                           "shift": list(RESAMPLE_SHIFT), "parallelism": "single" if world == 1 else f"replicas{world}",
                           "l2": "working set per step >> L2 (0.38 GB grid, 0.57 GB targets, 0.38 GB output)"},
                "clocks": clk, "e2e": e2e, "roofline": roof, "cpu_baseline": cpu, "gpu_launches": args.steps}
        print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist

        dist.destroy_process_group()
    return 0


NUFFT_RESAMPLE_SOURCES = ("polar_nufft.cu", "fft.cuh")


def run_nufft_resample(args):
    """NUFFT-based resampling of the polar Radon grid (Eq. 2.11, J = 6, K = 2n
    per axis): the 360 x 256 x 512 grid of the 256^3 workload's plane integrals
    onto the same grid shifted by (0.37, 0.21, 0.43) cells, 47,185,920 targets
    (nufft_resample128: the 180 x 128 x 256 grid of the 128^3 workload).
    A step is the whole method: the three axis passes (F P F^-1 into the
    720 x 512 x 1024 oversampled spectrum) and the gather."""
    import numpy as np
    import torch

    from paper_1605_05231_gb300 import binding
    from paper_1605_05231_gb300 import inputs as I

    world, rank, local = dist_setup(args)
    dev = torch.device("cuda", torch.cuda.current_device())
    # nufft_resample128: the 180 x 128 x 256 grid of the 128^3 workload (the
    # small case for detailed profiles)
    w = I.workload("mid128" if args.workload == "nufft_resample128" else "full256")
    shape = (w.n_az, w.n_pol, w.m)
    J = 6
    gen = torch.Generator(device=dev)
    gen.manual_seed(11)
    grid = torch.complex(torch.randn(shape, generator=gen, device=dev), torch.randn(shape, generator=gen, device=dev))
    targets = I.shifted_polar_targets(shape, RESAMPLE_SHIFT, device=dev)
    P = targets.shape[0]
    out = torch.empty(P, dtype=torch.complex64, device=dev)
    plan = binding.PolarNufft(*shape, J=J)
    stream = torch.cuda.current_stream(dev)
    for _ in range(max(args.warmup, 3)):
        plan.resample(grid, targets, out=out)
    torch.cuda.synchronize()
    clocks = ClockSampler(dev.index)
    barrier(world)
    torch.cuda.synchronize()
    clocks.start()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    for _ in range(args.steps):
        plan.resample(grid, targets, out=out)
    ev1.record(stream)
    torch.cuda.synchronize()
    barrier(world)
    clk = clocks.stop()
    ms = max_over_ranks(world, ev0.elapsed_time(ev1) / args.steps)
    if not bool(torch.isfinite(out[:: 997]).all()):
        raise RuntimeError("non-finite resampled values")
    # the two parts timed apart, on the same stream (the spectrum is 3 GB, so
    # every pass and the gather stream their inputs from HBM)
    evs = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
    n_part = max(3, min(args.steps, 10))
    t_prep = t_gath = 0.0
    for _ in range(n_part):
        evs[0].record(stream)
        plan.prepare(grid)
        evs[1].record(stream)
        plan.gather(targets, out=out)
        evs[2].record(stream)
        torch.cuda.synchronize()
        t_prep += evs[0].elapsed_time(evs[1]) / n_part
        t_gath += evs[1].elapsed_time(evs[2]) / n_part
    peaks = load_peaks()
    n_phi, n_theta, n_s = shape
    K = [2 * v for v in shape]
    # algorithmic bytes of the three passes: each reads its input once and
    # writes its output once (complex64)
    pass_bytes = 8 * (n_phi * n_theta * n_s + n_phi * n_theta * K[2]) + \
        8 * (n_phi * n_theta * K[2] + n_phi * K[1] * K[2]) + \
        8 * (n_phi * K[1] * K[2] + K[0] * K[1] * K[2])
    pass_gbs = pass_bytes / (t_prep * 1e-3) / 1e9
    # the gather: the spectrum read once, targets and outputs once
    gath_bytes = 8 * K[0] * K[1] * K[2] + 12 * P + 8 * P
    gath_gbs = gath_bytes / (t_gath * 1e-3) / 1e9
    dominant = "gather" if t_gath >= t_prep else "passes"
    parts = {"passes": {"kernel": "k_axis_pass<512>, <256>, <360> (s, theta, phi)", "ms": t_prep,
                        "algorithmic_bytes": pass_bytes, "achieved_gbs": pass_gbs,
                        "frac": pass_gbs / peaks["hbm_gbs"]},
             "gather": {"kernel": "k_polar_nufft_gather<6>", "ms": t_gath, "algorithmic_bytes": gath_bytes,
                        "achieved_gbs": gath_gbs, "frac": gath_gbs / peaks["hbm_gbs"],
                        "tap_bytes_through_l1": 8 * J ** 3 * P}}
    dp = parts[dominant]
    roof = {"bound": "hbm", "achieved": dp["achieved_gbs"], "peak": peaks["hbm_gbs"], "unit": "GB/s",
            "frac": dp["frac"], "kernel": dp["kernel"], "peak_source": peaks["source"],
            "algorithmic_bytes": dp["algorithmic_bytes"],
            "basis": "each array read once and written once (8 B per complex64 cell), targets 12 B and outputs 8 B",
            "parts": parts, "traffic": ncu_traffic("resample.nufft." + dominant, NUFFT_RESAMPLE_SOURCES)}
    e2e = None
    if not args.no_e2e:
        gh = grid.cpu().pin_memory()
        th = targets.cpu().pin_memory()
        oh = torch.empty(P, dtype=torch.complex64).pin_memory()
        gd = torch.empty_like(grid)
        td = torch.empty_like(targets)
        for _ in range(2):
            gd.copy_(gh, non_blocking=True)
            td.copy_(th, non_blocking=True)
            plan.resample(gd, td, out=out)
            oh.copy_(out, non_blocking=True)
        torch.cuda.synchronize()
        n_e2e = max(3, min(args.steps, 10))
        t0 = time.perf_counter()
        for _ in range(n_e2e):
            gd.copy_(gh, non_blocking=True)
            td.copy_(th, non_blocking=True)
            plan.resample(gd, td, out=out)
            oh.copy_(out, non_blocking=True)
        torch.cuda.synchronize()
        ms_e2e = max_over_ranks(world, (time.perf_counter() - t0) * 1e3 / n_e2e)
        e2e = {"value": world * P / (ms_e2e * 1e-3), "unit": "pts/s", "h2d_bytes_per_step": 8 * grid.numel() + 12 * P,
               "d2h_bytes_per_step": 8 * P, "ms_per_step": ms_e2e,
               "copies": "pinned host buffers, one stream: grid and targets in, result out, every step"}
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        # the oracle's FP64 FFTs of the full 720 x 512 x 1024 spectrum do not fit
        # a bounded sample: it runs the whole method on the 90 x 64 x 128 polar
        # grid (1/64 of the cells) with all its shifted targets
        from oracle import polar_nufft_resample as R

        small = (90, 64, 128)
        rng = np.random.default_rng(11)
        xs = rng.normal(size=small) + 1j * rng.normal(size=small)
        ts = I.shifted_polar_targets(small, RESAMPLE_SHIFT).astype(np.float64)
        t0 = time.perf_counter()
        R.nufft_resample(xs, ts, J=J)
        t_s = time.perf_counter() - t0
        cpu = {"value": ts.shape[0] / t_s, "unit": "pts/s", "cores": cpu_cores(), "kind": "oracle",
               "sample": f"the whole method on the 90 x 64 x 128 polar grid ({ts.shape[0]} shifted targets), "
                         f"FP64 NumPy; {t_s:.1f} s of CPU work"}
    plan.close()
    if rank == 0:
        line = {"metric": "resampled pts/s, polar Radon grid to shifted polar points (Eq. 2.11, J = 6, K = 2n)",
                "value": world * P / (ms * 1e-3), "unit": "pts/s", "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": "f32", "data": "synthetic",
                "config": {"workload": args.workload, "grid": list(shape), "oversampled": K, "targets": P,
                           "taps": J, "shift": list(RESAMPLE_SHIFT),
                           "parallelism": "single" if world == 1 else f"replicas{world}",
                           "l2": "working set per step >> L2 (3.0 GB spectrum, 1.5 GB intermediate)"},
                "clocks": clk, "e2e": e2e, "roofline": roof, "cpu_baseline": cpu, "gpu_launches": 4 * args.steps}
        print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist

        dist.destroy_process_group()
    return 0


GRANGEAT_SOURCES = ("grangeat.cu", "fft.cuh")


def run_grangeat(args):
    """Per-view reverse Grangeat step (Sec. 2.2.2, C3a-C3d) for the paper's
    128^3 experiment size: 256 views of 128 x 128 detector images, each view's
    umbrella subset L = 256 lines (2N, as the count of C3c implies) of M = 256
    samples, [5 5] taps, K = 256.  Seeded normal data, post-weights and pre-
    weights uniform in [0.5, 1.5] (the Grangeat weights are inputs)."""
    import numpy as np
    import torch

    from paper_1605_05231_gb300 import binding

    world, rank, local = dist_setup(args)
    dev = torch.device("cuda", torch.cuda.current_device())
    N, V, L, M, J = 128, 256, 256, 256, 5
    ang = np.pi * (np.arange(L) + 0.5) / L
    gen = torch.Generator(device=dev)
    gen.manual_seed(13)
    y = torch.complex(torch.randn((V, L, M), generator=gen, device=dev), torch.randn((V, L, M), generator=gen, device=dev))
    wpost = 0.5 + torch.rand((V, L, M), generator=gen, device=dev)
    wpre = 0.5 + torch.rand((V, N, N), generator=gen, device=dev)
    out = torch.empty((V, N, N), dtype=torch.complex64, device=dev)
    t0 = time.perf_counter()
    g = binding.ReverseGrangeat(N, ang, M, J=J, max_views=V)
    plan_s = time.perf_counter() - t0
    stream = torch.cuda.current_stream(dev)
    for _ in range(max(args.warmup, 3)):
        g.run(y, wpost, wpre, out=out)
    torch.cuda.synchronize()
    clocks = ClockSampler(dev.index)
    barrier(world)
    torch.cuda.synchronize()
    clocks.start()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    for _ in range(args.steps):
        g.run(y, wpost, wpre, out=out)
    ev1.record(stream)
    torch.cuda.synchronize()
    barrier(world)
    clk = clocks.stop()
    ms = max_over_ranks(world, ev0.elapsed_time(ev1) / args.steps)
    if not bool(torch.isfinite(out[:, :: 7, :: 7]).all()):
        raise RuntimeError("non-finite detector images")
    peaks = load_peaks()
    K = 2 * N
    P = L * M
    # HBM bytes of the four kernels: lines read y (8) and w_post (4), write the
    # spectra (8); the spread reads the sparse matrix (12 B per entry) and the
    # spectra, writes K^2 cells; the two inverse passes read / write the grid,
    # the cropped rows, w_pre and the images (8 B per complex64, 4 per float)
    nbytes = V * P * (8 + 4 + 8) + P * J * J * 12 + V * (P * 8 + K * K * 8) + \
        V * (K * K * 8 + N * K * 8) + V * (N * K * 8 + N * N * (4 + 8))
    achieved = nbytes / (ms * 1e-3) / 1e9
    info = g.info()
    roof = {"bound": "hbm", "achieved": achieved, "peak": peaks["hbm_gbs"], "unit": "GB/s",
            "frac": achieved / peaks["hbm_gbs"], "kernel": "k_view_lines, k_view_spread, k_view_ifft_y, k_view_ifft_x",
            "peak_source": peaks["source"], "algorithmic_bytes": nbytes,
            "basis": "every array of the chain read once and written once (whole step)",
            "traffic": ncu_traffic("grangeat.step", GRANGEAT_SOURCES)}
    e2e = None
    if not args.no_e2e:
        yh = y.cpu().pin_memory()
        ph = wpost.cpu().pin_memory()
        qh = wpre.cpu().pin_memory()
        oh = torch.empty_like(out, device="cpu").pin_memory()
        yd, pd, qd = torch.empty_like(y), torch.empty_like(wpost), torch.empty_like(wpre)
        for _ in range(2):
            yd.copy_(yh, non_blocking=True)
            pd.copy_(ph, non_blocking=True)
            qd.copy_(qh, non_blocking=True)
            g.run(yd, pd, qd, out=out)
            oh.copy_(out, non_blocking=True)
        torch.cuda.synchronize()
        n_e2e = max(3, min(args.steps, 10))
        t0 = time.perf_counter()
        for _ in range(n_e2e):
            yd.copy_(yh, non_blocking=True)
            pd.copy_(ph, non_blocking=True)
            qd.copy_(qh, non_blocking=True)
            g.run(yd, pd, qd, out=out)
            oh.copy_(out, non_blocking=True)
        torch.cuda.synchronize()
        ms_e2e = max_over_ranks(world, (time.perf_counter() - t0) * 1e3 / n_e2e)
        e2e = {"value": world * V / (ms_e2e * 1e-3), "unit": "views/s", "h2d_bytes_per_step": V * P * 12 + V * N * N * 4,
               "d2h_bytes_per_step": V * N * N * 8, "ms_per_step": ms_e2e,
               "copies": "pinned host buffers, one stream: data and weights in, images out, every step"}
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        from oracle import reverse_grangeat as R

        nv = 2
        yc = y[:nv].cpu().numpy().astype(np.complex128)
        pc = wpost[:nv].cpu().numpy().astype(np.float64)
        qc = wpre[:nv].cpu().numpy().astype(np.float64)
        t0 = time.perf_counter()
        R.reverse_grangeat(yc, pc, qc, ang, N, J=J)
        t_s = time.perf_counter() - t0
        cpu = {"value": nv / t_s, "unit": "views/s", "cores": cpu_cores(), "kind": "oracle",
               "sample": f"{nv} of {V} views, FP64 NumPy; {t_s:.1f} s of CPU work"}
    g.close()
    if rank == 0:
        line = {"metric": "detector views/s, reverse Grangeat step (Sec. 2.2.2, C3a-C3d, [5 5] taps)",
                "value": world * V / (ms * 1e-3), "unit": "views/s", "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": "f32", "data": "synthetic",
                "config": {"workload": "grangeat128", "detector": [N, N], "views": V, "lines_per_view": L,
                           "samples_per_line": M, "taps": J, "oversampled": K, "spread_nnz": info["nnz"],
                           "plan_s": plan_s, "parallelism": "single" if world == 1 else f"replicas{world}",
                           "l2": "working set per step above L2 (0.13 GB data, 0.08 GB weights, 0.13 GB spectra, 0.13 GB grid)"},
                "clocks": clk, "e2e": e2e, "roofline": roof, "cpu_baseline": cpu, "gpu_launches": 4 * args.steps}
        print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist

        dist.destroy_process_group()
    return 0


def main():
    args = parse_args()
    if args.impl == "reference":
        return run_reference(args)
    if args.workload == "batch24":
        return run_batch(args)
    if args.workload == "resample256":
        return run_resample(args)
    if args.workload in ("nufft_resample256", "nufft_resample128"):
        return run_nufft_resample(args)
    if args.workload == "grangeat128":
        return run_grangeat(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
