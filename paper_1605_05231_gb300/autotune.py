"""Autotuner for the interpolation kernels of a plan or a batch.

For a plan it times forward + adjoint with CUDA events for each candidate
(gather variant, spread variant, points per subproblem, tile edge), keeps the
fastest, applies it with Plan.tune and caches the choice in a JSON file keyed
by the problem signature (N, K, J, M, number of lines, volume type, grid dtype,
coefficient mode, GPU name).  Candidates a plan cannot run (NUFFT3D_ERR_UNSUPPORTED) are skipped.
"""
from __future__ import annotations

import json
import os
from typing import Dict, Iterable, Optional, Tuple

from .binding import NufftError

# (gather variant, spread variant, points per subproblem, tile edge)
CANDIDATES: Tuple[Tuple[int, int, int, int], ...] = (
    (10, 7, 256, 8),
    (11, 7, 256, 8),
    (10, 8, 256, 8),
    (9, 7, 256, 8),
    (5, 6, 256, 8),
    (8, 6, 256, 8),
    (3, 6, 256, 8),
    (3, 5, 512, 8),
    (5, 3, 256, 8),
    (5, 3, 512, 8),
    (3, 3, 256, 8),
    (3, 3, 512, 8),
    (3, 3, 1024, 8),
    (8, 3, 256, 8),
    (8, 3, 512, 8),
    (7, 3, 256, 8),
    (4, 3, 512, 8),
    (3, 2, 512, 8),
    (2, 2, 1024, 8),
    (0, 3, 512, 8),
    (3, 0, 1024, 16),
    (3, 1, 1024, 16),
)


def default_cache_path() -> str:
    return os.environ.get("NUFFT3D_TUNE_CACHE",
                          os.path.join(os.path.expanduser("~"), ".cache", "nufft3d_autotune.json"))


def signature(plan) -> str:
    import torch

    info = plan.info()
    name = torch.cuda.get_device_name(plan.device)
    return (f"N{plan.n}_K{plan.k}_J{plan.j}_M{plan.m}_D{plan.n_dirs}_"
            f"{'c' if plan.complex_volume else 'r'}_{plan.grid_dtype}_{'x' if plan.exact_coeffs else 't'}_{name}")


def _load(path):
    try:
        with open(path) as fh:
            return json.load(fh)
    except Exception:
        return {}


def _store(path, data):
    try:
        os.makedirs(os.path.dirname(path), exist_ok=True)
        tmp = path + ".tmp"
        with open(tmp, "w") as fh:
            json.dump(data, fh, indent=1)
        os.replace(tmp, path)
    except Exception:
        pass


def time_plan(plan, reps: int = 3) -> float:
    """Milliseconds of one forward + adjoint (mean of reps after one warm-up)."""
    import torch

    dev = plan.device
    vol = torch.randn((plan.n,) * 3, device=dev, dtype=torch.float32)
    if plan.complex_volume:
        vol = torch.complex(vol, torch.randn_like(vol))
    lines = torch.empty((plan.n_dirs, plan.m), dtype=torch.complex64, device=dev)
    out = torch.empty_like(vol)
    plan.forward(vol, out=lines)
    plan.adjoint(lines, out=out)
    s = torch.cuda.current_stream(dev)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(s)
    for _ in range(reps):
        plan.forward(vol, out=lines)
        plan.adjoint(lines, out=out)
    e1.record(s)
    e1.synchronize()
    return e0.elapsed_time(e1) / reps


def tune_plan(plan, candidates: Iterable = CANDIDATES, reps: int = 3, cache: Optional[str] = "default",
              force: bool = False) -> Dict:
    """Pick and apply the fastest candidate; returns {"best": cand, "ms": t, "timings": {...}}."""
    path = default_cache_path() if cache == "default" else cache
    key = signature(plan)
    if path and not force:
        hit = _load(path).get(key)
        if hit:
            try:
                plan.tune(*hit["best"])
                return dict(hit, cached=True)
            except NufftError:
                pass
    timings = {}
    for cand in candidates:
        try:
            plan.tune(*cand)
        except NufftError:
            continue
        timings[str(tuple(cand))] = time_plan(plan, reps)
    if not timings:
        raise RuntimeError("no candidate configuration runs on this plan")
    best = min(timings, key=timings.get)
    best_cand = [int(v) for v in best.strip("()").split(",")]
    plan.tune(*best_cand)
    res = {"best": best_cand, "ms": timings[best], "timings": timings}
    if path:
        data = _load(path)
        data[key] = {"best": best_cand, "ms": timings[best]}
        _store(path, data)
    return dict(res, cached=False)


def tune_batch(batch, candidates: Iterable = CANDIDATES, reps: int = 3, cache: Optional[str] = "default",
               force: bool = False) -> Dict[str, Dict]:
    """Tune one representative plan per distinct signature, apply its choice to
    every item with that signature, and re-capture the batch graph."""
    chosen = {}
    for plan in batch.items:
        key = signature(plan)
        if key not in chosen:
            chosen[key] = tune_plan(plan, candidates, reps, cache, force)
        else:
            plan.tune(*chosen[key]["best"])
    batch.invalidate()
    return chosen
