"""Autotuner for the block shape of the trajectory kernels.

A candidate is (threads per block, sites per thread); the tile of a series cut
into tiles is the largest the window allows.  Each candidate's plan is built
(`rsv_set_schedule` + `rsv_plan_create`) and one trajectory of the workload is
timed with CUDA events; the fastest wins.  Results are cached in a JSON file
keyed by GPU name, precision, n_md, mass and a size bucket of the workload, so
later runs skip the search.  Results never change the numbers a plan computes,
only its speed.
"""
from __future__ import annotations

import json
import math
import os

import numpy as np
import torch

from . import rsv

# bumped whenever the trajectory kernels change, so cached choices are redone
KERNEL_REV = 15

CANDIDATES = {
    "mixed": ([(nt, 20) for nt in (128, 192, 256, 320, 384)]
              + [(nt, 16) for nt in (128, 256, 384, 512)]
              + [(nt, 12) for nt in (192, 320, 448, 640)]
              + [(nt, 8) for nt in (256, 384, 512, 768)]),
    "fp64": [(nt, j) for j in (8, 16, 28) for nt in (64, 128, 192, 256)],
}


def _cache_path() -> str:
    d = os.environ.get("RSV_TUNE_CACHE") or os.path.join(os.path.expanduser("~"), ".cache",
                                                         "rsv_gb300")
    os.makedirs(d, exist_ok=True)
    return os.path.join(d, "schedules.json")


def _key(prec, n_md, mass, offsets) -> str:
    T = np.diff(np.asarray(offsets))
    name = torch.cuda.get_device_name()
    b_total = int(math.log2(max(int(T.sum()), 1)))
    b_max = int(math.log2(max(int(T.max()), 1)))
    return (f"{name}|k{KERNEL_REV}|{prec}|{n_md}|{int(bool(mass))}|n{len(T)}|tot2^{b_total}"
            f"|max2^{b_max}")


def tune_plan(ctx: rsv.Context, offsets, n_md: int, prec: str, y, lnrv, theta_dev, dtau: float,
              h_init, minv=None, reps: int = 3, use_cache: bool = True):
    """Return (Plan, schedule dict) with the fastest measured block shape."""
    key = _key(prec, n_md, minv is not None, offsets)
    path = _cache_path()
    cache = {}
    if use_cache and os.path.exists(path):
        try:
            cache = json.load(open(path))
        except (OSError, ValueError):
            cache = {}
    K = n_md + 1
    if use_cache and key in cache:
        nt, j = cache[key]["threads"], cache[key]["sites_per_thread"]
        rsv.rsv_set_schedule(ctx, nt, j, nt * j - 2 * K - 3)
        try:
            plan = rsv.Plan(ctx, offsets, n_md, prec, with_mass=minv is not None)
        finally:
            rsv.rsv_set_schedule(ctx)
        return plan, dict(cache[key], cached=True)
    results = []
    h = torch.empty_like(h_init)
    for nt, j in CANDIDATES["mixed" if prec == "mixed" else "fp64"]:
        tile = nt * j - 2 * K - 3
        if tile < 1:
            continue
        try:
            rsv.rsv_set_schedule(ctx, nt, j, tile)
            plan = rsv.Plan(ctx, offsets, n_md, prec, with_mass=minv is not None)
        except rsv.RSVError:
            continue
        finally:
            rsv.rsv_set_schedule(ctx)
        times = []
        for r in range(reps + 1):
            h.copy_(h_init)
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record()
            rsv.rsv_hmc_batched(ctx, plan, h, y, lnrv, theta_dev, dtau, minv=minv, seed=1,
                                traj0=r)
            b.record()
            b.synchronize()
            if r:
                times.append(a.elapsed_time(b))
        results.append((min(times), nt, j, plan.info()))
        plan.close()
    results.sort(key=lambda r: r[0])
    best_ms, nt, j, info = results[0]
    entry = {"threads": nt, "sites_per_thread": j, "ms": best_ms, "info": info,
             "candidates": [(round(t, 4), a, b) for t, a, b, _ in results]}
    cache[key] = entry
    try:
        with open(path, "w") as f:
            json.dump(cache, f, indent=1)
    except OSError:
        pass
    rsv.rsv_set_schedule(ctx, nt, j, nt * j - 2 * K - 3)
    try:
        plan = rsv.Plan(ctx, offsets, n_md, prec, with_mass=minv is not None)
    finally:
        rsv.rsv_set_schedule(ctx)
    return plan, dict(entry, cached=False)
