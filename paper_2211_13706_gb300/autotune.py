"""Autotuner for a plan's launch shapes (mz_plan_tune).

It times the transforms a caller is about to run (zeta and Moebius of one
batch, on the caller's own input) under a small grid of launch shapes, keeps
the fastest, and remembers it per workload key: (posets, nodes, largest chain
count, batch, dtype, schedule). Results never depend on the shapes, only the
time does. The cache lives in memory and, if MZ_TUNE_CACHE names a file, in
that JSON file as well.
"""
from __future__ import annotations

import json
import os

from . import mz_plan_tune

CANDIDATES = {
    "mobius_blocks_per_sm": (1, 2, 3, 4),
    "mobius_pace_ns": (300, 600, 1000, 1600),
    "gather_blocks_per_sm": (8, 16, 32),
    "mobius_lanes": (1, 32),               # one function per row only
}
_CACHE: dict = {}


def _key(plan, x, batch) -> str:
    info = plan.info
    return f"c{info['components']}-n{info['n']}-k{info['k']}-l{info['ulevels']}-b{batch}-{x.dtype}-s{info['schedule']}"


def _load_file():
    path = os.environ.get("MZ_TUNE_CACHE")
    if path and os.path.exists(path):
        try:
            with open(path) as fh:
                _CACHE.update(json.load(fh))
        except (OSError, ValueError):
            pass


def _save_file():
    path = os.environ.get("MZ_TUNE_CACHE")
    if path:
        tmp = path + f".{os.getpid()}.tmp"
        with open(tmp, "w") as fh:
            json.dump(_CACHE, fh, indent=1, sort_keys=True)
        os.replace(tmp, path)


def _time(fn, reps: int):
    import torch
    fn()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(reps):
        fn()
    e1.record()
    e1.synchronize()
    return e0.elapsed_time(e1) / reps


def tune(plan, x, reps: int = 3) -> dict:
    """Picks launch shapes for zeta + Moebius of `x` (a device tensor in the plan's
    layout) on `plan`, applies them, and returns them."""
    if not _CACHE:
        _load_file()
    import torch
    pair = x.dtype == torch.float32              # F32C values: [2, n] or [2, n, batch]
    batch = 1 if x.dim() == (2 if pair else 1) else x.shape[-1]
    key = _key(plan, x, batch)
    if key in _CACHE:
        mz_plan_tune(plan.handle, **_CACHE[key])
        return dict(_CACHE[key])
    g = plan.zeta(x)
    y = plan.mobius(g)
    best_g = None
    for gb in CANDIDATES["gather_blocks_per_sm"]:
        mz_plan_tune(plan.handle, gather_blocks_per_sm=gb)
        t = _time(lambda: plan.zeta(x, out=g), reps)
        if best_g is None or t < best_g[0]:
            best_g = (t, gb)
    best_l = None
    if batch == 1:    # lanes per row first, at the current blocks and pacing
        for lanes in CANDIDATES["mobius_lanes"]:
            mz_plan_tune(plan.handle, mobius_lanes=lanes)
            t = _time(lambda: plan.mobius(g, out=y), reps)
            if best_l is None or t < best_l[0]:
                best_l = (t, lanes)
        mz_plan_tune(plan.handle, mobius_lanes=best_l[1])
    best_m = None
    for bps in CANDIDATES["mobius_blocks_per_sm"]:
        for pace in CANDIDATES["mobius_pace_ns"]:
            mz_plan_tune(plan.handle, mobius_blocks_per_sm=bps, mobius_pace_ns=pace)
            t = _time(lambda: plan.mobius(g, out=y), reps)
            if best_m is None or t < best_m[0]:
                best_m = (t, bps, pace)
    plan.check()
    choice = {"gather_blocks_per_sm": best_g[1], "mobius_blocks_per_sm": best_m[1], "mobius_pace_ns": best_m[2]}
    if best_l is not None:
        choice["mobius_lanes"] = best_l[1]
    mz_plan_tune(plan.handle, **choice)
    _CACHE[key] = choice
    _save_file()
    return dict(choice)
