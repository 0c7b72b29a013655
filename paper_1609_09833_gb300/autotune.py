"""Launch-shape autotuner for the batched form.

For a batch of walker specs and a representative block of frames, times the
launch shapes the library exposes through ``abp_ctx_tune`` (threads per
walker group, walker groups per CTA, the shared-memory grid tile) with CUDA
events on scratch copies of the walkers (the caller's walkers and grids are
not touched), keeps the fastest, applies it to the context and caches it per
(device, batch signature) in a JSON file. The knobs only reschedule work:
tiles and groups-per-CTA give bit-identical results; another group width
changes the order of the CV sums (results agree to rounding).
"""
from __future__ import annotations

import json
import os

import numpy as np

from . import abp

DEFAULT_CACHE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "_build", "tune_cache.json")


def signature(specs, nsteps: int) -> str:
    """A key for the batch: walker shapes and the launch length."""
    kinds = {}
    for s in specs:
        cv = "-".join(c["type"] for c in s["cvs"])
        key = f"{s['natoms']}:{cv}:{'x'.join(map(str, s['grid']['n']))}"
        kinds[key] = kinds.get(key, 0) + 1
    body = ";".join(f"{k}*{v}" for k, v in sorted(kinds.items()))
    return f"n{len(specs)}|t{nsteps}|{body}"


def candidates(specs):
    cn = any(c["type"] == "coord" for s in specs for c in s["cvs"])
    out = []
    for G in ((64, 128, 256) if cn else (32, 64, 128, 256)):
        for gpc in ((1, 2) if G >= 128 else (1, 2, 4)):
            for lean in (0, 1):
                out.append({"group_threads": G, "groups_per_cta": gpc, "tile": 0, "lean": lean})
    if not cn:
        out.append({"group_threads": 32, "groups_per_cta": 1, "tile": 1, "lean": 0})
    return out


def _apply(ctx, c):
    abp.abp_ctx_tune(ctx.handle, abp.ABP_TUNE_GROUP_THREADS, c["group_threads"])
    abp.abp_ctx_tune(ctx.handle, abp.ABP_TUNE_GROUPS_PER_CTA, c["groups_per_cta"])
    abp.abp_ctx_tune(ctx.handle, abp.ABP_TUNE_TILE, c["tile"])
    abp.abp_ctx_tune(ctx.handle, abp.ABP_TUNE_LEAN, c.get("lean", 0))


def tune(ctx, specs, frames, offsets, nsteps: int, reps: int = 3, cache_path: str | None = DEFAULT_CACHE,
         cands=None, verbose: bool = False) -> dict:
    """Pick and apply the fastest launch shape. frames: device records
    [>= nsteps, atoms, 4] (float32); offsets: device int64 per walker."""
    import torch

    dev_name = torch.cuda.get_device_name(ctx.device)
    key = f"{dev_name}|{signature(specs, nsteps)}"
    cache = {}
    if cache_path and os.path.exists(cache_path):
        try:
            with open(cache_path) as f:
                cache = json.load(f)
        except (OSError, ValueError):
            cache = {}
    if key in cache:
        best = cache[key]["best"]
        _apply(ctx, best)
        return {"best": best, "cached": True, "timings": cache[key].get("timings", [])}
    A = frames.shape[1]
    F = torch.zeros(nsteps, A, 4, device=frames.device)
    ngrids = len(ctx.grids)
    scratch = ctx.make_walkers(specs)
    timings = []
    try:
        for c in (cands or candidates(specs)):
            try:
                _apply(ctx, c)
                abp.abp_run(ctx.handle, scratch, frames, abp.ABP_F32, offsets, A, F, offsets, A,
                            abp.ABP_FORCES_OVERWRITE, 0, nsteps)
                torch.cuda.synchronize()
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record()
                for r in range(reps):
                    abp.abp_run(ctx.handle, scratch, frames, abp.ABP_F32, offsets, A, F, offsets, A,
                                abp.ABP_FORCES_OVERWRITE, (r + 1) * nsteps, nsteps)
                e1.record()
                torch.cuda.synchronize()
                ms = e0.elapsed_time(e1) / reps
            except abp.AbpError:
                ms = float("inf")
            timings.append({**c, "ms": ms})
            if verbose:
                print("tune", c, ms)
    finally:
        torch.cuda.synchronize()
        for w in scratch:
            abp.abp_walker_destroy(w.handle)
            ctx.walkers.remove(w)
        for g in ctx.grids[ngrids:]:
            abp.abp_grid_destroy(g)
        del ctx.grids[ngrids:]
    best = min(timings, key=lambda r: r["ms"])
    best = {k: best[k] for k in ("group_threads", "groups_per_cta", "tile", "lean")}
    _apply(ctx, best)
    if cache_path:
        cache[key] = {"best": best, "timings": timings}
        os.makedirs(os.path.dirname(cache_path), exist_ok=True)
        tmp = cache_path + f".tmp{os.getpid()}"
        with open(tmp, "w") as f:
            json.dump(cache, f, indent=1)
        os.replace(tmp, cache_path)
    return {"best": best, "cached": False, "timings": timings}
