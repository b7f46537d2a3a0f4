"""Tile autotuner for the batched projection: picks the columns per work item that gives the
shortest mdp_project_batch on this GPU for a workload's shape, by timing candidates with CUDA
events, and caches the choice per (GPU, workload shape) in a JSON file
(MDP_AUTOTUNE_CACHE, default: _autotune_cache.json beside this module)."""
from __future__ import annotations

import json
import os

_DEFAULT_CACHE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "_autotune_cache.json")


def _signature(subdomains):
    shapes = sorted((s.nx, s.ny, s.ap_bc, s.n_modes) for s in subdomains)
    return ";".join("%dx%d:%d:%d" % t for t in shapes)


def tune_tile(subdomains, candidates=(32, 64, 128, 256, 512), reps=3, cache_path=None, force=False):
    """Best tile_cols for these subdomains (timed on the current CUDA device)."""
    import torch

    from . import Plan

    cache_path = cache_path or os.environ.get("MDP_AUTOTUNE_CACHE", _DEFAULT_CACHE)
    key = torch.cuda.get_device_name() + "|" + _signature(subdomains)
    cache = {}
    if os.path.exists(cache_path):
        try:
            cache = json.load(open(cache_path))
        except (OSError, ValueError):
            cache = {}
    if not force and key in cache:
        return int(cache[key]["tile_cols"])
    max_cols = max(8 * s.n_modes for s in subdomains)
    if sum(8 * s.n_modes for s in subdomains) >= 8192:
        # large batches fill the GPU at any tile: skip the small tiles (each candidate is a plan)
        candidates = [c for c in candidates if c >= 128] or list(candidates)
    cands = sorted({min(c, max_cols) for c in candidates})
    times = {}
    for tile in cands:
        plan = Plan(subdomains, tile_cols=tile)
        out = torch.empty(plan.output_size, dtype=torch.complex128, device="cuda")
        plan.project(out=out)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(reps):
            plan.project(out=out)
        e1.record()
        torch.cuda.synchronize()
        times[tile] = e0.elapsed_time(e1) / reps
        plan.close()
        del out
    best = min(times, key=times.get)
    cache[key] = {"tile_cols": best, "ms": times}
    try:
        with open(cache_path, "w") as f:
            json.dump(cache, f, indent=1, default=str)
    except OSError:
        pass
    return best
