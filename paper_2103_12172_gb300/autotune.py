"""Autotuner of the batched projection: picks, for a workload's shape on this GPU, the plan options
that give the shortest mdp_project_batch, by timing candidates with CUDA events, and caches the
choice per (GPU, workload shape) in a JSON file (MDP_AUTOTUNE_CACHE, default:
_autotune_cache.json beside this module).

Searched, by coordinate descent in this order (each step keeps the best of the previous ones):
  tile_cols         columns per work item (the batching tile);
  fp64_cols         the gamma columns of the middle rows by FP64 sums instead of the tensor cores
                    (only when some subdomain can take the tensor-core contraction);
  direct_rows       the dense-row sine transforms by direct sums instead of the FFT (only when
                    some subdomain has a power-of-two Nx);
  fft_block_points  complex values per block of the dense-row FFT kernels (FFT rows only);
  tri_stages        table rows the per-mode sweep stages ahead in shared memory;
  workspace_bytes   not timed: the budget that packs work items into waves, as large as a quarter
                    of the free device memory allows up to 32 GiB (fewer, larger waves: fewer
                    launch tails of the sweep; 224 -> 213 ms per step on the 8 x 8 workload from
                    4 to 32 GiB), never below the 4 GiB default.
Large workloads are timed on a sample: one subdomain of every (grid, AP, M*) class, all its
columns; the per-item kernel choices carry over, the batching effects of the full workload less
so (the bench reports the graph-replayed step beside the plain one for that)."""
from __future__ import annotations

import json
import os

_DEFAULT_CACHE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "_autotune_cache.json")
_DEFAULTS = {"tile_cols": 256, "fp64_cols": False, "direct_rows": False, "fft_block_points": 1024, "tri_stages": 2,
             "workspace_bytes": 0}
_WS_DEFAULT, _WS_MAX = 4 << 30, 32 << 30


def workspace_budget():
    """The workspace budget for a plan on the current device: a quarter of the free memory, in
    whole GiB, between the 4 GiB default and 32 GiB (0 = the default)."""
    import torch
    free, _ = torch.cuda.mem_get_info()
    ws = min(_WS_MAX, (free // 4) >> 30 << 30)
    return ws if ws > _WS_DEFAULT else 0


def _signature(subdomains):
    shapes = sorted((s.nx, s.ny, s.ap_bc, s.n_modes) for s in subdomains)
    return ";".join("%dx%d:%d:%d" % t for t in shapes)


def _sample(subdomains, max_full=8):
    """The workload itself when small, else one subdomain of each (grid, AP, M*) class."""
    subs = list(subdomains)
    if len(subs) <= max_full:
        return subs
    seen, out = set(), []
    for s in subs:
        key = (s.nx, s.ny, s.ap_bc, s.n_modes)
        if key not in seen:
            seen.add(key)
            out.append(s)
    return out


def _time_plan(subs, opts, reps):
    import torch

    from . import Plan
    plan = Plan(subs, **opts)
    out = torch.empty(plan.output_size, dtype=torch.complex128, device="cuda")
    plan.project(out=out)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(reps):
        plan.project(out=out)
    e1.record()
    torch.cuda.synchronize()
    plan.status()
    plan.close()
    del out
    return e0.elapsed_time(e1) / reps


def _load(cache_path):
    if os.path.exists(cache_path):
        try:
            return json.load(open(cache_path))
        except (OSError, ValueError):
            return {}
    return {}


def _store(cache_path, cache):
    try:
        with open(cache_path, "w") as f:
            json.dump(cache, f, indent=1, default=str)
    except OSError:
        pass


def tune_plan(subdomains, tiles=(64, 128, 256, 512), reps=3, cache_path=None, force=False):
    """Best plan options for these subdomains on the current CUDA device: a dict of Plan keyword
    arguments (tile_cols, fp64_cols, direct_rows, fft_block_points, tri_stages,
    workspace_bytes), plus the timings behind it under "ms" (not a Plan argument)."""
    import torch

    cache_path = cache_path or os.environ.get("MDP_AUTOTUNE_CACHE", _DEFAULT_CACHE)
    key = "plan|" + torch.cuda.get_device_name() + "|" + _signature(subdomains)
    cache = _load(cache_path)
    if not force and key in cache:
        return dict(cache[key])
    sample = _sample(subdomains)
    max_cols = max(8 * s.n_modes for s in sample)
    tc_possible = any(s.nx - 2 <= 2047 for s in sample)     # the plan decides per subdomain
    fft_possible = any(((s.nx - 1) & (s.nx - 2)) == 0 and 8 <= s.nx - 1 <= 2048 for s in sample)
    best = dict(_DEFAULTS)
    times = {}

    def run(opts):
        k = json.dumps(opts, sort_keys=True)
        if k not in times:
            times[k] = _time_plan(sample, opts, reps)
        return times[k]

    def descend(name, values):
        cands = [dict(best, **{name: v}) for v in values]
        t = [run(c) for c in cands]
        best.update(cands[t.index(min(t))])

    descend("tile_cols", sorted({min(c, max_cols) for c in tiles}))
    if tc_possible:
        descend("fp64_cols", [False, True])
    if fft_possible:
        descend("direct_rows", [False, True])
    if fft_possible and not best["direct_rows"]:
        descend("fft_block_points", [1024, 2048, 4096])
    descend("tri_stages", [2, 4])
    best["workspace_bytes"] = workspace_budget()
    result = dict(best, ms={k: v for k, v in times.items()}, sample_subdomains=len(sample))
    cache[key] = result
    _store(cache_path, cache)
    return dict(result)


def plan_kwargs(tuned):
    """The Plan keyword arguments of a tune_plan result."""
    return {k: tuned[k] for k in _DEFAULTS}


def tune_tile(subdomains, candidates=(32, 64, 128, 256, 512), reps=3, cache_path=None, force=False):
    """Best tile_cols alone for these subdomains (other options at their defaults), timed on the
    whole workload on the current CUDA device and cached."""
    import torch

    cache_path = cache_path or os.environ.get("MDP_AUTOTUNE_CACHE", _DEFAULT_CACHE)
    key = torch.cuda.get_device_name() + "|" + _signature(subdomains)
    cache = _load(cache_path)
    if not force and key in cache:
        return int(cache[key]["tile_cols"])
    max_cols = max(8 * s.n_modes for s in subdomains)
    cands = sorted({min(c, max_cols) for c in candidates})
    times = {tile: _time_plan(list(subdomains), {"tile_cols": tile}, reps) for tile in cands}
    best = min(times, key=times.get)
    cache[key] = {"tile_cols": best, "ms": times}
    _store(cache_path, cache)
    return best
