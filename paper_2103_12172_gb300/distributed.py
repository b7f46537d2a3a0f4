"""Sharding of the projection columns across ranks (one process per GPU).

The AP solves of different columns and subdomains are independent (the paper distributes the
columns of Q to parallel processors, Section 3.6), so the only exchange is one gather of the Q
blocks to the rank that assembles the global least-squares system. Units of work are
(subdomain, column tile) pairs; ranks receive them by greedy longest-processing-time-first on
a cost proportional to the swept mode-space volume (modes x rows), and units of subdomains
with the same grid and wavenumber are kept on one rank when balance allows, so each rank
factors each distinct (grid, k) once.
"""
from __future__ import annotations


def unit_cost(sub) -> float:
    """Relative cost of one column of `sub`: modes x rows of the tridiagonal sweeps."""
    return float((sub.nx - 2) * sub.ny)


def make_units(subdomains, tile_cols: int = 256):
    """(sub index, col0, ncols, cost) work units."""
    units = []
    for i, s in enumerate(subdomains):
        n = 8 * s.n_modes
        for c0 in range(0, n, tile_cols):
            nc = min(tile_cols, n - c0)
            units.append((i, c0, nc, nc * unit_cost(s)))
    return units


def lpt_partition(subdomains, world: int, tile_cols: int = 256):
    """Assign units to `world` ranks, largest cost first, each to the least-loaded rank unless a
    rank that already holds a subdomain with the same (grid, k) is within one unit of that load.
    The final loads differ by at most two units. Returns a list (per rank) of (sub, col0,
    ncols) and the per-rank loads."""
    if world < 1:
        raise ValueError("world must be >= 1")
    units = sorted(make_units(subdomains, tile_cols), key=lambda u: (-u[3], u[0], u[1]))
    load = [0.0] * world
    keys = [set() for _ in range(world)]
    out = [[] for _ in range(world)]
    for sub, c0, nc, cost in units:
        s = subdomains[sub]
        key = (s.nx, s.ny, s.k, s.ap_bc)
        lo = min(load)
        # a rank that already factors this (grid, k) takes the unit if its load is within one
        # unit of the minimum; otherwise the least-loaded rank does
        holders = [r for r in range(world) if key in keys[r] and load[r] <= lo + cost + 1e-9]
        r = min(holders, key=lambda x: load[x]) if holders else load.index(lo)
        out[r].append((sub, c0, nc))
        load[r] += cost
        keys[r].add(key)
    for lst in out:
        lst.sort()
    return out, load


def gather_blocks(blocks, dst: int = 0, group=None):
    """Gather per-rank dicts {(sub, col0, ncols): tensor[ncols, |gamma|]} onto rank `dst`
    (torch.distributed, any backend; tensors are moved to CPU for the object collective).
    Returns the merged dict on `dst`, None elsewhere."""
    import torch.distributed as dist
    payload = {k: v.detach().cpu() for k, v in blocks.items()}
    world = dist.get_world_size(group)
    gathered = [None] * world if dist.get_rank(group) == dst else None
    dist.gather_object(payload, gathered, dst=dst, group=group)
    if gathered is None:
        return None
    merged = {}
    for g in gathered:
        merged.update(g)
    return merged


def assemble(subdomains, merged, layout):
    """Per-subdomain column blocks [8M*][|gamma|] from gathered units; layout(sub) -> |gamma|."""
    import torch
    res = []
    for i, s in enumerate(subdomains):
        n = 8 * s.n_modes
        blk = torch.zeros(n, layout(i), dtype=torch.complex128)
        filled = 0
        for (sub, c0, nc), t in merged.items():
            if sub == i:
                blk[c0:c0 + nc] = t
                filled += nc
        if filled != n:
            raise RuntimeError(f"subdomain {i}: {filled} of {n} columns gathered")
        res.append(blk)
    return res
