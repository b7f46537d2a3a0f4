"""Persisted cache of projection blocks, keyed by everything the block depends on.

A subdomain's block of basis columns (Q = (P_gamma - I) Ex Psi, or P_gamma Ex Psi) depends only
on its auxiliary problem: grid, step, wavenumber, AP type, M* and the placement of the subdomain
relative to its grid, plus the conventions of this library (orientation, boundary rows, basis,
ordering). The paper precomputes Q once per distinct subdomain problem and reuses it across
experiments (Section 4); this cache does the same across runs and processes. Blocks are stored
as .npy files (complex128, [8 M*][|gamma|]) named by a sha256 of the key; translated copies of a
subdomain hit the same entry.

    cache = QCache("/path/to/dir")
    out = cache.project(plan)          # loads cached blocks, computes and stores the others
"""
from __future__ import annotations

import hashlib
import os

import numpy as np

# Conventions a cached block depends on. Change the string when any of them changes.
CONVENTIONS = ("mdp-2103.12172 v1; DST along x, tridiagonal along y; AP Dirichlet4 or Dirichlet-x/"
               "Sommerfeld-y with O(h^4) half-node rows; M+ strict; gamma 2-node ring row-major; "
               "side ownership by smallest |rho|, ties within 1e-9 h to the lower side; Taylor "
               "extension through rho^4; basis T_{j-1}(s) with (2/L)^p derivatives; columns "
               "[D: side x j][N: side x j]; FP64")


def problem_key(sub, kind: str) -> str:
    """sha256 of the subdomain's auxiliary problem (translation-invariant) and the output kind."""
    h = float(sub.h)
    rel = [(float(sub.x0) - float(sub.ax0)) / h, (float(sub.x1) - float(sub.ax0)) / h,
           (float(sub.y0) - float(sub.ay0)) / h, (float(sub.y1) - float(sub.ay0)) / h]
    fields = [CONVENTIONS, kind, repr(h), repr(float(sub.k)), str(int(sub.nx)), str(int(sub.ny)),
              str(int(sub.ap_bc)), str(int(sub.n_modes))] + [f"{v:.9f}" for v in rel]
    return hashlib.sha256("|".join(fields).encode()).hexdigest()


class QCache:
    def __init__(self, directory: str):
        self.dir = directory
        os.makedirs(directory, exist_ok=True)

    def path(self, sub, kind: str) -> str:
        return os.path.join(self.dir, problem_key(sub, kind) + ".npy")

    def project(self, plan, kind: str = "Q", out=None, stream=None):
        """All basis-column blocks of `plan` (a device Plan) in the layout of plan.project:
        cached blocks are read from disk, the others computed on the GPU (one batched call
        when none is cached, else per subdomain) and written to the cache."""
        import torch
        out = out if out is not None else torch.empty(plan.output_size, dtype=torch.complex128, device="cuda")
        blocks = plan.blocks(out)
        missing = []
        for i, sub in enumerate(plan.subdomains):
            p = self.path(sub, kind)
            if os.path.exists(p):
                arr = np.load(p)
                if arr.shape != tuple(blocks[i].shape):
                    raise ValueError(f"cached block {p} has shape {arr.shape}, expected {tuple(blocks[i].shape)}")
                blocks[i].copy_(torch.from_numpy(arr), non_blocking=False)
            else:
                missing.append(i)
        if not missing:
            return out
        if len(missing) == plan.n_subs:
            plan.project(kind=kind, out=out, stream=stream)
        else:
            for i in missing:
                g, nc, off, _ = plan.layout(i)
                blocks[i].copy_(plan.project_columns(i, 0, nc, kind=kind, stream=stream).view(nc, g))
        done = set()
        for i in missing:
            p = self.path(plan.subdomains[i], kind)
            if p in done:
                continue
            tmp = p[:-len(".npy")] + f".{os.getpid()}.tmp.npy"   # written whole, then renamed
            np.save(tmp, blocks[i].cpu().numpy())
            os.replace(tmp, p)
            done.add(p)
        return out
