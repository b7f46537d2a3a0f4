"""Grid sets of the Method of Difference Potentials (Section 3.2.2) -- oracle, test only.

Nodes of the auxiliary grid N0 are (m, n), m = 0..nx-1 along x, n = 0..ny-1 along y,
at x_m = ax0 + m*h, y_n = ay0 + n*h. Grid functions are numpy arrays indexed
[n, m] (row-major in y, then x), flattened index n*nx + m.

  M0   nodes strictly interior to the auxiliary rectangle (not on its boundary)
  M+   M0 nodes strictly inside the open subdomain Omega
  M-   M0 \\ M+
  N+   all nodes touched by the 3x3 stencil centred on an M+ node
  N-   the same for M-
  gamma = N+ intersected with N-   (the grid boundary)

gamma is listed in row-major (n, m) order; that order is the row order of every
projection column.

Side ownership of a gamma node (the paper is silent near corners): the side with
the smallest |rho|, where rho is the signed distance to the side's line, positive
outside Omega; distances within 1e-9*h of each other count as a tie, and ties go
to the lower side index. Sides: 1 = bottom (y = y0),
2 = top (y = y1), 3 = left (x = x0), 4 = right (x = x1). The foot-point parameter
s in [-1, 1] runs with x on sides 1-2 and with y on sides 3-4.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np


TIE_TOL = 1e-9


def node_coordinates(sub):
    """x_m = ax0 + m*h and y_n = ay0 + n*h (fp64, no fused multiply-add)."""
    x = np.array([sub.ax0 + float(m) * sub.h for m in range(sub.nx)])
    y = np.array([sub.ay0 + float(n) * sub.h for n in range(sub.ny)])
    return x, y


def _dilate3x3(mask):
    """Union of the 3x3 neighbourhoods of the True nodes (clipped to the grid)."""
    ny, nx = mask.shape
    out = np.zeros_like(mask)
    for dn in (-1, 0, 1):
        for dm in (-1, 0, 1):
            src = mask[max(0, -dn):ny - max(0, dn), max(0, -dm):nx - max(0, dm)]
            out[max(0, dn):ny - max(0, -dn), max(0, dm):nx - max(0, -dm)] |= src
    return out


@dataclass
class GridSets:
    M0: np.ndarray      # bool [ny, nx]
    Mp: np.ndarray
    Mm: np.ndarray
    Np: np.ndarray
    Nm: np.ndarray
    gamma: np.ndarray   # bool [ny, nx]
    gamma_n: np.ndarray  # int, row-major order
    gamma_m: np.ndarray
    owner: np.ndarray    # side 1..4 per gamma node
    rho: np.ndarray      # signed distance to the owner side's line, > 0 outside
    s: np.ndarray        # foot-point parameter on the owner side
    side_len: np.ndarray  # length of the owner side


def grid_sets(sub) -> GridSets:
    """Classify the nodes as Section 3.2.2 states (strict inequalities for M+)."""
    x, y = node_coordinates(sub)
    X, Y = np.meshgrid(x, y)  # [ny, nx]
    ny, nx = sub.ny, sub.nx
    M0 = np.zeros((ny, nx), dtype=bool)
    M0[1:ny - 1, 1:nx - 1] = True
    inside = (X > sub.x0) & (X < sub.x1) & (Y > sub.y0) & (Y < sub.y1)
    Mp = M0 & inside
    Mm = M0 & ~Mp
    Np = _dilate3x3(Mp)
    Nm = _dilate3x3(Mm)
    gamma = Np & Nm
    gn, gm = np.nonzero(gamma)  # row-major: sorted by n, then m
    gx, gy = x[gm], y[gn]
    rhos = np.stack([sub.y0 - gy, gy - sub.y1, sub.x0 - gx, gx - sub.x1])  # sides 1..4
    dist = np.abs(rhos)
    # first side whose |rho| is within TIE_TOL*h of the smallest one
    near = dist <= dist.min(axis=0) + TIE_TOL * sub.h
    owner = np.argmax(near, axis=0) + 1
    rho = rhos[owner - 1, np.arange(gn.size)]
    lx, ly = sub.x1 - sub.x0, sub.y1 - sub.y0
    s_h = 2.0 * (gx - sub.x0) / lx - 1.0
    s_v = 2.0 * (gy - sub.y0) / ly - 1.0
    s = np.where(owner <= 2, s_h, s_v)
    side_len = np.where(owner <= 2, lx, ly)
    return GridSets(M0, Mp, Mm, Np, Nm, gamma, gn, gm, owner, rho, s, side_len)
