"""Seeded synthetic inputs shaped like the paper's workloads.

This module is shared by the CPU oracle (``oracle/``) and by the CUDA path
(``paper_2103_12172_gb300``): it describes subdomain geometries, grids,
wavenumbers and random right-hand sides, and holds none of the method's
arithmetic (no stencils, no extension, no solves).

Geometry (the paper's experiments, Section 4): unit-square subdomains, each
embedded in its own square auxiliary domain enlarged by 0.1 on every side, with
a uniform grid of ``n`` nodes per side, ``h = 1.2 / (n - 1)``. The paper uses
side-2 squares in side-2.2 auxiliary domains; the unit-square version is the
same configuration scaled by 1/2.

Auxiliary-problem boundary types (Section 3.2.1, rotated so that the sine
transform runs along x):
  AP_DIRICHLET4        -- u = 0 on all four sides of the auxiliary rectangle;
  AP_DIRX_SOMMY        -- u = 0 at x = const, local Sommerfeld rows at y = const (the O(h^4)
                          half-node rows of our own derivation);
  AP_DIRX_SOMMY_PAPER  -- the same with the Sommerfeld rows as printed in the paper (Eqs.
                          AP_bounds_right/left), read with u_{M-1/2} = the half-node mean.
"""
from __future__ import annotations

import dataclasses
from dataclasses import dataclass

import numpy as np

AP_DIRICHLET4 = 0
AP_DIRX_SOMMY = 1
AP_DIRX_SOMMY_PAPER = 2


@dataclass(frozen=True)
class Subdomain:
    """One subdomain Omega_i and its auxiliary problem (Section 3.2.1-3.2.2).

    x0, x1, y0, y1 : open rectangle Omega_i
    ax0, ay0, h    : lower-left corner of the auxiliary grid and its step
    nx, ny         : nodes of the auxiliary grid along x and y
    k              : real wavenumber on Omega_i
    ap_bc          : AP_DIRICHLET4, AP_DIRX_SOMMY or AP_DIRX_SOMMY_PAPER
    n_modes        : M*, Chebyshev modes per side (Section 3.2.4)
    """
    x0: float
    x1: float
    y0: float
    y1: float
    ax0: float
    ay0: float
    h: float
    nx: int
    ny: int
    k: float
    ap_bc: int
    n_modes: int

    def with_k(self, k: float) -> "Subdomain":
        return dataclasses.replace(self, k=float(k))


def unit_subdomain(i: int, j: int, n: int, k: float, ap_bc: int, n_modes: int,
                   margin: float = 0.1) -> Subdomain:
    """Unit square [i, i+1] x [j, j+1] inside [i-margin, i+1+margin] x [j-margin, j+1+margin]."""
    nc = n - 1
    h = (1.0 + 2.0 * margin) / nc
    return Subdomain(float(i), float(i + 1), float(j), float(j + 1),
                     float(i) - margin, float(j) - margin, h, n, n, float(k), int(ap_bc), int(n_modes))


@dataclass(frozen=True)
class Workload:
    name: str
    subdomains: tuple
    description: str

    @property
    def n_columns(self) -> int:
        return sum(8 * s.n_modes for s in self.subdomains)


def single_129() -> Workload:
    """One unit subdomain, 129 x 129 auxiliary grid, k = 10, Dirichlet AP on all
    sides, 16 Chebyshev modes per side: 4 sides x 16 x {Dirichlet, Neumann} = 128 columns."""
    return Workload("single_129_k10_dir4_m16",
                    (unit_subdomain(0, 0, 129, 10.0, AP_DIRICHLET4, 16),),
                    "1 subdomain, 129^2 AP grid, k=10, Dirichlet AP, M*=16, 128 columns")


def dd2x2_257() -> Workload:
    """2 x 2 decomposition of [0,2]^2, 257 x 257 auxiliary grid per subdomain, k = 30,
    mixed (Dirichlet-x / Sommerfeld-y) AP, 32 modes per side: 4 x 256 = 1024 columns."""
    subs = tuple(unit_subdomain(i, j, 257, 30.0, AP_DIRX_SOMMY, 32) for j in range(2) for i in range(2))
    return Workload("dd2x2_257_k30_m32", subs,
                    "2x2 subdomains of [0,2]^2, 257^2 AP grids, k=30, mixed AP, M*=32, 1024 columns")


def checker2x2() -> Workload:
    """2 x 2 checkerboard: k = 10 on 129^2 grids where i+j is even, k = 100 on 513^2
    grids where i+j is odd; mixed AP; 48 modes per side: 4 x 384 = 1536 columns."""
    subs = []
    for j in range(2):
        for i in range(2):
            if (i + j) % 2 == 0:
                subs.append(unit_subdomain(i, j, 129, 10.0, AP_DIRX_SOMMY, 48))
            else:
                subs.append(unit_subdomain(i, j, 513, 100.0, AP_DIRX_SOMMY, 48))
    return Workload("checker2x2_k10_129_k100_513_m48", tuple(subs),
                    "2x2 checkerboard, k=10 on 129^2 and k=100 on 513^2, mixed AP, M*=48, 1536 columns")


def grid_nodes_for_k(k: float) -> int:
    """Auxiliary-grid nodes for the 8 x 8 workload: N_c = clamp(2^ceil(log2(8k)), 256, 1024)."""
    nc = int(np.clip(2 ** np.ceil(np.log2(8.0 * k)), 256, 1024))
    return nc + 1


def dd8x8_mixed(seed: int = 7) -> Workload:
    """8 x 8 decomposition of [0,8]^2, k ~ U[20, 80] from numpy default_rng(seed) in
    row-major subdomain order, grids 257^2 / 513^2 / 1025^2, mixed AP, 64 modes per side
    (64 x 512 = 32768 columns)."""
    ks = np.random.default_rng(seed).uniform(20.0, 80.0, 64)
    subs = []
    for j in range(8):
        for i in range(8):
            k = float(ks[j * 8 + i])
            subs.append(unit_subdomain(i, j, grid_nodes_for_k(k), k, AP_DIRX_SOMMY, 64))
    return Workload("dd8x8_k20to80_seed7_m64", tuple(subs),
                    "8x8 subdomains, k~U[20,80] seed 7, 257^2-1025^2 AP grids, mixed AP, M*=64, 32768 columns")


def strip4x1(k_init: float = 40.0, n_modes: int = 24) -> Workload:
    """4 x 1 layered strip [0,4] x [0,1], 129^2 auxiliary grid per subdomain, per-layer
    wavenumbers (all k_init), mixed AP, 24 modes per side (with 48 the stacked least-squares
    system of the coupling has condition ~1e11 on these grids)."""
    subs = tuple(unit_subdomain(i, 0, 129, k_init, AP_DIRX_SOMMY, n_modes) for i in range(4))
    return Workload(f"strip4x1_129_k40_m{n_modes}", subs,
                    f"4x1 layered strip, 129^2 AP grids, k_j=40 (parameters), mixed AP, M*={n_modes}")


def strip_targets(seed: int = 3):
    """Target wavenumbers of the layered strip: U[30, 60] from default_rng(seed)."""
    return np.random.default_rng(seed).uniform(30.0, 60.0, 4)


def small_subdomain(n: int, k: float, ap_bc: int, n_modes: int) -> Subdomain:
    """A unit subdomain on a small grid (for parity cases the oracle finishes fast)."""
    return unit_subdomain(0, 0, n, k, ap_bc, n_modes)


WORKLOADS = {
    "single_129": single_129,
    "dd2x2_257": dd2x2_257,
    "checker2x2": checker2x2,
    "dd8x8": dd8x8_mixed,
    "strip4x1": strip4x1,
}


def random_complex(shape, seed: int) -> np.ndarray:
    """Complex normal samples, real and imaginary parts ~ N(0, 1), numpy default_rng(seed)."""
    rng = np.random.default_rng(seed)
    return rng.standard_normal(shape) + 1j * rng.standard_normal(shape)
