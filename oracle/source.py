"""The inhomogeneous terms of the method, for a source f -- oracle, test only.

Helmholtz with a source, Delta u + k^2 u = f (Eq. helmholtz), adds three terms to the
homogeneous path:

  * the right-hand side of the compact scheme, g = B^(h) f (Eq. rhs_g): on interior nodes
    B f = f + (f_{m+1,n} + f_{m-1,n} + f_{m,n+1} + f_{m,n-1} - 4 f_{m,n}) / 12, and g = 0 on the
    outermost nodes of the auxiliary grid (Section 3.2.1);
  * the inhomogeneous part of the extension (Eqs. extension_split, cartesian_extension): the
    source terms of the equation-based normal derivatives at the foot point on the owner side,
    Ex^(I) f = rho^2/2 f + rho^3/6 d_n f + rho^4/24 (d_nn f - d_tt f - k^2 f)
    (d_n along the outward normal, d_t along the side);
  * the right-hand side of the per-subdomain system Q c = F (Eq. linear_system_equations):
    F = (I - P_gamma) Ex^(I) f - Tr G^(h) B^(h) f.
The solution inside is u = P_N+ xi + G^(h) B^(h) f on N+ (Eq. potential_solution), with the
density xi = Ex^(H) (xi_0, xi_1) + Ex^(I) f: the source adds P_N+ Ex^(I) f + G^(h) B^(h) f.

B^(h) f enters G^(h) restricted to M+: the discrete Green's formula behind Eqs. discrete_BEP
and potential_solution holds for a solution of L^(h) u = g on M+, and only g on M+ takes part
(a right-hand side on M- would add G of it, which is not a trace of an interior solution).
"""
from __future__ import annotations

import numpy as np

from .dd import side_points


def apply_B(f):
    """g = B^(h) f on the interior nodes of the grid f[ny, nx], 0 on the outermost nodes."""
    g = np.zeros_like(f, dtype=complex)
    c = f[1:-1, 1:-1]
    g[1:-1, 1:-1] = c + (f[1:-1, 2:] + f[1:-1, :-2] + f[2:, 1:-1] + f[:-2, 1:-1] - 4.0 * c) / 12.0
    return g


def source_on_grid(sub, fun):
    """f on every node of the auxiliary grid; fun(x, y) -> (f, f_x, f_y, f_xx, f_yy)."""
    x = sub.ax0 + np.arange(sub.nx) * sub.h
    y = sub.ay0 + np.arange(sub.ny) * sub.h
    X, Y = np.meshgrid(x, y)
    return np.asarray(fun(X, Y)[0], dtype=complex)


def source_foot_data(gs, sub, fun):
    """[|gamma|, 4] complex: f, d_n f, d_nn f, d_tt f at the foot point of every gamma node on its
    owner side (1 bottom, 2 top: n = -y, +y; 3 left, 4 right: n = -x, +x)."""
    out = np.zeros((gs.owner.size, 4), dtype=complex)
    for side in (1, 2, 3, 4):
        sel = gs.owner == side
        if not sel.any():
            continue
        x, y = side_points(sub, side, gs.s[sel])
        f, fx, fy, fxx, fyy = (np.asarray(v, dtype=complex) * np.ones_like(x) for v in fun(x, y))
        if side in (1, 2):
            sgn = -1.0 if side == 1 else 1.0
            out[sel] = np.stack([f, sgn * fy, fyy, fxx], axis=1)
        else:
            sgn = -1.0 if side == 3 else 1.0
            out[sel] = np.stack([f, sgn * fx, fxx, fyy], axis=1)
    return out


def extend_source(gs, k, src4):
    """Ex^(I) f on gamma from the foot data [|gamma|, 4] (f, d_n f, d_nn f, d_tt f)."""
    rho = gs.rho
    f, fn, fnn, ftt = src4.T
    return rho**2 / 2.0 * f + rho**3 / 6.0 * fn + rho**4 / 24.0 * (fnn - ftt - k**2 * f)


def source_terms(S, fgrid, src4):
    """(F on gamma, the source's part of the solution P_N+ Ex^(I) f + G (B f)|M+ on the grid)
    for the APSystem S."""
    ub = S.solve(np.where(S.gs.Mp, apply_B(fgrid), 0.0))
    xi_i = extend_source(S.gs, S.k, src4)
    F = -S.apply(xi_i, kind="Q") - S.trace(ub)
    return F, S.potential(xi_i) + ub
