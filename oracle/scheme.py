"""Compact fourth-order scheme and the discrete auxiliary problem -- oracle, test only.

L^(h) (Section 3.1, Eq. FD_scheme; Section 3.2.1, Eq. aux_FD_scheme), at node (m, n):

    (1/h^2)    [E + W + N + S - 4C]
  + (1/(6h^2)) [NE + NW + SE + SW + 4C - 2(E + W + N + S)]
  + (k^2/12)   [E + W + N + S + 8C]

Discrete AP (Section 3.2.1, Eqs. aux_FD_scheme, AP_bounds_top_bottom,
AP_bounds_right/left), with the sine transform along x (the paper's figure
rotated by 90 degrees):
  * interior rows: L^(h) u = g on M0;
  * u = 0 on the two sides x = const (AP_DIRX_SOMMY) or on all four sides
    (AP_DIRICHLET4); those nodes are not unknowns;
  * AP_DIRX_SOMMY: at the sides y = const, the local Sommerfeld condition
    du/dn + i k u = 0 (outward normal, the paper's sign) imposed at the half node
    between the last two node rows with equation-based O(h^4) corrections. At the
    top, with delta_m = u(m,N) - u(m,N-1), abar_m = (u(m,N) + u(m,N-1))/2 and D the
    undivided second difference along x:
        (1/h)[delta + D delta/24 + (k^2 h^2/24) delta]
      + i k [abar + D abar/8 + (k^2 h^2/8) abar] = 0,
    and the mirror image at the bottom (delta_m = u(m,0) - u(m,1)). The printed
    rows are dimensionally inconsistent (their i k bracket mixes a difference
    quotient with u); these rows are our own Taylor derivation of the same
    condition: du/dy = delta/h - (h^2/24) u_yyy and u = abar - (h^2/8) u_yy at the
    half node, with u_yy = -u_xx - k^2 u from the homogeneous equation (g = 0 next
    to the auxiliary boundary, Section 3.2.1).
  * AP_DIRX_SOMMY_PAPER: the Sommerfeld rows as printed (Eqs. AP_bounds_right/left), rotated,
    with the undefined u_{M-1/2} read as abar and the i k bracket's difference quotient read as
    abar, so that the bracket is dimensionally consistent:
        (1/h)[delta - D delta/6 - (k^2 h^2/24) delta] + i k [abar + D abar/2 + (k^2 h^2/8) abar] = 0.
    It is consistent with du/dn + i k u = 0 but only to O(h^2) (pinned); it exists to show that
    the range of P_gamma does not depend on the choice of these rows.

The unknowns are the nodes not fixed by a Dirichlet condition, in row-major
(n, m) order.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp

from workloads import AP_DIRICHLET4, AP_DIRX_SOMMY, AP_DIRX_SOMMY_PAPER


def apply_L(w, h, k):
    """L^(h) w on M0 (zero on the auxiliary boundary), written as the three brackets of
    Eq. FD_scheme. w is a [ny, nx] array (real or complex)."""
    out = np.zeros_like(w)
    C = w[1:-1, 1:-1]
    E, W = w[1:-1, 2:], w[1:-1, :-2]
    N, S = w[2:, 1:-1], w[:-2, 1:-1]
    NE, NW, SE, SW = w[2:, 2:], w[2:, :-2], w[:-2, 2:], w[:-2, :-2]
    edges = E + W + N + S
    out[1:-1, 1:-1] = ((edges - 4.0 * C) / h**2
                       + (NE + NW + SE + SW + 4.0 * C - 2.0 * edges) / (6.0 * h**2)
                       + (k**2 / 12.0) * (edges + 8.0 * C))
    return out


def apply_dL_dk(w, h, k):
    """d L^(h) / dk applied to w: (k/6)(E + W + N + S + 8C) on M0."""
    out = np.zeros_like(w)
    C = w[1:-1, 1:-1]
    edges = w[1:-1, 2:] + w[1:-1, :-2] + w[2:, 1:-1] + w[:-2, 1:-1]
    out[1:-1, 1:-1] = (k / 6.0) * (edges + 8.0 * C)
    return out


def unknown_mask(sub):
    """Nodes that are unknowns of the discrete AP."""
    m = np.ones((sub.ny, sub.nx), dtype=bool)
    m[:, 0] = m[:, -1] = False           # u = 0 at x = const (both AP types)
    if sub.ap_bc == AP_DIRICHLET4:
        m[0, :] = m[-1, :] = False       # and at y = const
    elif sub.ap_bc not in (AP_DIRX_SOMMY, AP_DIRX_SOMMY_PAPER):
        raise ValueError("unknown AP type")
    return m


def _stencil_entries(sub, k, deriv=False):
    """(row_node, col_node, value) triples of the interior rows on M0.

    deriv=False: the 9-point L^(h); deriv=True: its derivative in k."""
    h = sub.h
    if not deriv:
        c_edge = 1.0 / h**2 - 2.0 / (6.0 * h**2) + k**2 / 12.0
        c_corner = 1.0 / (6.0 * h**2)
        c_centre = -4.0 / h**2 + 4.0 / (6.0 * h**2) + 8.0 * k**2 / 12.0
    else:
        c_edge, c_corner, c_centre = k / 6.0, 0.0, 8.0 * k / 6.0
    ny, nx = sub.ny, sub.nx
    nn, mm = np.meshgrid(np.arange(1, ny - 1), np.arange(1, nx - 1), indexing="ij")
    nn, mm = nn.ravel(), mm.ravel()
    rows, cols, vals = [], [], []
    for dn in (-1, 0, 1):
        for dm in (-1, 0, 1):
            nb = abs(dn) + abs(dm)
            c = c_centre if nb == 0 else (c_edge if nb == 1 else c_corner)
            if c == 0.0:
                continue
            rows.append((nn, mm))
            cols.append((nn + dn, mm + dm))
            vals.append(np.full(nn.size, c, dtype=complex))
    return rows, cols, vals


def sommerfeld_row_weights(h, k, deriv=False, paper=False):
    """Weights of the Sommerfeld row on (delta, D delta, abar, D abar):
    row = wd*delta + wdd*D(delta) + wa*abar + wda*D(abar). deriv=True gives d/dk.
    paper=True: the printed rows (AP_DIRX_SOMMY_PAPER)."""
    if paper:
        if not deriv:
            wd = (1.0 / h) * (1.0 - k**2 * h**2 / 24.0)
            wdd = -(1.0 / h) / 6.0
            wa = 1j * k * (1.0 + k**2 * h**2 / 8.0)
            wda = 1j * k / 2.0
        else:
            wd = -(1.0 / h) * (2.0 * k * h**2 / 24.0)
            wdd = 0.0
            wa = 1j * (1.0 + 3.0 * k**2 * h**2 / 8.0)
            wda = 1j / 2.0
        return wd, wdd, wa, wda
    if not deriv:
        wd = (1.0 / h) * (1.0 + k**2 * h**2 / 24.0)
        wdd = (1.0 / h) / 24.0
        wa = 1j * k * (1.0 + k**2 * h**2 / 8.0)
        wda = 1j * k / 8.0
    else:
        wd = (1.0 / h) * (2.0 * k * h**2 / 24.0)
        wdd = 0.0
        wa = 1j * (1.0 + 3.0 * k**2 * h**2 / 8.0)
        wda = 1j / 8.0
    return wd, wdd, wa, wda


def _sommerfeld_entries(sub, k, deriv=False):
    """(row_node, col_node, value) triples of the Sommerfeld rows at n = 0 and n = ny-1."""
    wd, wdd, wa, wda = sommerfeld_row_weights(sub.h, k, deriv, paper=sub.ap_bc == AP_DIRX_SOMMY_PAPER)
    nx, ny = sub.nx, sub.ny
    rows, cols, vals = [], [], []
    for (nb, ni) in ((ny - 1, ny - 2), (0, 1)):   # (boundary row, its inner neighbour)
        for m in range(1, nx - 1):
            # delta_j = u(j, nb) - u(j, ni); abar_j = (u(j, nb) + u(j, ni))/2, for j = m-1, m, m+1
            for dm, wgt_delta, wgt_abar in ((0, wd - 2.0 * wdd, wa - 2.0 * wda),
                                            (-1, wdd, wda), (1, wdd, wda)):
                j = m + dm
                for node_n, sgn in ((nb, 1.0), (ni, -1.0)):
                    rows.append((nb, m))
                    cols.append((node_n, j))
                    vals.append(sgn * wgt_delta + 0.5 * wgt_abar)
    return rows, cols, vals


def assemble(sub, k=None, deriv=False):
    """Sparse AP matrix A (or dA/dk with deriv=True) over the unknown nodes, CSC, complex128.

    Returns (A, unknown_mask, index_map) with index_map[n, m] = unknown number or -1."""
    k = sub.k if k is None else k
    U = unknown_mask(sub)
    idx = -np.ones(U.shape, dtype=np.int64)
    idx[U] = np.arange(U.sum())
    R, C, V = [], [], []
    rows, cols, vals = _stencil_entries(sub, k, deriv)
    for (rn, rm), (cn, cm), v in zip(rows, cols, vals):
        keep = U[cn, cm]
        R.append(idx[rn, rm][keep])
        C.append(idx[cn, cm][keep])
        V.append(v[keep])
    if sub.ap_bc in (AP_DIRX_SOMMY, AP_DIRX_SOMMY_PAPER):
        rows, cols, vals = _sommerfeld_entries(sub, k, deriv)
        for (rn, rm), (cn, cm), v in zip(rows, cols, vals):
            if U[cn, cm]:
                R.append(np.array([idx[rn, rm]]))
                C.append(np.array([idx[cn, cm]]))
                V.append(np.array([v], dtype=complex))
    n = int(U.sum())
    A = sp.coo_matrix((np.concatenate(V), (np.concatenate(R), np.concatenate(C))), shape=(n, n))
    return A.tocsc(), U, idx
