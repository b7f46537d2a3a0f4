"""Boundary basis and equation-based extension -- oracle, test only.

Basis (Section 3.2.4, Eqs. basis_functions, Psi_def): on each side i = 1..4,
psi_j(s) = T_{j-1}(s), j = 1..M*, with s in [-1, 1] the affine side parameter.
Column order of Q (Eq. Q_construction): first the Dirichlet pairs (psi, 0) for
side 1..4 x j = 1..M*, then the Neumann pairs (0, psi) in the same order; column
c = kind*4M* + (side-1)*M* + (j-1).

Extension Ex^(H) (Section 3.2.3, Eqs. general_extension, cartesian_extension,
f = 0): with rho the signed distance along the outward normal of the owner side and
xi0, xi1 the Dirichlet and outward-Neumann data (tangential derivatives taken in
arc length, i.e. d/ds scaled by (2/L)^p),

  v = xi0 + rho xi1 + rho^2/2 (-xi0'' - k^2 xi0) + rho^3/6 (-xi1'' - k^2 xi1)
      + rho^4/24 (xi0'''' + 2 k^2 xi0'' + k^4 xi0).

Chebyshev values and derivatives come from numpy.polynomial.chebyshev
(chebval / chebder), a library routine.
"""
from __future__ import annotations

import numpy as np
from numpy.polynomial import chebyshev as C


def extend(rho, k, d0, d0_2, d0_4, d1, d1_2):
    """Ex^(H) at distance rho from data xi0 (d0), xi0'' (d0_2), xi0'''' (d0_4),
    xi1 (d1), xi1'' (d1_2) at the foot point (Eq. general_extension with f = 0)."""
    n2 = -d0_2 - k**2 * d0
    n3 = -d1_2 - k**2 * d1
    n4 = d0_4 + 2.0 * k**2 * d0_2 + k**4 * d0
    return d0 + rho * d1 + rho**2 / 2.0 * n2 + rho**3 / 6.0 * n3 + rho**4 / 24.0 * n4


def extend_dk(rho, k, d0, d0_2, d0_4, d1, d1_2):
    """d/dk of extend() at fixed data."""
    return (rho**2 / 2.0 * (-2.0 * k * d0) + rho**3 / 6.0 * (-2.0 * k * d1)
            + rho**4 / 24.0 * (4.0 * k * d0_2 + 4.0 * k**3 * d0))


def chebyshev_derivs(j, s, L):
    """T_{j-1}(s) and its 2nd and 4th derivatives in arc length along a side of length L."""
    c = np.zeros(j)
    c[j - 1] = 1.0
    t0 = C.chebval(s, c)
    t2 = C.chebval(s, C.chebder(c, 2)) * (2.0 / L) ** 2 if j > 2 else np.zeros_like(s)
    t4 = C.chebval(s, C.chebder(c, 4)) * (2.0 / L) ** 4 if j > 4 else np.zeros_like(s)
    return t0, t2, t4


def basis_column(gs, k, n_modes, col, dk=False):
    """xi_gamma = Ex^(H) Psi_col on gamma (real), or its k-derivative when dk=True."""
    kind, rest = divmod(col, 4 * n_modes)
    side, jm1 = divmod(rest, n_modes)
    side += 1
    sel = gs.owner == side
    out = np.zeros(gs.owner.size)
    t0, t2, t4 = chebyshev_derivs(jm1 + 1, gs.s[sel], gs.side_len[sel])
    z = np.zeros_like(t0)
    f = extend_dk if dk else extend
    if kind == 0:
        out[sel] = f(gs.rho[sel], k, t0, t2, t4, z, z)
    else:
        out[sel] = f(gs.rho[sel], k, z, z, z, t0, t2)
    return out


def extend_data(gs, k, data):
    """Ex^(H) of arbitrary boundary data. data(side, s, L) returns the tuple
    (xi0, xi0'', xi0'''', xi1, xi1'') at the foot points (arc-length derivatives)."""
    out = np.zeros(gs.owner.size, dtype=complex)
    for side in (1, 2, 3, 4):
        sel = gs.owner == side
        if not sel.any():
            continue
        d0, d0_2, d0_4, d1, d1_2 = data(side, gs.s[sel], gs.side_len[sel])
        out[sel] = extend(gs.rho[sel], k, d0, d0_2, d0_4, d1, d1_2)
    return out
