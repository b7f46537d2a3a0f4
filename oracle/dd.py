"""Domain-decomposition coupling for a layered strip of subdomains -- oracle, test only.

Subdomains Omega_j = [x0_j, x0_j + 1] x [0, 1] side by side along x (the paper's duct, Section 4),
each with its own wavenumber and auxiliary problem. Following Sections 3.3-3.5:
  * per subdomain the BEP  Q_j c_j = 0  (homogeneous equation, f = 0; Eq. linear_system_equations),
    with c_j = [c^(j,s,0) for sides s = 1..4 ; c^(j,s,1) for s = 1..4], M* Chebyshev
    coefficients each (Eq. Psi_def);
  * outer sides carry  alpha u + beta du/dn = phi  (Eq. helmholtz_robin), expanded in the same
    basis, phi = sum d_m psi_m, giving  alpha c^(0)_m + beta c^(1)_m = d_m  (Eq. BC_coefficients);
  * the interface between Omega_j (side 4, right) and Omega_{j+1} (side 3, left) carries
    continuity of u and of the flux:  c^(j,4,0) = c^(j+1,3,0),  c^(j,4,1) = -c^(j+1,3,1)
    (Section 3.3.2: the two outward normals are opposite);
  * the BC and interface equations are solved for one coefficient set per side and substituted
    (Section 3.3.3), leaving 16 M* unknowns for four subdomains; the stacked system is solved
    in the least-squares sense (steps 2(b)-(c) use QR; numpy.linalg.lstsq gives the same
    minimiser);
  * the solution inside is the difference potential of the extended boundary data, u = P_N+ xi
    (Eq. potential_solution_homo), evaluated here at receiver nodes.
The Chebyshev coefficients of the boundary data come from numpy.polynomial.chebyshev.
chebinterpolate (a library routine)."""
from __future__ import annotations

import numpy as np
from numpy.polynomial import chebyshev as C

from .projection import APSystem


def side_points(sub, side, s):
    """(x, y) of the side parameter s in [-1, 1] (sides 1 bottom, 2 top, 3 left, 4 right)."""
    if side in (1, 2):
        return sub.x0 + (s + 1) / 2 * (sub.x1 - sub.x0), np.full_like(s, sub.y0 if side == 1 else sub.y1)
    return np.full_like(s, sub.x0 if side == 3 else sub.x1), sub.y0 + (s + 1) / 2 * (sub.y1 - sub.y0)


def cheb_coeffs(f, n_modes):
    """Chebyshev coefficients (degree n_modes - 1 interpolant) of a complex function on [-1, 1]."""
    return C.chebinterpolate(lambda s: f(s).real, n_modes - 1) + 1j * C.chebinterpolate(lambda s: f(s).imag, n_modes - 1)


class Strip:
    """DD solve of a strip of subdomains. bc(j, side) -> (alpha, beta, phi(s)) gives the outer
    boundary condition of side `side` of subdomain j as a function of the side parameter s.
    source(j) -> fun or None: the source of subdomain j, fun(x, y) -> (f, f_x, f_y, f_xx, f_yy)
    (Delta u + k^2 u = f); it adds F_j to the right-hand side of Q_j c_j = F_j and G B f to the
    solution (oracle/source.py)."""

    def __init__(self, subdomains, bc, source=None, positions=None):
        self.subs = list(subdomains)
        self.bc = bc
        self.source = source
        self.M = self.subs[0].n_modes
        self.N = len(self.subs)
        # cell (i, j) of every subdomain in a rectangular layout (Section 3.4: subdomains that
        # share whole sides); default: a strip along x
        self.pos = [tuple(p) for p in positions] if positions is not None else [(j, 0) for j in range(self.N)]
        self.at = {p: j for j, p in enumerate(self.pos)}

    def neighbour(self, j, side):
        i, jj = self.pos[j]
        d = {1: (0, -1), 2: (0, 1), 3: (-1, 0), 4: (1, 0)}[side]
        return self.at.get((i + d[0], jj + d[1]))

    def outer(self, j, side):
        return self.neighbour(j, side) is None

    def iface(self, j, side):
        """(key, sign) of the interface on side `side` of subdomain j: the left/bottom subdomain
        names it (its side 4 or 2), and the two outward normals are opposite, so c^(1) enters with
        + on that side and - on the neighbour's (Section 3.3.2)."""
        if side in (4, 2):
            return (j, side), 1.0
        nb = self.neighbour(j, side)
        return (nb, 4 if side == 3 else 2), -1.0

    def unknown_map(self):
        """Column offsets of the unknowns: one block of M per outer side (its c^(0), or c^(1) on a
        Dirichlet side), and two blocks (X, Y) per interface."""
        off, idx = 0, {}
        for j in range(self.N):
            for side in (1, 2, 3, 4):
                if self.outer(j, side):
                    idx[(j, side)] = off
                    off += self.M
            for side in (4, 2):
                if not self.outer(j, side):
                    idx[("if", j, side)] = off
                    off += 2 * self.M
        return idx, off

    def assemble(self, Qs, Fs=None):
        """Global least-squares system A x = b from the per-subdomain Q_j [|gamma_j|, 8M] and the
        right-hand sides F_j of Q_j c_j = F_j (zero without a source)."""
        M = self.M
        idx, n = self.unknown_map()
        rows = sum(Q.shape[0] for Q in Qs)
        A = np.zeros((rows, n), complex)
        b = np.zeros(rows, complex)
        r0 = 0
        for j, Q in enumerate(Qs):
            g = Q.shape[0]
            if Fs is not None and Fs[j] is not None:
                b[r0:r0 + g] += Fs[j]
            blk = lambda side, kind: Q[:, kind * 4 * M + (side - 1) * M: kind * 4 * M + side * M]
            for side in (1, 2, 3, 4):
                Q0, Q1 = blk(side, 0), blk(side, 1)
                if self.outer(j, side):
                    alpha, beta, phi = self.bc(j, side)
                    d = cheb_coeffs(phi, M)
                    c = idx[(j, side)]
                    if beta != 0:       # c1 = (d - alpha c0) / beta, unknown c0
                        A[r0:r0 + g, c:c + M] += Q0 - (alpha / beta) * Q1
                        b[r0:r0 + g] -= Q1 @ (d / beta)
                    else:               # Dirichlet: c0 = d / alpha, unknown c1
                        A[r0:r0 + g, c:c + M] += Q1
                        b[r0:r0 + g] -= Q0 @ (d / alpha)
                else:
                    key, sgn = self.iface(j, side)
                    c = idx[("if",) + key]
                    A[r0:r0 + g, c:c + M] += Q0                 # X
                    A[r0:r0 + g, c + M:c + 2 * M] += sgn * Q1   # +Y on the naming subdomain, -Y on the other
            r0 += g
        return A, b

    def coefficients(self, x):
        """Per-subdomain coefficient vectors c_j [8M] from the unknowns."""
        M = self.M
        idx, _ = self.unknown_map()
        cs = []
        for j in range(self.N):
            c = np.zeros(8 * M, complex)
            for side in (1, 2, 3, 4):
                sl0 = slice((side - 1) * M, side * M)
                sl1 = slice(4 * M + (side - 1) * M, 4 * M + side * M)
                if self.outer(j, side):
                    alpha, beta, phi = self.bc(j, side)
                    d = cheb_coeffs(phi, M)
                    u = x[idx[(j, side)]: idx[(j, side)] + M]
                    if beta != 0:
                        c[sl0], c[sl1] = u, (d - alpha * u) / beta
                    else:
                        c[sl0], c[sl1] = d / alpha, u
                else:
                    key, sgn = self.iface(j, side)
                    o = idx[("if",) + key]
                    c[sl0] = x[o:o + M]
                    c[sl1] = sgn * x[o + M:o + 2 * M]
            cs.append(c)
        return cs

    def solve(self, rec_rows):
        """Coefficients and the solution at the receivers (row rec_rows[j], m = mlo+1 .. mhi-1)."""
        from .source import source_foot_data, source_on_grid, source_terms
        systems = [APSystem(s) for s in self.subs]
        Qs = [S.columns().T for S in systems]   # [|gamma|, 8M]
        Fs, Us = [], []
        for j, (S, sub) in enumerate(zip(systems, self.subs)):
            fun = self.source(j) if self.source is not None else None
            if fun is None:
                Fs.append(None)
                Us.append(None)
                continue
            F, ub = source_terms(S, source_on_grid(sub, fun), source_foot_data(S.gs, sub, fun))
            Fs.append(F)
            Us.append(ub)
        A, b = self.assemble(Qs, Fs)
        x = np.linalg.lstsq(A, b, rcond=None)[0]
        cs = self.coefficients(x)
        urec = []
        for S, r, c, ub in zip(systems, rec_rows, cs, Us):
            u = S.receivers(r).T @ c
            if ub is not None:
                mlo, mhi, _, _ = S.mplus_range()
                u = u + ub[r, mlo + 1:mhi]
            urec.append(u)
        return cs, urec, (A, b, x)
