"""G^(h), difference potentials, P_gamma and Q columns, and their adjoint -- oracle, test only.

Definitions followed:
  * G^(h): u = G^(h) g solves the discrete AP with right-hand side g on M0
    (Section 3.2.1, after Eq. AP_bounds_left). Here: one SuperLU factorisation of
    the assembled sparse matrix (scipy.sparse.linalg.splu, partial pivoting).
  * Difference potential (Section 3.2.2, Eq. Potential_def):
        P_N+ xi = w - G^(h)( L^(h) w |_{M+} ),  w = xi on gamma, 0 elsewhere.
  * P_gamma xi = (P_N+ xi)|_gamma (Eq. def_Pgamma).
  * Q column (Section 3.2.5, Eq. Q_construction): (P_gamma - I) Ex^(H) Psi_j
    = -Tr_gamma G^(h)(L^(h) w|_{M+}).

Adjoint of out = (P_gamma - I) xi  (Q kind) or P_gamma xi (P kind), for a real loss
with cotangent c = dLoss/d conj(out) (the torch convention):
  grad_xi = -W^T L^T R^T G^H Tr^T c   (+ c for the P kind),
  dLoss/dk = Re sum_b [ <mu_b, A' u_b> - <E^T mu_b, R(L' w_b + L w'_b)> ]  (+ Re<c_b, xi'_b>, P kind)
with mu_b = A^{-H} Tr^T c_b, u_b = A^{-1} E r_b, A' = dA/dk, L' = dL/dk, w' the
k-derivative of the extension (basis columns only), <a, b> = sum conj(a) b.
"""
from __future__ import annotations

import numpy as np
from scipy.sparse.linalg import splu

from .extension import basis_column
from .grid import grid_sets
from .scheme import apply_L, apply_dL_dk, assemble


class APSystem:
    """Discrete AP of one subdomain at wavenumber k, factored once."""

    def __init__(self, sub, k=None):
        self.sub = sub
        self.k = float(sub.k if k is None else k)
        self.A, self.U, self.idx = assemble(sub, self.k)
        self.lu = splu(self.A)
        self._luH = None
        self.gs = grid_sets(sub)
        M0 = np.zeros_like(self.U)
        M0[1:-1, 1:-1] = True
        self.M0 = M0

    @property
    def n_gamma(self):
        return self.gs.gamma_n.size

    def luH(self):
        if self._luH is None:
            self._luH = splu(self.A.conj().T.tocsc())
        return self._luH

    def solve(self, g):
        """u = G^(h) g for g given on the [ny, nx] grid (values on M0 are used)."""
        b = np.zeros(self.A.shape[0], dtype=complex)
        b[self.idx[self.M0]] = g[self.M0]
        u = np.zeros(self.U.shape, dtype=complex)
        u[self.U] = self.lu.solve(b)
        return u

    def solve_adjoint(self, y):
        """A^{-H} y for y given on the unknown nodes of the [ny, nx] grid."""
        out = np.zeros(self.U.shape, dtype=complex)
        out[self.U] = self.luH().solve(y[self.U].astype(complex))
        return out

    def embed(self, xi):
        """w = xi on gamma, 0 elsewhere."""
        w = np.zeros(self.U.shape, dtype=complex)
        w[self.gs.gamma_n, self.gs.gamma_m] = xi
        return w

    def residual(self, w, k=None):
        """r = L^(h) w restricted to M+."""
        r = apply_L(w, self.sub.h, self.k if k is None else k)
        r[~self.gs.Mp] = 0.0
        return r

    def trace(self, u):
        return u[self.gs.gamma_n, self.gs.gamma_m]

    def potential(self, xi):
        """P_N+ xi on the whole grid (Eq. Potential_def)."""
        w = self.embed(xi)
        return w - self.solve(self.residual(w))

    def apply(self, xi, kind="Q"):
        """(P_gamma - I) xi (kind 'Q') or P_gamma xi (kind 'P') for one density on gamma."""
        u = self.solve(self.residual(self.embed(xi)))
        tr = self.trace(u)
        return -tr if kind == "Q" else xi - tr

    def basis_density(self, col, dk=False):
        return basis_column(self.gs, self.k, self.sub.n_modes, col, dk=dk)

    def columns(self, cols=None, kind="Q", xi=None):
        """Projection columns as an array [n_cols, |gamma|]: of the basis columns
        Ex^(H) Psi_col (xi None) or of the given densities xi[n_cols, |gamma|]."""
        if xi is not None:
            return np.stack([self.apply(x, kind) for x in xi])
        cols = range(8 * self.sub.n_modes) if cols is None else cols
        return np.stack([self.apply(self.basis_density(c), kind) for c in cols])

    def mplus_range(self):
        """(mlo, mhi, nlo, nhi): the node rectangle of M+."""
        cols = np.nonzero(self.gs.Mp.any(axis=0))[0]
        rows = np.nonzero(self.gs.Mp.any(axis=1))[0]
        return cols[0], cols[-1], rows[0], rows[-1]

    def receivers(self, row, cols=None, xi=None):
        """Difference potential P_N+ xi (Eq. Potential_def) at the nodes (row, m), m = mlo+1 ..
        mhi-1, for the basis columns (xi None) or given densities: array [n_cols, Px - 2]."""
        mlo, mhi, _, _ = self.mplus_range()
        if xi is None:
            cols = range(8 * self.sub.n_modes) if cols is None else cols
            xi = [self.basis_density(c) for c in cols]
        return np.stack([self.potential(x)[row, mlo + 1:mhi] for x in xi])

    def pgamma_matrix(self):
        """Dense P_gamma (|gamma| x |gamma|), one solve per unit density."""
        n = self.n_gamma
        P = np.zeros((n, n), dtype=complex)
        e = np.zeros(n)
        for i in range(n):
            e[:] = 0.0
            e[i] = 1.0
            P[:, i] = self.apply(e, "P")
        return P

    def adjoint(self, cot, kind="Q", xi=None, cols=None, cot_rec=None, rec_row=None):
        """(grad_xi, dLoss/dk) for out = columns(cols, kind, xi) and cotangent cot[n_cols, |gamma|];
        with cot_rec[n_cols, Px - 2] also the receiver output receivers(rec_row, ...), which is
        -R_rec G^(h) L^(h) w as well (w = 0 at the receivers), so its cotangent joins Tr^T cot."""
        gs = self.gs
        h, k = self.sub.h, self.k
        dA = assemble(self.sub, k, deriv=True)[0]
        if xi is None:
            cols = list(range(8 * self.sub.n_modes)) if cols is None else list(cols)
            dens = [self.basis_density(c) for c in cols]
            ddens = [self.basis_density(c, dk=True) for c in cols]
        else:
            dens = list(xi)
            ddens = [None] * len(dens)
        grad_xi = np.zeros((len(dens), self.n_gamma), dtype=complex)
        grad_k = 0.0
        for b, (x, dx) in enumerate(zip(dens, ddens)):
            c = cot[b]
            y = np.zeros(self.U.shape, dtype=complex)
            y[gs.gamma_n, gs.gamma_m] = c              # Tr^T c
            if cot_rec is not None:
                mlo, mhi, _, _ = self.mplus_range()
                y[rec_row, mlo + 1:mhi] += cot_rec[b]    # R_rec^T c_rec
            mu = self.solve_adjoint(y)                   # A^{-H} Tr^T c (on unknown nodes)
            v = np.where(gs.Mp, mu, 0.0)                 # R^T E^T mu
            g = -apply_L(v, h, k)[gs.gamma_n, gs.gamma_m]  # -W^T L^T R^T E^T mu (L symmetric, real)
            if kind == "P":
                g = g + c
            grad_xi[b] = g
            w = self.embed(x)
            u = self.solve(self.residual(w))
            Au = np.zeros(self.U.shape, dtype=complex)
            Au[self.U] = dA @ u[self.U]
            dr = apply_dL_dk(w, h, k)
            if dx is not None:
                dr = dr + apply_L(self.embed(dx), h, k)
            dr[~gs.Mp] = 0.0
            grad_k += np.real(np.vdot(mu[self.U], Au[self.U]) - np.vdot(v, dr))
            if kind == "P" and dx is not None:
                grad_k += np.real(np.vdot(c, dx))
        return grad_xi, grad_k
