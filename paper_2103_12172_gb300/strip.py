"""Layered strip: domain-decomposition coupling on top of the batched projection columns, and
its gradient with respect to the per-layer wavenumbers.

Subdomains Omega_j = [j, j+1] x [0, 1] (a duct, Section 4) with wavenumbers k_j. Per layer the
library computes Q_j = (P_gamma - I) Ex Psi (Section 3.2.5) and the difference potential of
every basis column at a receiver row (Eq. potential_solution_homo) in one batched pass. The
coupling follows Sections 3.3-3.5: outer sides carry alpha u + beta du/dn = phi expanded in the
Chebyshev basis (Eq. BC_coefficients), interfaces carry c^(0) continuous and c^(1) opposite
(Section 3.3.2); the BC and interface equations are eliminated (Section 3.3.3) and the stacked
system is solved in the least-squares sense by QR (steps 2(b)-(c)). The loss is the squared
misfit of the reconstructed solution at the receivers.

The coupling is small dense linear algebra (hundreds of unknowns) written with torch so that
autograd carries the chain rule; the AP solves, the projection columns, the receiver values and
their wavenumber derivatives run in libmdp (forward: mdp_project_batch_rec; backward:
mdp_ap_adjoint_rec).
"""
from __future__ import annotations

import math

import torch

from . import Plan, linalg


class ProjectWithReceivers(torch.autograd.Function):
    """(Q, receiver values) of the basis columns of every subdomain as functions of k."""

    @staticmethod
    def forward(ctx, k, plan):
        ks = [float(v) for v in k.detach().cpu().tolist()]
        if getattr(plan, "_k_current", None) != ks:
            plan.update_k(ks)
            plan._k_current = ks
        out, rec = plan.project(out_rec=True)
        ctx.plan, ctx.ks = plan, ks
        ctx.k_meta = (k.dtype, k.device)
        return out, rec

    @staticmethod
    def backward(ctx, g_out, g_rec):
        plan = ctx.plan
        if getattr(plan, "_k_current", None) != ctx.ks:
            plan.update_k(ctx.ks)
            plan._k_current = ctx.ks
        g_out = torch.zeros(plan.output_size, dtype=torch.complex128, device="cuda") if g_out is None else g_out
        g_rec = None if g_rec is None else g_rec.contiguous()
        _, gk = plan.adjoint(g_out.contiguous(), grad_xi=False, cot_rec=g_rec)
        dtype, device = ctx.k_meta
        return gk.to(dtype=dtype, device=device), None


def least_squares_grads(A, b, x, w, mm):
    """Gradients of the least-squares minimiser x of ||A x - b|| for the incoming gradient g,
    given w = (A^H A)^{-1} g: with r = b - A x, grad_b = A w and grad_A = r w^H - (A w) x^H.
    mm: the matrix-vector product to use."""
    Aw = mm(A, w)
    r = b - mm(A, x)
    grad_A = torch.outer(r, w.conj()) - torch.outer(Aw, x.conj())
    return grad_A, Aw


class LeastSquares(torch.autograd.Function):
    """x = argmin ||A x - b|| for a full-column-rank CUDA matrix A (m >= n) by Householder QR of
    the column-equilibrated A D (Section 3.5, steps 2(b)-(c); the scaling leaves the minimiser
    unchanged and improves the conditioning of R), all on libmdp's kernels: the QR
    (mdp_householder_qr, or the two-stage structured form when the row blocks are given), the
    triangular solves (mdp_triangular_solve) and the products (mdp_complex_matmul). The backward
    pass uses the closed form of the minimiser's derivative instead of differentiating the
    factorisation: w = (A^H A)^{-1} g = D R^{-1} R^{-H} D g for the incoming gradient g, then
    least_squares_grads."""

    @staticmethod
    def forward(ctx, A, b, blocks=None):
        if not A.is_cuda:
            raise TypeError("LeastSquares runs on libmdp's CUDA kernels: A must be a CUDA tensor")
        linalg.check_pending()                         # status words of earlier solves that have completed
        D = 1.0 / torch.linalg.vector_norm(A, dim=0)
        if blocks is not None:
            fac = linalg.structured_qr(A * D, b, *blocks)   # per-subdomain QRs, then the shared unknowns
        else:
            fac = linalg.householder_qr(A * D, b)
        linalg.defer_check(fac)                        # checked later, without stalling the stream
        x = D * fac.lstsq()
        ctx.fac = fac
        ctx.save_for_backward(A, b, x, D)
        return x

    @staticmethod
    def backward(ctx, g):
        A, b, x, D = ctx.saved_tensors
        w = D * ctx.fac.gram_solve((D * g).to(torch.complex128))
        grad_A, grad_b = least_squares_grads(A, b, x, w, linalg.matmul)
        return grad_A, grad_b, None


def cheb_coeffs(fvals, n):
    """Chebyshev coefficients of the degree n-1 interpolant from values at the n first-kind
    Chebyshev points x_i = cos(pi (i + 1/2) / n) (i = 0..n-1): c_m = (2/n) sum_i f(x_i) T_m(x_i),
    c_0 halved. fvals [n] complex (CUDA; the product runs on mdp_complex_matmul)."""
    i = torch.arange(n, dtype=torch.float64, device=fvals.device)
    m = torch.arange(n, dtype=torch.float64, device=fvals.device)
    T = torch.cos(m[:, None] * math.pi * (i[None, :] + 0.5) / n)   # T_m(x_i)
    c = (2.0 / n) * linalg.matmul(T, fvals)
    c[0] = c[0] / 2
    return c


def cheb_points(n, device):
    i = torch.arange(n, dtype=torch.float64, device=device)
    return torch.cos(math.pi * (i + 0.5) / n)


class LayeredStrip:
    """A rectangular layout of square subdomains that share whole sides (default: a strip
    along x; `positions[j]` = cell (i, j) of subdomain j otherwise, Section 3.4) with outer
    boundary data bc(j, side, k_j, x, y) -> (alpha, beta, phi values) (torch, differentiable in
    k_j), a receiver row per subdomain and optionally a source per subdomain."""

    def __init__(self, subdomains, bc, receiver_rows, tile_cols=0, source=None, positions=None):
        self.subs = list(subdomains)
        self.N = len(self.subs)
        self.M = self.subs[0].n_modes
        self.bc = bc
        self.source = source        # source(j) -> fun(x, y) -> (f, f_x, f_y, f_xx, f_yy), or None
        self._src_cache = {}
        self.pos = [tuple(p) for p in positions] if positions is not None else [(j, 0) for j in range(self.N)]
        self.at = {p: j for j, p in enumerate(self.pos)}
        self.plan = Plan(self.subs, tile_cols=tile_cols)
        self.plan.set_receivers(receiver_rows)
        self.layout = [self.plan.layout(j) for j in range(self.N)]
        self.rlayout = [self.plan.receiver_layout(j) for j in range(self.N)]

    def neighbour(self, j, side):
        i, jj = self.pos[j]
        di, dj = {1: (0, -1), 2: (0, 1), 3: (-1, 0), 4: (1, 0)}[side]
        return self.at.get((i + di, jj + dj))

    def outer(self, j, side):
        return self.neighbour(j, side) is None

    def iface(self, j, side):
        """(key, sign) of an interface: named by the left/bottom subdomain's side 4 or 2; c^(1)
        enters with + there and - on the neighbour (opposite outward normals)."""
        if side in (4, 2):
            return (j, side), 1.0
        return (self.neighbour(j, side), 4 if side == 3 else 2), -1.0

    def _side_xy(self, j, side, s):
        sb = self.subs[j]
        if side in (1, 2):
            return sb.x0 + (s + 1) / 2 * (sb.x1 - sb.x0), torch.full_like(s, sb.y0 if side == 1 else sb.y1)
        return torch.full_like(s, sb.x0 if side == 3 else sb.x1), sb.y0 + (s + 1) / 2 * (sb.y1 - sb.y0)

    def source_terms(self, j, kj):
        """(F_j, u_j) of layer j's source at wavenumber kj (None without a source), cached per k."""
        if self.source is None or self.source(j) is None:
            return None
        key = (j, float(kj))
        if key not in self._src_cache:
            fgrid, src4 = self.plan.source_foot_data(j, self.source(j))
            self._src_cache = {kk: v for kk, v in self._src_cache.items() if kk[0] != j}
            self._src_cache[key] = self.plan.source_terms(j, torch.from_numpy(fgrid).cuda(),
                                                          torch.from_numpy(src4).cuda())
        return self._src_cache[key]

    def receivers(self, k):
        """Solution at the receivers of every layer (list of complex tensors), differentiable in k
        (without a source; the source terms are not differentiated)."""
        if self.source is not None and k.requires_grad:
            raise NotImplementedError("the k-gradient of the source terms is not implemented")
        cvecs, rec = self.coefficients(k)
        res = []
        for j in range(self.N):
            row, m0, cnt, roff = self.rlayout[j]
            nc = self.layout[j][1]
            K = rec[roff:roff + nc * cnt].view(nc, cnt).transpose(0, 1)    # [cnt, 8M]
            val = linalg.matmul(K, cvecs[j])
            st = self.source_terms(j, self.plan_k(j))
            if st is not None:
                val = val + st[1][row, m0:m0 + cnt]
            res.append(val)
        return res

    def plan_k(self, j):
        """The wavenumber the plan is factored for in layer j."""
        ks = getattr(self.plan, "_k_current", None)
        return ks[j] if ks is not None else self.subs[j].k

    def field(self, k):
        """The solution on the whole grid of every layer, [ny, nx] complex tensors (the difference
        potential of the layer's boundary density, Eq. potential_solution_homo; meaningful on
        N+). Not differentiable."""
        with torch.no_grad():
            cvecs, _ = self.coefficients(k)
            out = []
            for j in range(self.N):
                dens = self.plan.basis_densities(j)                      # [8M, |gamma|]
                xi = linalg.matmul(dens.transpose(0, 1), cvecs[j])[None, :].contiguous()
                u = self.plan.potential(j, xi)[0]
                st = self.source_terms(j, self.plan_k(j))
                out.append(u if st is None else u + st[1])
            return out

    def _structure(self, device):
        """What the coupled system's shape depends on, built once: the unknowns (one block of M
        per outer side, two per interface), each subdomain's sides as ("outer", c) or
        ("if", c, sign), the unknowns each subdomain's rows touch, the Chebyshev points of every
        outer side, and the Chebyshev analysis matrix."""
        if getattr(self, "_st", None) is not None and self._st["device"] == device:
            return self._st
        M, N = self.M, self.N
        idx, n = {}, 0
        for j in range(N):
            for side in (1, 2, 3, 4):
                if self.outer(j, side):
                    idx[(j, side)] = n
                    n += M
            for side in (4, 2):
                if not self.outer(j, side):
                    idx[("if", j, side)] = n
                    n += 2 * M
        s = cheb_points(M, device)
        sides, col_sets, pts = [], [], {}
        for j in range(N):
            spec, used = [], []
            for side in (1, 2, 3, 4):
                if self.outer(j, side):
                    c = idx[(j, side)]
                    spec.append(("outer", c))
                    used.extend(range(c, c + M))
                    pts[(j, side)] = self._side_xy(j, side, s)
                else:
                    key, sgn = self.iface(j, side)
                    c = idx[("if",) + key]
                    spec.append(("if", c, sgn))
                    used.extend(range(c, c + 2 * M))
            sides.append(spec)
            col_sets.append(sorted(set(used)))
        i_ = torch.arange(M, dtype=torch.float64, device=device)
        T = torch.cos(i_[:, None] * math.pi * (i_[None, :] + 0.5) / M)   # T_m(x_i)
        w = torch.full((M,), 2.0 / M, dtype=torch.float64, device=device)
        w[0] = 1.0 / M
        self._st = {"device": device, "n": n, "sides": sides, "col_sets": col_sets, "pts": pts,
                    "cheb": (T.transpose(0, 1).to(torch.complex128).contiguous(), w)}
        return self._st

    def coefficients(self, k):
        """The Chebyshev coefficients [c^(0) sides 1..4, c^(1) sides 1..4] of every layer's boundary
        data from the coupled least-squares solve, and the receiver output of the projection.
        Outer side of unknown block u: alpha c0 + beta c1 = d (d the Chebyshev coefficients of
        the data); with beta != 0 the unknown is c0 and the side's rows read Q0 - (alpha/beta) Q1
        against u and -Q1 d / beta on the right; with beta = 0 the unknown is c1 (rows Q1) and
        the right-hand side -Q0 d / alpha. Interfaces: c0 shared, c1 with opposite signs."""
        M, N = self.M, self.N
        out, rec = ProjectWithReceivers.apply(k, self.plan)
        st = self._structure(out.device)
        n = st["n"]
        # boundary data of every outer side, analysed into Chebyshev coefficients in one product
        bcs, phis = [], []
        for j in range(N):
            for side, spec in zip((1, 2, 3, 4), st["sides"][j]):
                if spec[0] == "outer":
                    x, y = st["pts"][(j, side)]
                    alpha, beta, phi = self.bc(j, side, k[j], x, y)
                    bcs.append((alpha, beta))
                    phis.append(phi.to(torch.complex128))
        Tt, w = st["cheb"]
        d_all = linalg.matmul(torch.stack(phis), Tt) * w if phis else None   # [outer sides, M]
        A_rows, b_rows, coef = [], [], []
        q = 0
        for j in range(N):
            G, nc, off, _ = self.layout[j]
            Q = out[off:off + G * nc].view(nc, G).transpose(0, 1)          # [G, 8M]
            A = torch.zeros(G, n, dtype=torch.complex128, device=out.device)
            e = []                      # Q e is minus the right-hand side
            cj = []
            for side, spec in zip((1, 2, 3, 4), st["sides"][j]):
                Q0 = Q[:, (side - 1) * M: side * M]
                Q1 = Q[:, 4 * M + (side - 1) * M: 4 * M + side * M]
                if spec[0] == "outer":
                    c = spec[1]
                    alpha, beta = bcs[q]
                    d = d_all[q]
                    q += 1
                    if beta != 0:
                        A[:, c:c + M] = Q0 - (alpha / beta) * Q1
                        e.append((4 * M + (side - 1) * M, d / beta))
                        cj.append(("robin", c, d, alpha, beta))
                    else:
                        A[:, c:c + M] = Q1
                        e.append(((side - 1) * M, d / alpha))
                        cj.append(("dirichlet", c, d, alpha, beta))
                else:
                    _, c, sgn = spec
                    A[:, c:c + M] = Q0
                    A[:, c + M:c + 2 * M] = sgn * Q1
                    cj.append(("if", c, sgn))
            if e:
                ev = torch.zeros(8 * M, dtype=torch.complex128, device=out.device)
                for r, val in e:
                    ev[r:r + M] = val
                b = -linalg.matmul(Q, ev)
            else:
                b = torch.zeros(G, dtype=torch.complex128, device=out.device)
            src = self.source_terms(j, self.plan_k(j))
            if src is not None:
                b = b + src[0]
            A_rows.append(A)
            b_rows.append(b)
            coef.append(cj)
        A = torch.cat(A_rows)
        b = torch.cat(b_rows)
        xsol = LeastSquares.apply(A, b, ([r.shape[0] for r in A_rows], st["col_sets"]))
        cvecs = []
        for j in range(N):
            parts0, parts1 = [], []
            for spec in coef[j]:
                if spec[0] == "robin":
                    _, c, d, alpha, beta = spec
                    u0 = xsol[c:c + M]
                    parts0.append(u0)
                    parts1.append((d - alpha * u0) / beta)
                elif spec[0] == "dirichlet":
                    _, c, d, alpha, beta = spec
                    parts0.append(d / alpha)
                    parts1.append(xsol[c:c + M])
                else:
                    _, c, sgn = spec
                    parts0.append(xsol[c:c + M])
                    parts1.append(sgn * xsol[c + M:c + 2 * M])
            cvecs.append(torch.cat(parts0 + parts1))
        return cvecs, rec


def incident_impedance_bc(theta):
    """Outer data of config `strip4x1`: impedance sides du/dn + i k_j u = phi with phi from the
    plane wave exp(i k_j (x cos theta + y sin theta)) of the layer's own wavenumber."""
    def bc(j, side, kj, x, y):
        kx, ky = kj * math.cos(theta), kj * math.sin(theta)
        u = torch.exp(1j * (kx * x + ky * y))
        dn = {1: -1j * ky, 2: 1j * ky, 3: -1j * kx, 4: 1j * kx}[side] * u
        return 1j * kj, 1.0, dn + 1j * kj * u
    return bc


def receiver_row(sub, y_target=0.9):
    """Grid row whose y is nearest y_target (within M+)."""
    import numpy as np
    y = sub.ay0 + np.arange(sub.ny) * sub.h
    return int(np.argmin(np.abs(y - y_target)))
