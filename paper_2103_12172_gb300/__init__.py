"""GB300 (sm_103a) batched auxiliary-problem solves for the Method of Difference Potentials.

Python binding of libmdp (C ABI in include/mdp.h). Every step of the projection path runs in
the library's CUDA kernels; this module only allocates device tensors with PyTorch, picks the
current CUDA stream and marshals arguments. There is no CPU fallback: without the built
library or a GPU the compute calls raise.

    plan = Plan(subdomains)              # grid sets, per-mode LU factors, schedule, workspace
    Q = plan.project()                   # all basis columns, (P_gamma - I) Ex Psi_c
    P = plan.project(kind="P")           # P_gamma Ex Psi_c
    Qx = plan.project(xi=densities)      # user densities on gamma
    u = plan.solve(sub, g)               # full-grid G^(h) g
"""
from __future__ import annotations

import ctypes as C

import numpy as np

from . import _lib
from ._lib import MdpError, MDP_OUT_P, MDP_OUT_Q, MDP_PLAN_DEDUPE, MDP_PLAN_GRAPH, MDP_PLAN_HOST_ONLY

__all__ = ["Plan", "MdpError", "probe_fp64_gflops", "as_c_subdomains", "solve_noalloc"]

_KINDS = {"Q": MDP_OUT_Q, "P": MDP_OUT_P}


def as_c_subdomains(subs):
    """Array of mdp_subdomain structs from objects with the mdp_subdomain fields."""
    arr = (_lib.mdp_subdomain * len(subs))()
    for i, s in enumerate(subs):
        arr[i] = _lib.mdp_subdomain(float(s.x0), float(s.x1), float(s.y0), float(s.y1), float(s.ax0),
                                    float(s.ay0), float(s.h), int(s.nx), int(s.ny), float(s.k),
                                    int(s.ap_bc), int(s.n_modes))
    return arr


def _stream_ptr(stream):
    import torch
    s = torch.cuda.current_stream() if stream is None else stream
    return C.c_void_p(s.cuda_stream)


def _ptr(t):
    return C.c_void_p(t.data_ptr()) if t is not None else C.c_void_p(0)


class Plan:
    """A plan over a list of subdomains (objects with the mdp_subdomain fields)."""

    def __init__(self, subdomains, host_only: bool = False, graph: bool = False, tile_cols: int = 0,
                 workspace_bytes: int = 0, dedupe: bool = False, fp64_cols: bool = False,
                 direct_rows: bool = False, fft_block_points: int = 0, tri_stages: int = 0):
        """Kernel variants (same results to rounding; see autotune.tune_plan): fp64_cols sums the
        gamma columns of the middle rows on the FP64 pipe instead of the tensor cores, direct_rows
        takes the dense-row sine transforms by direct sums instead of the FFT, fft_block_points
        sets the complex values per FFT block (1024, 2048 or 4096), tri_stages the rows the per-mode
        sweep stages ahead (2 or 4); 0 selects the defaults."""
        self.L = _lib.lib()
        self.subdomains = list(subdomains)
        self._c_subs = as_c_subdomains(self.subdomains)
        handle = C.c_void_p()
        flags = ((MDP_PLAN_HOST_ONLY if host_only else 0) | (MDP_PLAN_GRAPH if graph else 0)
                 | (MDP_PLAN_DEDUPE if dedupe else 0) | (_lib.MDP_PLAN_FP64_COLS if fp64_cols else 0)
                 | (_lib.MDP_PLAN_DIRECT_ROWS if direct_rows else 0))
        opts = _lib.mdp_plan_options(int(tile_cols), int(workspace_bytes), int(fft_block_points), int(tri_stages))
        _lib.check(self.L.mdp_ap_plan_ex(self._c_subs, len(self.subdomains), flags, C.byref(opts), C.byref(handle)),
                   "mdp_ap_plan")
        self.handle = handle
        self.host_only = host_only
        self.n_subs = len(self.subdomains)
        self.output_size = int(self.L.mdp_plan_output_size(self.handle))

    def close(self):
        if getattr(self, "handle", None):
            self.L.mdp_plan_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # ---- layout
    def layout(self, sub: int):
        """(|gamma|, n_cols, out_offset, gamma_nm[|gamma|, 2] as (n, m))."""
        g, nc, off = C.c_int(), C.c_int(), C.c_longlong()
        ptr = C.POINTER(C.c_int)()
        _lib.check(self.L.mdp_plan_layout(self.handle, sub, C.byref(g), C.byref(nc), C.byref(off), C.byref(ptr)),
                   "mdp_plan_layout")
        nm = np.ctypeslib.as_array(ptr, shape=(g.value * 2,)).reshape(g.value, 2).copy()
        return g.value, nc.value, off.value, nm

    def gamma_geometry(self, sub: int):
        g = self.layout(sub)[0]
        owner = np.zeros(g, np.int32)
        rho = np.zeros(g)
        s = np.zeros(g)
        _lib.check(self.L.mdp_plan_gamma_geometry(self.handle, sub, owner.ctypes.data_as(C.POINTER(C.c_int)),
                                                  rho.ctypes.data_as(C.POINTER(C.c_double)),
                                                  s.ctypes.data_as(C.POINTER(C.c_double))), "mdp_plan_gamma_geometry")
        return owner, rho, s

    def host_mode_solve(self, sub: int, q: int, b, adjoint: bool = False):
        """T_q^{-1} b (or T_q^{-H} b) on the host: b holds one value per unknown row of the
        mode system (Nt values; the C call reads and writes exactly that many)."""
        b = np.ascontiguousarray(b, dtype=np.complex128)
        nt = self.sub_info(sub)["Nt"]
        if b.ndim != 1 or b.size != nt:
            raise ValueError(f"host_mode_solve: b must hold {nt} values, got shape {b.shape}")
        x = np.zeros_like(b)
        _lib.check(self.L.mdp_host_mode_solve(self.handle, sub, q, int(adjoint), b.ctypes.data_as(C.c_void_p),
                                              x.ctypes.data_as(C.c_void_p)), "mdp_host_mode_solve")
        return x

    def blocks(self, out):
        """Split a flat output tensor into per-subdomain [n_cols, |gamma|] views."""
        res = []
        for s in range(self.n_subs):
            g, nc, off, _ = self.layout(s)
            res.append(out[off:off + g * nc].view(nc, g))
        return res

    # ---- compute (device tensors, complex128)
    def _check_dev(self, t, n, name):
        import torch
        if t.dtype != torch.complex128 or not t.is_cuda or not t.is_contiguous() or t.numel() < n:
            raise ValueError(f"{name} must be a contiguous complex128 CUDA tensor with >= {n} elements")

    def project(self, xi=None, kind: str = "Q", out=None, stream=None, out_rec=None):
        """Projection columns of all subdomains as a flat complex128 CUDA tensor. With
        out_rec (a tensor, or True to allocate one) also the receiver values; returns
        (out, out_rec) then."""
        import torch
        n = self.output_size
        if out is None:
            out = torch.empty(n, dtype=torch.complex128, device="cuda")
        self._check_dev(out, n, "out")
        if xi is not None:
            self._check_dev(xi, n, "xi")
        if out_rec is True:
            out_rec = torch.empty(max(self.receiver_size, 1), dtype=torch.complex128, device="cuda")
        if out_rec is not None:
            self._check_dev(out_rec, self.receiver_size, "out_rec")
        _lib.check(self.L.mdp_project_batch_rec(self.handle, _ptr(xi), _ptr(out), _ptr(out_rec), _KINDS[kind],
                                                _stream_ptr(stream)), "mdp_project_batch")
        return out if out_rec is None else (out, out_rec)

    def set_receivers(self, rows):
        """Receiver grid row per subdomain (-1: none); see mdp_plan_set_receivers."""
        arr = (C.c_int * self.n_subs)(*[int(r) for r in rows])
        _lib.check(self.L.mdp_plan_set_receivers(self.handle, arr), "mdp_plan_set_receivers")

    @property
    def receiver_size(self):
        return int(self.L.mdp_plan_receiver_size(self.handle))

    def receiver_layout(self, sub):
        """(row, first m, count, offset) of subdomain `sub`'s receiver block."""
        r, m0, cnt, off = C.c_int(), C.c_int(), C.c_int(), C.c_longlong()
        _lib.check(self.L.mdp_plan_receiver_layout(self.handle, sub, C.byref(r), C.byref(m0), C.byref(cnt),
                                                   C.byref(off)), "mdp_plan_receiver_layout")
        return r.value, m0.value, cnt.value, off.value

    def project_columns(self, sub: int, col0: int, ncols: int, xi=None, kind: str = "Q", out=None, stream=None):
        import torch
        g = self.layout(sub)[0]
        if out is None:
            out = torch.empty(ncols * g, dtype=torch.complex128, device="cuda")
        self._check_dev(out, ncols * g, "out")
        if xi is not None:
            self._check_dev(xi, ncols * g, "xi")
        _lib.check(self.L.mdp_project_columns(self.handle, sub, col0, ncols, _ptr(xi), _ptr(out), _KINDS[kind],
                                              _stream_ptr(stream)), "mdp_project_columns")
        return out

    def potential(self, sub: int, xi, out=None, stream=None):
        """Difference potential w - G (L w)|M+ on the whole grid of subdomain `sub` for densities
        xi [ncols, |gamma|] (device complex128): tensor [ncols, ny, nx]."""
        import torch
        g = self.layout(sub)[0]
        xi = xi.reshape(-1, g).contiguous()
        ncols = xi.shape[0]
        s = self.subdomains[sub]
        if out is None:
            out = torch.empty((ncols, s.ny, s.nx), dtype=torch.complex128, device="cuda")
        self._check_dev(out, ncols * s.ny * s.nx, "out")
        self._check_dev(xi, ncols * g, "xi")
        _lib.check(self.L.mdp_potential(self.handle, sub, ncols, _ptr(xi), _ptr(out), _stream_ptr(stream)),
                   "mdp_potential")
        return out

    def source_terms(self, sub: int, f, src4, stream=None):
        """(F [|gamma|], u [ny, nx]) of a source: the right-hand side of the subdomain's system
        Q c = F and the source's part of its solution (device complex128 tensors). f: [ny, nx]
        on the auxiliary grid; src4: [|gamma|, 4] foot data (see source_foot_data)."""
        import torch
        g = self.layout(sub)[0]
        s = self.subdomains[sub]
        f = f.reshape(s.ny, s.nx).contiguous()
        src4 = src4.reshape(g, 4).contiguous()
        self._check_dev(f, s.ny * s.nx, "f")
        self._check_dev(src4, 4 * g, "src4")
        F = torch.empty(g, dtype=torch.complex128, device="cuda")
        u = torch.empty((s.ny, s.nx), dtype=torch.complex128, device="cuda")
        _lib.check(self.L.mdp_source_terms(self.handle, sub, _ptr(f), _ptr(src4), _ptr(F), _ptr(u),
                                           _stream_ptr(stream)), "mdp_source_terms")
        return F, u

    def source_foot_data(self, sub: int, fun):
        """Host evaluation of a source at what mdp_source_terms needs: (f on the grid [ny, nx],
        foot data [|gamma|, 4] = f, d_n f, d_nn f, d_tt f at each gamma node's foot point on its
        owner side) as numpy complex arrays. fun(x, y) -> (f, f_x, f_y, f_xx, f_yy)."""
        s = self.subdomains[sub]
        x = s.ax0 + np.arange(s.nx) * s.h
        y = s.ay0 + np.arange(s.ny) * s.h
        X, Y = np.meshgrid(x, y)
        fgrid = np.asarray(fun(X, Y)[0], dtype=complex) * np.ones_like(X)
        owner, _, sp = self.gamma_geometry(sub)
        src4 = np.zeros((owner.size, 4), dtype=complex)
        for side in (1, 2, 3, 4):
            sel = owner == side
            if not sel.any():
                continue
            t = (sp[sel] + 1.0) / 2.0
            if side in (1, 2):
                fx, fy = s.x0 + t * (s.x1 - s.x0), np.full(t.shape, s.y0 if side == 1 else s.y1)
            else:
                fx, fy = np.full(t.shape, s.x0 if side == 3 else s.x1), s.y0 + t * (s.y1 - s.y0)
            f, gx, gy, gxx, gyy = (np.asarray(v, dtype=complex) * np.ones_like(fx) for v in fun(fx, fy))
            if side in (1, 2):
                src4[sel] = np.stack([f, (-1.0 if side == 1 else 1.0) * gy, gyy, gxx], axis=1)
            else:
                src4[sel] = np.stack([f, (-1.0 if side == 3 else 1.0) * gx, gxx, gyy], axis=1)
        return fgrid, src4

    def basis_densities(self, sub: int, col0: int = 0, ncols=None, out=None, stream=None):
        """Extended basis densities Ex Psi_c on gamma: tensor [ncols, |gamma|] (complex128)."""
        import torch
        g, nc, _, _ = self.layout(sub)
        ncols = nc - col0 if ncols is None else ncols
        if out is None:
            out = torch.empty((ncols, g), dtype=torch.complex128, device="cuda")
        self._check_dev(out, ncols * g, "out")
        _lib.check(self.L.mdp_basis_densities(self.handle, sub, col0, ncols, _ptr(out), _stream_ptr(stream)),
                   "mdp_basis_densities")
        return out

    def adjoint(self, cot, xi=None, kind: str = "Q", grad_xi=True, grad_k=None, stream=None, cot_rec=None):
        """(grad_xi or None, grad_k) of a real loss with cotangent `cot` (layout of project())
        and optionally `cot_rec` on the receiver output."""
        import torch
        n = self.output_size
        self._check_dev(cot, n, "cot")
        if cot_rec is not None:
            self._check_dev(cot_rec, self.receiver_size, "cot_rec")
        gx = torch.empty(n, dtype=torch.complex128, device="cuda") if grad_xi else None
        if grad_k is None:
            grad_k = torch.zeros(self.n_subs, dtype=torch.float64, device="cuda")
        elif grad_k is False:
            grad_k = None
        _lib.check(self.L.mdp_ap_adjoint_rec(self.handle, _ptr(xi), _ptr(cot), _ptr(cot_rec), _ptr(gx), _ptr(grad_k),
                                             _KINDS[kind], _stream_ptr(stream)), "mdp_ap_adjoint")
        return gx, grad_k

    def solve(self, sub: int, g, adjoint: bool = False, out=None, stream=None):
        """u = G^(h) g (or A^{-H} g) on the full grid; g: complex128 CUDA tensor [nrhs, ny, nx]."""
        import torch
        s = self.subdomains[sub]
        g = g.reshape(-1, s.ny, s.nx)
        if out is None:
            out = torch.empty_like(g)
        self._check_dev(g, g.numel(), "g")
        self._check_dev(out, g.numel(), "out")
        _lib.check(self.L.mdp_ap_solve_batch(self.handle, sub, g.shape[0], _ptr(g), _ptr(out), int(adjoint),
                                             _stream_ptr(stream)), "mdp_ap_solve_batch")
        return out

    def update_k(self, ks, stream=None):
        """New wavenumbers: every mode is refactored (on the GPU for device plans, on `stream`,
        default the current torch stream; the call returns when the tables are rebuilt)."""
        arr = (C.c_double * self.n_subs)(*[float(k) for k in ks])
        st = None if self.host_only else _stream_ptr(stream)
        _lib.check(self.L.mdp_plan_update_k_stream(self.handle, arr, st), "mdp_plan_update_k_stream")

    def update_k_async(self, ks, stream=None):
        """New wavenumbers without waiting: the modes are refactored on `stream` (default the
        current torch stream) into a second table set, overlapping work queued on other streams;
        later calls on any stream wait for the new tables. A singular mode shows in status()."""
        arr = (C.c_double * self.n_subs)(*[float(k) for k in ks])
        st = None if self.host_only else _stream_ptr(stream)
        _lib.check(self.L.mdp_plan_update_k_async(self.handle, arr, st), "mdp_plan_update_k_async")

    def leaders(self) -> list:
        """Per subdomain, the subdomain whose tables and basis columns it shares (dedupe)."""
        a = (C.c_int * self.n_subs)()
        _lib.check(self.L.mdp_plan_leaders(self.handle, a), "mdp_plan_leaders")
        return list(a)

    def table_offsets(self, sub: int) -> dict:
        a = (C.c_longlong * 7)()
        _lib.check(self.L.mdp_plan_table_offsets(self.handle, sub, a), "mdp_plan_table_offsets")
        return dict(zip(["fact", "dT", "sin", "seg", "fs", "geo", "piv"], list(a)))

    def read_tables(self, device_side: bool):
        """(tables float64, pivot flags uint8) numpy copies of the device or host tables."""
        import numpy as np
        nd, npv = C.c_longlong(), C.c_longlong()
        _lib.check(self.L.mdp_plan_table_sizes(self.handle, C.byref(nd), C.byref(npv)), "mdp_plan_table_sizes")
        tab = np.empty(nd.value, dtype=np.float64)
        piv = np.empty(npv.value, dtype=np.uint8)
        _lib.check(self.L.mdp_plan_read_tables(self.handle, int(device_side), tab.ctypes.data_as(C.c_void_p),
                                               piv.ctypes.data_as(C.c_void_p)), "mdp_plan_read_tables")
        return tab, piv

    def sub_info(self, sub: int) -> dict:
        a = (C.c_int * 14)()
        _lib.check(self.L.mdp_plan_sub_info(self.handle, sub, a), "mdp_plan_sub_info")
        keys = ["Px", "Py", "Nq", "Nt", "i0", "nfirst", "cplx", "G", "R", "npiv", "n_cols", "Nx", "xsym",
                "complex_rows"]
        return dict(zip(keys, list(a)))

    def profile(self, enable: bool):
        _lib.check(self.L.mdp_plan_profile(self.handle, int(enable)), "mdp_plan_profile")

    def profile_read(self) -> dict:
        """{kernel name: (total ms, launches)} since the last read."""
        res = {}
        for f in range(self.L.mdp_kernel_family_count()):
            ms, n = C.c_double(), C.c_int()
            _lib.check(self.L.mdp_plan_profile_read(self.handle, f, C.byref(ms), C.byref(n)), "profile_read")
            if n.value:
                res[self.L.mdp_kernel_family_name(f).decode()] = (ms.value, n.value)
        return res

    def status(self):
        _lib.check(self.L.mdp_plan_status(self.handle), "device status")


def solve_noalloc(sub, g, adjoint: bool = False, out=None, stream=None):
    """Full-grid AP solve of one subdomain without a plan and without device allocation
    inside the library (mdp_ap_solve_noalloc); g, out: complex128 CUDA tensors [nrhs, ny, nx]."""
    import torch
    g = g.reshape(-1, sub.ny, sub.nx)
    if out is None:
        out = torch.empty_like(g)
    arr = as_c_subdomains([sub])
    _lib.check(_lib.lib().mdp_ap_solve_noalloc(arr, g.shape[0], _ptr(g), _ptr(out), int(adjoint), _stream_ptr(stream)),
               "mdp_ap_solve_noalloc")
    return out


def probe_fp64_gflops(iters: int = 0, stream=None) -> float:
    """Measured FP64 FMA throughput (GFLOP/s) of the current device."""
    v = C.c_double()
    _lib.check(_lib.lib().mdp_probe_dfma_gflops(int(iters), C.byref(v), _stream_ptr(stream)), "mdp_probe_dfma_gflops")
    return v.value


def probe_dmma_gflops(iters: int = 0, stream=None) -> float:
    """Measured FP64 tensor-core (mma.sync m8n8k4) throughput (GFLOP/s) of the current device."""
    v = C.c_double()
    _lib.check(_lib.lib().mdp_probe_dmma_gflops(int(iters), C.byref(v), _stream_ptr(stream)), "mdp_probe_dmma_gflops")
    return v.value
