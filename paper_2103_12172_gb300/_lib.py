"""ctypes view of libmdp.so (the C ABI in include/mdp.h). Argument marshalling only."""
from __future__ import annotations

import ctypes as C
import os

_PKG = os.path.dirname(os.path.abspath(__file__))
# MDP_LIB_CHECKED=1 loads the bounds-checked build (libmdp_checked.so) instead
LIB_PATH = os.path.join(_PKG, "libmdp_checked.so" if os.environ.get("MDP_LIB_CHECKED") == "1" else "libmdp.so")

MDP_OK, MDP_ERR_ARG, MDP_ERR_CUDA, MDP_ERR_NOMEM, MDP_ERR_SINGULAR, MDP_ERR_TIMEOUT, MDP_ERR_STATE, MDP_ERR_BOUNDS = range(8)
MDP_AP_DIRICHLET4, MDP_AP_DIRX_SOMMY, MDP_AP_DIRX_SOMMY_PAPER = 0, 1, 2
MDP_OUT_Q, MDP_OUT_P = 0, 1
MDP_PLAN_HOST_ONLY = 0x1
MDP_PLAN_GRAPH = 0x2
MDP_PLAN_DEDUPE = 0x4
MDP_PLAN_FP64_COLS = 0x8
MDP_PLAN_DIRECT_ROWS = 0x10

EXPORTED = [
    "mdp_ap_plan", "mdp_plan_update_k", "mdp_plan_layout", "mdp_plan_output_size", "mdp_project_batch",
    "mdp_project_columns", "mdp_ap_adjoint", "mdp_ap_solve_batch", "mdp_plan_status", "mdp_plan_destroy",
    "mdp_status_string", "mdp_plan_gamma_geometry", "mdp_host_mode_solve", "mdp_probe_dfma_gflops", "mdp_probe_dmma_gflops",
]


class mdp_subdomain(C.Structure):
    _fields_ = [("x0", C.c_double), ("x1", C.c_double), ("y0", C.c_double), ("y1", C.c_double),
                ("ax0", C.c_double), ("ay0", C.c_double), ("h", C.c_double),
                ("nx", C.c_int), ("ny", C.c_int), ("k", C.c_double), ("ap_bc", C.c_int), ("n_modes", C.c_int)]


class mdp_plan_options(C.Structure):
    _fields_ = [("tile_cols", C.c_int), ("workspace_bytes", C.c_longlong), ("fft_block_points", C.c_int),
                ("tri_stages", C.c_int)]


class MdpError(RuntimeError):
    def __init__(self, code, what):
        self.code = code
        super().__init__(f"{what}: {status_string(code)} (status {code})")


_lib = None


def lib():
    """Load libmdp.so; raises if it has not been built (there is no fallback path)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"{os.path.basename(LIB_PATH)} not found at {LIB_PATH}: build it with "
                          "`python -c 'import __graft_entry__ as g; g.build()'`")
    L = C.CDLL(LIB_PATH)
    vp, i, ll, d = C.c_void_p, C.c_int, C.c_longlong, C.c_double
    sig = {
        "mdp_ap_plan": (i, [C.POINTER(mdp_subdomain), i, C.c_uint, C.POINTER(vp)]),
        "mdp_ap_plan_ex": (i, [C.POINTER(mdp_subdomain), i, C.c_uint, C.POINTER(mdp_plan_options), C.POINTER(vp)]),
        "mdp_plan_update_k": (i, [vp, C.POINTER(d)]),
        "mdp_plan_update_k_stream": (i, [vp, C.POINTER(d), vp]),
        "mdp_plan_update_k_async": (i, [vp, C.POINTER(d), vp]),
        "mdp_plan_table_sizes": (i, [vp, C.POINTER(ll), C.POINTER(ll)]),
        "mdp_plan_update_bytes": (ll, [vp]),
        "mdp_plan_leaders": (i, [vp, C.POINTER(i)]),
        "mdp_potential": (i, [vp, i, i, vp, vp, vp]),
        "mdp_basis_densities": (i, [vp, i, i, i, vp, vp]),
        "mdp_source_terms": (i, [vp, i, vp, vp, vp, vp, vp]),
        "mdp_householder_qr_work_ints": (ll, [i]),
        "mdp_householder_qr": (i, [i, i, i, vp, ll, vp, vp, vp]),
        "mdp_householder_qr_batched": (i, [i, i, i, i, vp, ll, ll, vp, vp, vp]),
        "mdp_triangular_solve": (i, [i, i, vp, ll, i, vp, ll, vp]),
        "mdp_complex_matmul": (i, [i, i, i, vp, ll, ll, i, vp, ll, ll, i, vp, ll, ll, i, vp]),
        "mdp_probe_rcp": (i, [vp, vp, i, vp]),
        "mdp_plan_read_tables": (i, [vp, i, vp, vp]),
        "mdp_plan_table_offsets": (i, [vp, i, C.POINTER(ll)]),
        "mdp_plan_layout": (i, [vp, i, C.POINTER(i), C.POINTER(i), C.POINTER(ll), C.POINTER(C.POINTER(i))]),
        "mdp_plan_output_size": (ll, [vp]),
        "mdp_project_batch": (i, [vp, vp, vp, i, vp]),
        "mdp_project_columns": (i, [vp, i, i, i, vp, vp, i, vp]),
        "mdp_ap_adjoint": (i, [vp, vp, vp, vp, vp, i, vp]),
        "mdp_ap_solve_batch": (i, [vp, i, i, vp, vp, i, vp]),
        "mdp_plan_status": (i, [vp]),
        "mdp_plan_destroy": (None, [vp]),
        "mdp_status_string": (C.c_char_p, [i]),
        "mdp_plan_gamma_geometry": (i, [vp, i, C.POINTER(i), C.POINTER(d), C.POINTER(d)]),
        "mdp_host_mode_solve": (i, [vp, i, i, i, vp, vp]),
        "mdp_probe_dfma_gflops": (i, [i, C.POINTER(d), vp]),
        "mdp_probe_dmma_gflops": (i, [i, C.POINTER(d), vp]),
        "mdp_plan_profile": (i, [vp, i]),
        "mdp_plan_profile_read": (i, [vp, i, C.POINTER(d), C.POINTER(i)]),
        "mdp_kernel_family_count": (i, []),
        "mdp_kernel_family_name": (C.c_char_p, [i]),
        "mdp_plan_sub_info": (i, [vp, i, C.POINTER(i)]),
        "mdp_ap_solve_noalloc": (i, [C.POINTER(mdp_subdomain), i, vp, vp, i, vp]),
        "mdp_ap_solve_noalloc_limit_bytes": (ll, []),
        "mdp_plan_set_receivers": (i, [vp, C.POINTER(i)]),
        "mdp_plan_receiver_layout": (i, [vp, i, C.POINTER(i), C.POINTER(i), C.POINTER(i), C.POINTER(ll)]),
        "mdp_plan_receiver_size": (ll, [vp]),
        "mdp_plan_table_bytes": (ll, [vp]),
        "mdp_project_batch_rec": (i, [vp, vp, vp, vp, i, vp]),
        "mdp_ap_adjoint_rec": (i, [vp, vp, vp, vp, vp, vp, i, vp]),
    }
    for name, (res, args) in sig.items():
        f = getattr(L, name)
        f.restype = res
        f.argtypes = args
    _lib = L
    return L


def status_string(code: int) -> str:
    try:
        return lib().mdp_status_string(int(code)).decode()
    except ImportError:
        return str(code)


def check(code: int, what: str):
    if code != MDP_OK:
        raise MdpError(code, what)
