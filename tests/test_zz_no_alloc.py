"""mdp_ap_solve_noalloc: the full-grid AP solve for callers that cannot allocate device memory
(no plan, no cudaMalloc inside the call; its scratch is a fixed device array of the library).
Checked against mdp_ap_solve_batch on two calls in a row, through the C ABI. This file is
collected last so that a stop at the first failure has already run every other test."""
import ctypes

import numpy as np
import pytest

import workloads as W

torch = pytest.importorskip("torch")

TOL = 1e-10


def c_sub(mdp, sub):
    return mdp.as_c_subdomains([sub])


def call_noalloc(mdp, sub, g, adjoint):
    from paper_2103_12172_gb300 import _lib
    u = torch.empty_like(g)
    rc = _lib.lib().mdp_ap_solve_noalloc(c_sub(mdp, sub), g.shape[0], ctypes.c_void_p(g.data_ptr()),
                                         ctypes.c_void_p(u.data_ptr()), int(adjoint),
                                         ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert rc == 0, _lib.status_string(rc)
    return u


def rel_err(a, b):
    a = a.reshape(a.shape[0], -1)
    b = b.reshape(b.shape[0], -1)
    return float((np.abs(a - b).max(axis=1) / np.abs(b).max(axis=1)).max())


def test_noalloc_rejects_grids_beyond_its_scratch(mdp):
    from paper_2103_12172_gb300 import _lib
    L = _lib.lib()
    assert L.mdp_ap_solve_noalloc_limit_bytes() == 32 << 20
    for n in (705, 1025):                                      # factor rows + one right-hand side > 32 MiB
        big = W.small_subdomain(n, 40.0, W.AP_DIRX_SOMMY, 2)
        rc = L.mdp_ap_solve_noalloc(c_sub(mdp, big), 1, ctypes.c_void_p(0), ctypes.c_void_p(0), 0,
                                    ctypes.c_void_p(0))
        assert rc == _lib.MDP_ERR_ARG
    fits = W.small_subdomain(641, 40.0, W.AP_DIRX_SOMMY, 2)    # zero right-hand sides: size check only
    assert L.mdp_ap_solve_noalloc(c_sub(mdp, fits), 0, ctypes.c_void_p(0), ctypes.c_void_p(0), 0,
                                  ctypes.c_void_p(0)) == 0


def scratch_chunk(mdp, sub):
    """Right-hand sides per chunk of the scratch's mode-space buffer (an estimate within one
    of the library's own: the descriptor, the factor rows, the sine table and the pivot flags
    of the same subdomain come first)."""
    from paper_2103_12172_gb300 import _lib
    p = mdp.Plan([sub], host_only=True)
    info = p.sub_info(0)
    p.close()
    a = lambda v: (v + 255) // 256 * 256                      # noqa: E731
    qt = info["Nq"] * info["Nt"]
    sin_off = (qt * (8 if info["cplx"] else 4) + 31) // 32 * 32
    used = a(512) + a((sin_off + 4 * info["Nx"]) * 8) + a(qt)
    return (_lib.lib().mdp_ap_solve_noalloc_limit_bytes() - used) // (qt * 16)


@pytest.mark.gpu
def test_noalloc_matches_plan_solve_on_two_calls(mdp):
    if not torch.cuda.is_available():
        pytest.fail("CUDA device required")
    cases = [(W.small_subdomain(129, 10.0, W.AP_DIRX_SOMMY, 2), 0, 0),
             (W.small_subdomain(65, 7.0, W.AP_DIRICHLET4, 2), 1, 1)]
    for sub, seed, adjoint in cases:               # two calls in a row, different grids
        g = W.random_complex((3, sub.ny, sub.nx), seed=seed)
        g[:, :, 0] = g[:, :, -1] = 0
        gd = torch.from_numpy(g).cuda()
        u_na = call_noalloc(mdp, sub, gd, adjoint)
        u_ref = mdp.Plan([sub]).solve(0, gd, adjoint=bool(adjoint))
        torch.cuda.synchronize()
        assert rel_err(u_na.cpu().numpy(), u_ref.cpu().numpy()) < TOL
    # and the first case again after the second overwrote the scratch
    sub, seed, adjoint = cases[0]
    g = torch.from_numpy(W.random_complex((2, sub.ny, sub.nx), seed=9)).cuda()
    assert rel_err(call_noalloc(mdp, sub, g, 0).cpu().numpy(), mdp.Plan([sub]).solve(0, g).cpu().numpy()) < TOL


@pytest.mark.gpu
def test_noalloc_chunks_and_in_place(mdp):
    """More right-hand sides than one chunk of the scratch buffer (the per-chunk offsets into g
    and u), solved in place (u == g), against the plan's solve."""
    if not torch.cuda.is_available():
        pytest.fail("CUDA device required")
    from paper_2103_12172_gb300 import _lib
    sub = W.small_subdomain(257, 30.0, W.AP_DIRX_SOMMY, 2)
    chunk = scratch_chunk(mdp, sub)
    assert 1 <= chunk < 64
    g = torch.from_numpy(W.random_complex((chunk + 2, sub.ny, sub.nx), seed=5)).cuda()
    ref = mdp.Plan([sub]).solve(0, g)
    u = g.clone()
    rc = _lib.lib().mdp_ap_solve_noalloc(c_sub(mdp, sub), u.shape[0], ctypes.c_void_p(u.data_ptr()),
                                         ctypes.c_void_p(u.data_ptr()), 0,
                                         ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert rc == 0, _lib.status_string(rc)
    torch.cuda.synchronize()
    assert rel_err(u.cpu().numpy(), ref.cpu().numpy()) < TOL


@pytest.mark.gpu
def test_noalloc_refuses_a_capturing_stream(mdp):
    """A call on a stream that is capturing a CUDA graph returns MDP_ERR_STATE and enqueues
    nothing; the same call outside the capture still solves."""
    if not torch.cuda.is_available():
        pytest.fail("CUDA device required")
    from paper_2103_12172_gb300 import _lib
    sub = W.small_subdomain(65, 7.0, W.AP_DIRX_SOMMY, 2)
    g = torch.from_numpy(W.random_complex((2, sub.ny, sub.nx), seed=11)).cuda()
    u = torch.zeros_like(g)
    torch.cuda.synchronize()
    graph = torch.cuda.CUDAGraph()
    s = torch.cuda.Stream()
    with torch.cuda.graph(graph, stream=s):
        u.add_(0.0)                                  # keeps the captured graph non-empty
        rc = _lib.lib().mdp_ap_solve_noalloc(c_sub(mdp, sub), g.shape[0], ctypes.c_void_p(g.data_ptr()),
                                             ctypes.c_void_p(u.data_ptr()), 0, ctypes.c_void_p(s.cuda_stream))
    torch.cuda.synchronize()
    assert rc == _lib.MDP_ERR_STATE
    graph.replay()
    torch.cuda.synchronize()
    assert float(u.abs().max()) == 0.0               # nothing of the refused call was captured
    assert rel_err(call_noalloc(mdp, sub, g, 0).cpu().numpy(), mdp.Plan([sub]).solve(0, g).cpu().numpy()) < TOL
