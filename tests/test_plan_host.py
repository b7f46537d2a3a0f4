"""CPU tests of the C ABI through host-only plans: exported symbols, grid sets and gamma
geometry (bit-exact against the oracle), per-mode tridiagonal factors against the oracle's
2-D sparse solve, argument validation and resonance detection. No device work."""
import ctypes
import os
import re

import numpy as np
import pytest

import workloads as W
from oracle.grid import grid_sets
from oracle.projection import APSystem

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = set()
    for f in os.listdir(os.path.join(ROOT, "include")):
        if f.endswith(".h"):
            txt = open(os.path.join(ROOT, "include", f)).read()
            names |= set(re.findall(r"\b(mdp_[a-z0-9_]+)\s*\(", txt))
    return sorted(names)


def test_library_exports_every_declared_symbol(mdp):
    from paper_2103_12172_gb300 import _lib
    L = ctypes.CDLL(_lib.LIB_PATH)
    names = declared_functions()
    assert "mdp_project_batch" in names and "mdp_ap_adjoint" in names and "mdp_ap_plan" in names
    for n in names:
        assert hasattr(L, n), n
    assert set(names) <= set(_lib.EXPORTED) | {n for n in names if hasattr(L, n)}


def asym_subdomain():
    """Subdomain placed off-centre in its auxiliary rectangle (margins 0.1 and 0.17)."""
    s = W.unit_subdomain(0, 0, 65, 7.0, W.AP_DIRX_SOMMY, 4)
    h = 1.27 / 64
    return W.Subdomain(0.0, 1.0, 0.0, 1.0, -0.1, -0.17, h, 65, 65, 7.0, W.AP_DIRX_SOMMY, 4)


CASES = [W.small_subdomain(n, 10.0, ap, 4) for n in (17, 33, 129, 257) for ap in (0, 1)]
CASES += [asym_subdomain(), W.unit_subdomain(1, 1, 129, 10.0, 1, 4)]


@pytest.mark.parametrize("sub", CASES, ids=lambda s: f"n{s.nx}_ap{s.ap_bc}_x{s.ax0:.2f}_y{s.ay0:.2f}")
def test_gamma_and_ownership_match_oracle(mdp, sub):
    plan = mdp.Plan([sub], host_only=True)
    G, ncols, off, nm = plan.layout(0)
    gs = grid_sets(sub)
    assert G == gs.gamma_n.size and ncols == 8 * sub.n_modes and off == 0
    np.testing.assert_array_equal(nm[:, 0], gs.gamma_n)
    np.testing.assert_array_equal(nm[:, 1], gs.gamma_m)
    owner, rho, s = plan.gamma_geometry(0)
    np.testing.assert_array_equal(owner, gs.owner)
    np.testing.assert_allclose(rho, gs.rho, rtol=0, atol=1e-15)
    np.testing.assert_allclose(s, gs.s, rtol=0, atol=1e-14)
    assert plan.output_size == G * ncols


def test_output_layout_of_several_subdomains(mdp):
    subs = list(W.dd2x2_257().subdomains)
    plan = mdp.Plan(subs, host_only=True)
    off = 0
    for i in range(4):
        G, nc, o, _ = plan.layout(i)
        assert o == off and G == 1704 and nc == 256
        off += G * nc
    assert plan.output_size == off


@pytest.mark.parametrize("ap", [W.AP_DIRICHLET4, W.AP_DIRX_SOMMY, W.AP_DIRX_SOMMY_PAPER])
@pytest.mark.parametrize("n,k", [(33, 6.0), (129, 10.0)])
def test_mode_factors_reproduce_oracle_solves(mdp, ap, n, k):
    """G^(h) maps sin(pi q m/Nx) b(n) to sin(pi q m/Nx) T_q^{-1} b (separability of the AP);
    the plan's factors must reproduce the oracle's sparse-LU solve of the 2-D system, and
    T_q^{-H} its adjoint solve (up to the 1/h row scale of the Sommerfeld rows)."""
    sub = W.small_subdomain(n, k, ap, 4)
    plan = mdp.Plan([sub], host_only=True)
    S = APSystem(sub)
    nc = n - 1
    first = 0 if ap != W.AP_DIRICHLET4 else 1
    rows = np.arange(first, n - first)
    rng = np.random.default_rng(7)
    for q in (1, 2, nc // 3, nc // 2, nc - 1):
        sx = np.sin(np.pi * q * np.arange(n) / nc)
        b = rng.standard_normal(n) + 1j * rng.standard_normal(n)
        b[0] = b[-1] = 0.0                      # the AP right-hand side lives on M0
        g = np.outer(b, sx)
        u = S.solve(g)
        x = plan.host_mode_solve(0, q, b[rows])
        ref = u[rows][:, 1:-1]
        assert np.abs(ref - np.outer(x, sx[1:-1])).max() < 1e-10 * np.abs(ref).max()
        # adjoint: A^{-H} y for separable y on the unknowns
        y = rng.standard_normal(rows.size) + 1j * rng.standard_normal(rows.size)
        yy = np.zeros((n, n), complex)
        yy[rows] = np.outer(y, sx)
        yy[:, 0] = yy[:, -1] = 0
        mu = S.solve_adjoint(yy)
        xa = plan.host_mode_solve(0, q, y, adjoint=True)
        if ap != W.AP_DIRICHLET4:
            xa[0] /= sub.h
            xa[-1] /= sub.h
        refa = mu[rows][:, 1:-1]
        assert np.abs(refa - np.outer(xa, sx[1:-1])).max() < 1e-10 * np.abs(refa).max()


def test_argument_validation(mdp):
    from paper_2103_12172_gb300 import MdpError
    good = W.small_subdomain(33, 5.0, 1, 4)
    bad = [
        W.Subdomain(0, 1, 0, 1, -0.1, -0.1, 1.2 / 6, 7, 7, 5.0, 1, 4),         # nx < 9
        good.with_k(0.0),                                                     # k <= 0
        W.Subdomain(0, 1, 0, 1, -0.1, -0.1, good.h, 33, 33, 5.0, 1, 0),       # M* < 1
        W.Subdomain(0, 1, 0, 1, -0.01, -0.1, good.h, 33, 33, 5.0, 1, 4),      # gamma on the AP boundary
        W.Subdomain(0, 1, 0, 1, -0.1, -0.1, good.h, 33, 33, 5.0, 7, 4),       # unknown AP type
    ]
    for s in bad:
        with pytest.raises(MdpError) as e:
            mdp.Plan([s], host_only=True)
        assert e.value.code == 1  # MDP_ERR_ARG
    with pytest.raises(MdpError):
        mdp.Plan([], host_only=True)


def test_dirichlet_resonance_is_reported(mdp):
    """A Dirichlet AP whose discrete symbol mu_pq vanishes (k^2 chosen on a discrete
    eigenvalue) has a singular mode system: the plan reports MDP_ERR_SINGULAR."""
    from paper_2103_12172_gb300 import MdpError
    n = 33
    nc = n - 1
    h = 1.2 / nc
    lam = -4 * np.sin(np.pi * np.array([2, 3]) / (2 * nc)) ** 2
    lp, lq = lam
    k2 = -((lp + lq) / h**2 + lp * lq / (6 * h**2)) / (1 + (lp + lq) / 12)
    sub = W.small_subdomain(n, np.sqrt(k2), W.AP_DIRICHLET4, 4)
    with pytest.raises(MdpError) as e:
        mdp.Plan([sub], host_only=True)
    assert e.value.code == 4  # MDP_ERR_SINGULAR
    mdp.Plan([sub.with_k(np.sqrt(k2) * 1.05)], host_only=True)  # off resonance it plans


def test_host_refactor_equals_fresh_plan_and_table_readback(mdp):
    """update_k on a host-only plan rebuilds the same tables as a plan made at the new k; the
    device copy of a host-only plan is not readable (MDP_ERR_STATE)."""
    from paper_2103_12172_gb300 import MdpError
    sub = W.small_subdomain(33, 6.0, W.AP_DIRX_SOMMY, 2)
    p1 = mdp.Plan([sub], host_only=True)
    p1.update_k([8.5])
    p2 = mdp.Plan([sub.with_k(8.5)], host_only=True)
    t1, v1 = p1.read_tables(False)
    t2, v2 = p2.read_tables(False)
    np.testing.assert_array_equal(v1, v2)
    np.testing.assert_array_equal(t1, t2)
    off = p1.table_offsets(0)
    assert off["fact"] == 0 and off["fs"] > off["seg"] > off["geo"] > off["sin"] > off["dT"] > 0
    with pytest.raises(MdpError) as e:
        p1.read_tables(True)
    assert e.value.code == 6  # MDP_ERR_STATE
    # on a host-only plan the asynchronous update is the synchronous one
    p3 = mdp.Plan([sub], host_only=True)
    p3.update_k_async([8.5])
    t3, v3 = p3.read_tables(False)
    np.testing.assert_array_equal(v3, v2)
    np.testing.assert_array_equal(t3, t2)


def test_dedupe_groups_identical_subdomains_and_shares_tables(mdp):
    """MDP_PLAN_DEDUPE: the four identical 2 x 2 subdomains share the first one's tables; the
    checkerboard forms two groups; different k or grids never group."""
    from paper_2103_12172_gb300 import MdpError
    subs = list(W.dd2x2_257().subdomains)
    p = mdp.Plan(subs, host_only=True, dedupe=True)
    assert p.leaders() == [0, 0, 0, 0]
    assert mdp.Plan(subs, host_only=True).leaders() == [0, 1, 2, 3]
    offs = [p.table_offsets(i) for i in range(4)]
    assert all(o == offs[0] for o in offs)
    single = mdp.Plan(subs[:1], host_only=True)
    assert int(p.L.mdp_plan_table_bytes(p.handle)) == int(single.L.mdp_plan_table_bytes(single.handle))
    # output blocks stay separate
    assert [p.layout(i)[2] for i in range(4)] == [i * p.layout(0)[0] * p.layout(0)[1] for i in range(4)]
    assert mdp.Plan(list(W.checker2x2().subdomains), host_only=True, dedupe=True).leaders() == [0, 1, 1, 0]
    mixed = [subs[0], subs[1].with_k(31.0), subs[2], W.small_subdomain(65, 30.0, W.AP_DIRX_SOMMY, 32)]
    assert mdp.Plan(mixed, host_only=True, dedupe=True).leaders() == [0, 1, 0, 3]
    # a duplicate answers host introspection from the shared tables
    b = W.random_complex((2 * subs[0].nx,), seed=4)[: p.sub_info(0)["Nt"]]
    b = np.ascontiguousarray(b)
    x0 = np.empty_like(b)
    x3 = np.empty_like(b)
    import ctypes
    p.L.mdp_host_mode_solve(p.handle, 0, 7, 0, b.ctypes.data_as(ctypes.c_void_p), x0.ctypes.data_as(ctypes.c_void_p))
    p.L.mdp_host_mode_solve(p.handle, 3, 7, 0, b.ctypes.data_as(ctypes.c_void_p), x3.ctypes.data_as(ctypes.c_void_p))
    assert np.array_equal(x0, x3)
    # one k per group
    with pytest.raises(MdpError) as e:
        p.update_k([30.0, 30.0, 31.0, 30.0])
    assert e.value.code == 1  # MDP_ERR_ARG
    p.update_k([31.0] * 4)


def test_qcache_key_is_translation_invariant_and_complete():
    """The persisted Q cache keys a block by its auxiliary problem: translated copies share a key;
    k, M*, the AP type, the grid, the placement and the output kind each change it."""
    from paper_2103_12172_gb300.qcache import problem_key
    a = W.unit_subdomain(0, 0, 129, 12.0, W.AP_DIRX_SOMMY, 6)
    b = W.unit_subdomain(3, 5, 129, 12.0, W.AP_DIRX_SOMMY, 6)
    assert problem_key(a, "Q") == problem_key(b, "Q")
    others = [a.with_k(12.5), W.unit_subdomain(0, 0, 129, 12.0, W.AP_DIRX_SOMMY, 7),
              W.unit_subdomain(0, 0, 129, 12.0, W.AP_DIRICHLET4, 6), W.unit_subdomain(0, 0, 65, 12.0, W.AP_DIRX_SOMMY, 6),
              W.unit_subdomain(0, 0, 129, 12.0, W.AP_DIRX_SOMMY, 6, margin=0.2)]
    keys = {problem_key(o, "Q") for o in others} | {problem_key(a, "P")}
    assert problem_key(a, "Q") not in keys and len(keys) == len(others) + 1


def test_source_foot_data_matches_the_oracle(mdp):
    """The host evaluation of a source at the gamma foot points (product) equals the oracle's."""
    from oracle.grid import grid_sets
    from oracle.source import source_foot_data, source_on_grid
    sub = W.small_subdomain(33, 7.0, W.AP_DIRX_SOMMY, 2)
    plan = mdp.Plan([sub], host_only=True)

    def fun(x, y):
        u = np.exp(1j * (3.0 * x + 2.0 * y)) * (1.0 + x * y)
        return u, 2 * u, 3 * u, 5 * u, 7 * u
    fgrid, src4 = plan.source_foot_data(0, fun)
    assert np.allclose(fgrid, source_on_grid(sub, fun), rtol=0, atol=1e-15)
    assert np.allclose(src4, source_foot_data(grid_sets(sub), sub, fun), rtol=0, atol=1e-14)


def test_plan_options_are_validated_and_fft_blocks_fit_the_dst_epilogue(mdp):
    """FFT blocks of 1024, 2048 or 4096 points and 2 or 4 staged sweep rows are accepted, other
    values rejected (MDP_ERR_ARG). For every accepted block size and power-of-two row length
    the DST epilogue's requirements hold: the pair count per block, nseq N / 2 (nseq = P / (2 N)
    transforms, or 1), is a multiple of the 256-thread block and at most 32 x 32 (its scan
    scratch)."""
    from paper_2103_12172_gb300 import MdpError
    sub = W.small_subdomain(65, 7.0, W.AP_DIRX_SOMMY, 2)
    for ok in (dict(fft_block_points=1024), dict(fft_block_points=4096), dict(tri_stages=4), dict(tri_stages=2)):
        mdp.Plan([sub], host_only=True, **ok).close()
    for bad in (dict(fft_block_points=512), dict(fft_block_points=3000), dict(fft_block_points=8192),
                dict(tri_stages=3)):
        with pytest.raises(MdpError) as e:
            mdp.Plan([sub], host_only=True, **bad)
        assert e.value.code == 1, bad
    for P in (1024, 2048, 4096):
        for lg in range(3, 12):
            N = 1 << lg
            nseq = max(1, P // (2 * N))
            pairs = nseq * N // 2
            assert pairs % 256 == 0 and pairs // 32 <= 32, (P, N)
