"""GPU parity: the CUDA path (through the C ABI) against the CPU oracle, element by element.

Bar (relative L-infinity per column, max over columns): 1e-10 for fields and projection
columns. Inputs are seeded and synthetic (workloads.py)."""
import os

import numpy as np
import pytest

import workloads as W
from oracle.projection import APSystem

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = 1e-10


def rel_col_err(gpu, ref):
    """max over columns of max|gpu - ref| / max|ref| (rows = columns)."""
    gpu = np.asarray(gpu).reshape(ref.shape)
    num = np.abs(gpu - ref).max(axis=1)
    den = np.abs(ref).max(axis=1)
    return float((num / den).max())


@pytest.fixture(scope="module")
def dev(mdp):
    if not torch.cuda.is_available():
        pytest.fail("CUDA device required for -m gpu tests")
    return mdp


def make_plan(mdp, subs, tile=None):
    old = os.environ.get("MDP_TILE_COLS")
    if tile is not None:
        os.environ["MDP_TILE_COLS"] = str(tile)
    try:
        return mdp.Plan(subs)
    finally:
        if tile is not None:
            if old is None:
                del os.environ["MDP_TILE_COLS"]
            else:
                os.environ["MDP_TILE_COLS"] = old


@pytest.mark.parametrize("ap", [W.AP_DIRICHLET4, W.AP_DIRX_SOMMY, W.AP_DIRX_SOMMY_PAPER])
@pytest.mark.parametrize("n,k", [(33, 6.0), (129, 10.0)])
def test_full_grid_solve_and_adjoint(dev, ap, n, k):
    sub = W.small_subdomain(n, k, ap, 4)
    plan = dev.Plan([sub])
    S = APSystem(sub)
    g = W.random_complex((3, n, n), seed=0)
    u = plan.solve(0, torch.from_numpy(g).cuda()).cpu().numpy()
    ref = np.stack([S.solve(x) for x in g])
    assert rel_col_err(u.reshape(3, -1), ref.reshape(3, -1)) < TOL
    # adjoint: input on the unknown nodes
    y = g.copy()
    y[:, :, 0] = y[:, :, -1] = 0
    if ap == W.AP_DIRICHLET4:
        y[:, 0, :] = y[:, -1, :] = 0
    ua = plan.solve(0, torch.from_numpy(y).cuda(), adjoint=True).cpu().numpy()
    refa = np.stack([S.solve_adjoint(x) for x in y])
    assert rel_col_err(ua.reshape(3, -1), refa.reshape(3, -1)) < TOL


PROJ_CASES = [
    ("single_129_dir4", W.single_129().subdomains[0], None),
    ("n65_somm_m5_ragged", W.small_subdomain(65, 12.0, W.AP_DIRX_SOMMY, 5), 16),
    ("n33_dir4_m3", W.small_subdomain(33, 6.0, W.AP_DIRICHLET4, 3), 7),
    ("n17_somm_m1", W.small_subdomain(17, 3.0, W.AP_DIRX_SOMMY, 1), None),
    ("strip_129_k40", W.strip4x1().subdomains[2], 96),
    # grids whose Nx is not a power of 2: the dense rows take the direct sine sums
    ("n61_somm_m3_direct", W.small_subdomain(61, 8.0, W.AP_DIRX_SOMMY, 3), 8),
    ("n50_dir4_m2_direct_oddNx", W.small_subdomain(50, 7.0, W.AP_DIRICHLET4, 2), None),
    # the Sommerfeld rows as printed in the paper; FFT and direct dense rows
    ("n65_somm_paper_m3", W.small_subdomain(65, 10.0, W.AP_DIRX_SOMMY_PAPER, 3), 16),
    ("n61_somm_paper_m2_direct", W.small_subdomain(61, 8.0, W.AP_DIRX_SOMMY_PAPER, 2), None),
]


@pytest.mark.parametrize("name,sub,tile", PROJ_CASES, ids=[c[0] for c in PROJ_CASES])
@pytest.mark.parametrize("kind", ["Q", "P"])
def test_basis_columns_match_oracle(dev, name, sub, tile, kind):
    plan = make_plan(dev, [sub], tile)
    out = plan.project(kind=kind)
    torch.cuda.synchronize()
    plan.status()
    G, nc, _, _ = plan.layout(0)
    got = out.cpu().numpy().reshape(nc, G)
    ref = APSystem(sub).columns(kind=kind)
    assert rel_col_err(got, ref) < TOL


@pytest.mark.parametrize("ap", [W.AP_DIRICHLET4, W.AP_DIRX_SOMMY])
@pytest.mark.parametrize("kind", ["Q", "P"])
def test_user_densities_match_oracle(dev, ap, kind):
    sub = W.small_subdomain(65, 9.0, ap, 2)
    plan = make_plan(dev, [sub], 8)
    G, nc, _, _ = plan.layout(0)
    xi = W.random_complex((nc, G), seed=11)
    out = plan.project(xi=torch.from_numpy(xi.ravel()).cuda(), kind=kind).cpu().numpy().reshape(nc, G)
    ref = APSystem(sub).columns(xi=xi, kind=kind)
    assert rel_col_err(out, ref) < TOL


def test_fft_and_direct_subdomains_in_one_launch(dev):
    """A batch mixing a power-of-2 grid (FFT dense rows) with a 61-node grid (direct sums)."""
    subs = [W.small_subdomain(65, 10.0, W.AP_DIRX_SOMMY, 3), W.small_subdomain(61, 9.0, W.AP_DIRX_SOMMY, 3)]
    plan = make_plan(dev, subs, 16)
    blocks = [b.cpu().numpy() for b in plan.blocks(plan.project())]
    for blk, sub in zip(blocks, subs):
        assert rel_col_err(blk, APSystem(sub).columns()) < TOL


def test_unbatched_path_equals_batched(dev):
    """The per-column path runs the same kernels one column at a time: identical results."""
    sub = W.small_subdomain(129, 10.0, W.AP_DIRX_SOMMY, 4)
    plan = make_plan(dev, [sub], 32)
    full = plan.project().cpu().numpy()
    G = plan.layout(0)[0]
    for c in (0, 5, 17, 31):
        one = plan.project_columns(0, c, 1).cpu().numpy()
        assert np.array_equal(one, full[c * G:(c + 1) * G])


def test_asymmetric_placement(dev):
    sub = W.Subdomain(0.0, 1.0, 0.0, 1.0, -0.1, -0.17, 1.27 / 64, 65, 65, 7.0, W.AP_DIRX_SOMMY, 3)
    plan = dev.Plan([sub])
    G, nc, _, _ = plan.layout(0)
    got = plan.project().cpu().numpy().reshape(nc, G)
    assert rel_col_err(got, APSystem(sub).columns()) < TOL


def test_dd2x2_257_workload(dev):
    """The 2x2 decomposition at 257^2 (k = 30, mixed AP, 1024 columns in one launch):
    every column of subdomain 0 and 32 sampled columns of each other subdomain."""
    wl = W.dd2x2_257()
    plan = dev.Plan(list(wl.subdomains))
    out = plan.project()
    blocks = [b.cpu().numpy() for b in plan.blocks(out)]
    rng = np.random.default_rng(0)
    for i, sub in enumerate(wl.subdomains):
        S = APSystem(sub)
        cols = list(range(256)) if i == 0 else sorted(rng.choice(256, 32, replace=False).tolist())
        ref = S.columns(cols=cols)
        assert rel_col_err(blocks[i][cols], ref) < TOL, i


def test_checkerboard_workload_sampled(dev):
    """2x2 checkerboard with 129^2 (k = 10) and 513^2 (k = 100) subdomains in one batch: every
    subdomain on 12 random columns, and each 513^2, k = 100 subdomain (the most near-propagating
    modes) also on the highest Chebyshev mode T_47 of every side and both kinds."""
    wl = W.checker2x2()
    plan = dev.Plan(list(wl.subdomains))
    out = plan.project()
    blocks = plan.blocks(out)
    rng = np.random.default_rng(1)
    for i, sub in enumerate(wl.subdomains):
        M = sub.n_modes
        cols = set(rng.choice(8 * M, 12, replace=False).tolist())
        if sub.nx == 513:
            cols |= {M * j + M - 1 for j in range(8)}
        cols = sorted(cols)
        ref = APSystem(sub).columns(cols=cols)
        assert rel_col_err(blocks[i].cpu().numpy()[cols], ref) < TOL, i


@pytest.mark.slow
def test_dd8x8_workload_sampled(dev):
    """The 8 x 8 decomposition at full size (64 subdomains, 257^2 / 513^2 / 1025^2 grids, 32768
    columns) in one batched pass; one subdomain per grid class is checked against the oracle on
    4 sampled columns (the 1025^2 SuperLU factorisation alone takes about a minute)."""
    wl = W.dd8x8_mixed()
    subs = list(wl.subdomains)
    plan = dev.Plan(subs)
    out = plan.project()
    torch.cuda.synchronize()
    plan.status()
    blocks = plan.blocks(out)
    seen = set()
    for i, s in enumerate(subs):
        if s.nx in seen:
            continue
        seen.add(s.nx)
        cols = [0, 129, 300, 511]
        ref = APSystem(s).columns(cols=cols)
        assert rel_col_err(blocks[i].cpu().numpy()[cols], ref) < TOL, (i, s.nx)
    assert seen == {257, 513, 1025}


@pytest.mark.parametrize("ap", [W.AP_DIRICHLET4, W.AP_DIRX_SOMMY])
@pytest.mark.parametrize("n", [65, 61])
def test_potential_on_the_grid_matches_oracle(dev, ap, n):
    """mdp_potential (the difference potential w - G (L w)|M+ on every node) against the oracle."""
    sub = W.small_subdomain(n, 10.0, ap, 2)
    plan = make_plan(dev, [sub], 8)
    S = APSystem(sub)
    G = plan.layout(0)[0]
    xi = W.random_complex((3, G), seed=41)
    u = plan.potential(0, torch.from_numpy(xi).cuda()).cpu().numpy()
    ref = np.stack([S.potential(x) for x in xi])
    assert rel_col_err(u.reshape(3, -1), ref.reshape(3, -1)) < TOL


def test_basis_densities_match_oracle(dev):
    sub = W.small_subdomain(65, 12.0, W.AP_DIRX_SOMMY, 5)
    plan = make_plan(dev, [sub], 16)
    S = APSystem(sub)
    got = plan.basis_densities(0).cpu().numpy()
    ref = np.stack([S.basis_density(c) for c in range(8 * sub.n_modes)])
    assert np.abs(got - ref).max() <= 1e-13 * np.abs(ref).max()
    part = plan.basis_densities(0, col0=7, ncols=20).cpu().numpy()
    assert np.array_equal(part, got[7:27])


@pytest.mark.parametrize("ap", [W.AP_DIRICHLET4, W.AP_DIRX_SOMMY])
@pytest.mark.parametrize("n", [65, 61])
def test_source_terms_match_oracle(dev, ap, n):
    """mdp_source_terms (F = (I - P_gamma) Ex^(I) f - Tr G (B f)|M+ and the source's part of the
    solution on the grid) against the oracle, on the same f and foot data."""
    from oracle.source import source_foot_data, source_on_grid, source_terms

    def fun(x, y):
        u = np.exp(1j * (3.0 * x + 2.0 * y))
        return (1.0 + x) * u, u, 2 * u, -3 * u, -4 * u
    sub = W.small_subdomain(n, 9.0, ap, 2)
    plan = make_plan(dev, [sub], 8)
    S = APSystem(sub)
    fgrid = source_on_grid(sub, fun)
    src4 = source_foot_data(S.gs, sub, fun)
    F, u = plan.source_terms(0, torch.from_numpy(fgrid).cuda(), torch.from_numpy(src4).cuda())
    Fr, ur = source_terms(S, fgrid, src4)
    F, u = F.cpu().numpy(), u.cpu().numpy()
    assert np.abs(F - Fr).max() <= TOL * np.abs(Fr).max()
    assert np.abs(u - ur).max() <= TOL * np.abs(ur).max()


@pytest.mark.slow
@pytest.mark.parametrize("n", [2049, 1001])
def test_largest_grids_against_the_sine_transform_closed_form(dev, n):
    """Maximum sizes: a 2049^2 Dirichlet AP (the longest dense-row FFT, 2 Nx = 4096, one column
    per block) and a 1001^2 one (Nx = 1000: the direct sums), every basis column against the
    oracle's extension and stencil with the AP solved in closed form by the 2-D DST-I (the
    closed form is pinned against the sparse LU; a sparse LU at these sizes is out of reach)."""
    import scipy.fft
    from oracle.extension import basis_column
    from oracle.grid import grid_sets
    from oracle.scheme import apply_L
    k = 37.3
    sub = W.small_subdomain(n, k, W.AP_DIRICHLET4, 2)
    plan = make_plan(dev, [sub], 16)
    G, nc, _, _ = plan.layout(0)
    got = plan.project().cpu().numpy().reshape(nc, G)
    gs = grid_sets(sub)
    h, ncell = sub.h, n - 1
    lam = -4 * np.sin(np.pi * np.arange(1, ncell) / (2 * ncell)) ** 2
    LP, LQ = np.meshgrid(lam, lam)
    mu = (LP + LQ) / h**2 + LP * LQ / (6 * h**2) + k**2 + k**2 * (LP + LQ) / 12
    ref = np.zeros((nc, G), complex)
    for c in range(nc):
        w = np.zeros((n, n), complex)
        w[gs.gamma_n, gs.gamma_m] = basis_column(gs, k, sub.n_modes, c)
        r = apply_L(w, h, k)
        r[~gs.Mp] = 0.0
        u = np.zeros((n, n), complex)
        u[1:-1, 1:-1] = scipy.fft.idstn(scipy.fft.dstn(r[1:-1, 1:-1], type=1) / mu, type=1)
        ref[c] = -u[gs.gamma_n, gs.gamma_m]
    assert rel_col_err(got, ref) < TOL
