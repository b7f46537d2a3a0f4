"""GPU adjoint (mdp_ap_adjoint) against the oracle's adjoint, finite differences of the GPU
forward map, and the dot-product identity. Bars: grad_xi relative L-infinity per column 1e-10;
grad_k 1e-9 relative to the oracle's (itself pinned by finite differences) and 1e-6 relative
to central differences of the GPU forward."""
import os

import numpy as np
import pytest

import workloads as W
from oracle.projection import APSystem

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


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


def rel_col_err(got, ref):
    return float((np.abs(got - ref).max(axis=1) / np.abs(ref).max(axis=1)).max())


CASES = [("dir4_n65", W.small_subdomain(65, 9.0, W.AP_DIRICHLET4, 2), 8),
         ("somm_n65", W.small_subdomain(65, 11.0, W.AP_DIRX_SOMMY, 2), 8),
         ("somm_n129", W.small_subdomain(129, 20.0, W.AP_DIRX_SOMMY, 3), None),
         # Nx not a power of 2: direct dense-row sums in the adjoint
         ("somm_n61_direct", W.small_subdomain(61, 10.0, W.AP_DIRX_SOMMY, 2), 8),
         ("dir4_n50_direct_oddNx", W.small_subdomain(50, 8.0, W.AP_DIRICHLET4, 2), None),
         # the Sommerfeld rows as printed in the paper (their own k-derivatives)
         ("somm_paper_n65", W.small_subdomain(65, 11.0, W.AP_DIRX_SOMMY_PAPER, 2), 8)]


@pytest.mark.parametrize("name,sub,tile", CASES, ids=[c[0] for c in CASES])
@pytest.mark.parametrize("kind", ["Q", "P"])
def test_grad_xi_matches_oracle(mdp, name, sub, tile, kind):
    plan = make_plan(mdp, [sub], tile)
    G, nc, _, _ = plan.layout(0)
    xi = W.random_complex((nc, G), seed=21)
    cot = W.random_complex((nc, G), seed=22)
    gx, _ = plan.adjoint(torch.from_numpy(cot.ravel()).cuda(), xi=torch.from_numpy(xi.ravel()).cuda(), kind=kind)
    ref, _ = APSystem(sub).adjoint(cot, kind=kind, xi=xi)
    assert rel_col_err(gx.cpu().numpy().reshape(nc, G), ref) < 1e-10


@pytest.mark.parametrize("name,sub,tile", CASES, ids=[c[0] for c in CASES])
@pytest.mark.parametrize("kind", ["Q", "P"])
@pytest.mark.parametrize("basis", [True, False])
def test_grad_k_matches_oracle(mdp, name, sub, tile, kind, basis):
    plan = make_plan(mdp, [sub], tile)
    G, nc, _, _ = plan.layout(0)
    cot = W.random_complex((nc, G), seed=23)
    xi = None if basis else W.random_complex((nc, G), seed=24)
    xt = None if basis else torch.from_numpy(xi.ravel()).cuda()
    _, gk = plan.adjoint(torch.from_numpy(cot.ravel()).cuda(), xi=xt, kind=kind, grad_xi=False)
    _, ref = APSystem(sub).adjoint(cot, kind=kind, xi=xi)
    assert abs(gk.item() - ref) < 1e-9 * abs(ref), (gk.item(), ref)


def test_grad_k_matches_central_differences_of_gpu_forward(mdp):
    sub = W.small_subdomain(129, 20.0, W.AP_DIRX_SOMMY, 3)
    plan = mdp.Plan([sub])
    G, nc, _, _ = plan.layout(0)
    cot = torch.from_numpy(W.random_complex((nc, G), seed=25).ravel()).cuda()

    def loss(k):
        plan.update_k([k])
        return float(torch.real(torch.vdot(cot, plan.project())).item())

    d = 1e-4 * sub.k
    fd = (8 * (loss(sub.k + d) - loss(sub.k - d)) - (loss(sub.k + 2 * d) - loss(sub.k - 2 * d))) / (12 * d)
    plan.update_k([sub.k])
    _, gk = plan.adjoint(cot, grad_xi=False)
    assert abs(gk.item() - fd) < 1e-6 * abs(fd), (gk.item(), fd)


@pytest.mark.parametrize("ap", [W.AP_DIRICHLET4, W.AP_DIRX_SOMMY, W.AP_DIRX_SOMMY_PAPER])
def test_dot_product_identity(mdp, ap):
    sub = W.small_subdomain(129, 14.0, ap, 2)
    plan = make_plan(mdp, [sub], 16)
    G, nc, _, _ = plan.layout(0)
    xi = torch.from_numpy(W.random_complex((nc, G), seed=26).ravel()).cuda()
    c = torch.from_numpy(W.random_complex((nc, G), seed=27).ravel()).cuda()
    for kind in ("Q", "P"):
        lhs = torch.vdot(c, plan.project(xi=xi, kind=kind)).item()
        gx, _ = plan.adjoint(c, xi=xi, kind=kind)
        rhs = torch.vdot(gx, xi).item()
        assert abs(lhs - rhs) < 1e-11 * abs(lhs)


def test_multi_subdomain_gradient_is_deterministic_and_per_subdomain(mdp):
    """Four subdomains with different k in one batch over several waves: each grad_k entry
    equals the oracle's for that subdomain, and two runs give identical bits."""
    ks = [12.0, 15.0, 18.0, 21.0]
    subs = [W.unit_subdomain(i, 0, 65, k, W.AP_DIRX_SOMMY, 2) for i, k in enumerate(ks)]
    old = os.environ.get("MDP_WS_MB")
    os.environ["MDP_WS_MB"] = "8"          # force several waves
    try:
        plan = make_plan(mdp, subs, 8)
    finally:
        if old is None:
            del os.environ["MDP_WS_MB"]
        else:
            os.environ["MDP_WS_MB"] = old
    n = plan.output_size
    cot = torch.from_numpy(W.random_complex(n, seed=28)).cuda()
    _, g1 = plan.adjoint(cot, grad_xi=False)
    _, g2 = plan.adjoint(cot, grad_xi=False)
    assert torch.equal(g1, g2)
    blocks = plan.blocks(cot)
    for i, s in enumerate(subs):
        _, ref = APSystem(s).adjoint(blocks[i].cpu().numpy(), kind="Q")
        assert abs(g1[i].item() - ref) < 1e-9 * abs(ref)


def _sampled_adjoint_against_oracle(mdp, subs, picks, tile, seed):
    """One batched gradient pass over every basis column of `subs` (the launch shape the bench
    times), checked on sampled columns: picks[i] lists the columns of subdomain i checked (an
    empty list skips it). grad_xi of the picked columns, for a cotangent on every column,
    against the oracle's; grad_k of each checked subdomain, for the cotangent restricted to
    its picked columns (zero on every other column, so the oracle needs only those), against
    the oracle's; and grad_xi of a zero cotangent column is exactly zero."""
    plan = mdp.Plan(subs, tile_cols=tile)
    n = plan.output_size
    cot = W.random_complex(n, seed=seed)
    gx, _ = plan.adjoint(torch.from_numpy(cot).cuda(), grad_k=False)
    masked = np.zeros_like(cot)
    for i, cols in enumerate(picks):
        G, nc, off, _ = plan.layout(i)
        for c in cols:
            masked[off + c * G: off + (c + 1) * G] = cot[off + c * G: off + (c + 1) * G]
    gx0, gk = plan.adjoint(torch.from_numpy(masked).cuda())
    torch.cuda.synchronize()
    plan.status()
    gxb = [b.cpu().numpy() for b in plan.blocks(gx)]
    gx0b = [b.cpu().numpy() for b in plan.blocks(gx0)]
    cotb = [b.cpu().numpy() for b in plan.blocks(torch.from_numpy(cot))]
    for i, cols in enumerate(picks):
        if not cols:
            continue
        ref_x, ref_k = APSystem(subs[i]).adjoint(cotb[i][cols], kind="Q", cols=cols)
        assert rel_col_err(gxb[i][cols], ref_x) < 1e-10, i
        assert rel_col_err(gx0b[i][cols], ref_x) < 1e-10, i
        others = np.setdiff1d(np.arange(gx0b[i].shape[0]), cols)
        assert np.all(gx0b[i][others] == 0), i
        assert abs(gk[i].item() - ref_k) < 1e-9 * abs(ref_k), (i, gk[i].item(), ref_k)


@pytest.mark.slow
def test_adjoint_at_dd2x2_257_sampled(mdp):
    """The bench's gradient shape: 2x2 subdomains at 257^2, k = 30, mixed AP, M* = 32, tile of
    256 columns, all 1024 columns in one pass; 24 sampled columns of each subdomain (every side
    and both kinds, the highest Chebyshev mode included)."""
    wl = W.dd2x2_257()
    rng = np.random.default_rng(3)
    picks = []
    for s in wl.subdomains:
        nc = 8 * s.n_modes
        hi = [s.n_modes * j + s.n_modes - 1 for j in range(8)]          # T_31 of every side and kind
        rest = rng.choice(np.setdiff1d(np.arange(nc), hi), 16, replace=False).tolist()
        picks.append(sorted(hi + rest))
    _sampled_adjoint_against_oracle(mdp, list(wl.subdomains), picks, 256, seed=31)


@pytest.mark.slow
def test_adjoint_at_checker2x2_513_k100_sampled(mdp):
    """The checkerboard batch (129^2 at k = 10 and 513^2 at k = 100, M* = 48) in one gradient
    pass; checked on the first 513^2, k = 100 subdomain (the most near-propagating modes) at 16
    columns: T_47 of every side and kind, and 8 random ones, and on one 129^2 subdomain."""
    wl = W.checker2x2()
    subs = list(wl.subdomains)
    rng = np.random.default_rng(4)
    picks = [[] for _ in subs]
    big = next(i for i, s in enumerate(subs) if s.nx == 513)
    small = next(i for i, s in enumerate(subs) if s.nx == 129)
    M = subs[big].n_modes
    hi = [M * j + M - 1 for j in range(8)]
    picks[big] = sorted(hi + rng.choice(np.setdiff1d(np.arange(8 * M), hi), 8, replace=False).tolist())
    picks[small] = sorted(rng.choice(8 * M, 8, replace=False).tolist())
    _sampled_adjoint_against_oracle(mdp, subs, picks, 256, seed=32)
