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
