"""The gamma columns of the middle rows on the tensor cores (k_inv_cols_tc: bf16 digit products
with exact integer accumulation, Ozaki-style splitting) against the FP64 sums of k_inv_cols and
the oracle. Bars: 1e-12 per column against the FP64 kernel (both approximate the same sums),
1e-10 against the oracle; the kernel that ran is read from the plan's per-kernel launch record."""
import os

import numpy as np
import pytest

import workloads as W
from oracle.projection import APSystem

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def rel_col_err(got, ref):
    return float((np.abs(got - ref).max(axis=1) / np.abs(ref).max(axis=1)).max())


def off_centre(n, k, n_modes):
    """Unit subdomain placed off-centre along x in its auxiliary square (margins 0.1 and 0.17)."""
    h = 1.27 / (n - 1)
    return W.Subdomain(0.0, 1.0, 0.0, 1.0, -0.1, -0.17, h, n, n, k, W.AP_DIRX_SOMMY, n_modes)


def project(mdp, subs, tc, xi=None, kind="Q"):
    old = os.environ.get("MDP_TC_COLS")
    os.environ["MDP_TC_COLS"] = "1" if tc else "0"
    try:
        plan = mdp.Plan(subs)
    finally:
        if old is None:
            del os.environ["MDP_TC_COLS"]
        else:
            os.environ["MDP_TC_COLS"] = old
    plan.profile(True)
    out = plan.project(xi=None if xi is None else torch.from_numpy(xi.ravel()).cuda(), kind=kind)
    torch.cuda.synchronize()
    plan.status()
    plan.profile(False)
    prof = plan.profile_read()
    G, nc, _, _ = plan.layout(0)
    res = out.cpu().numpy()[: G * nc].reshape(nc, G)
    plan.close()
    return res, prof


CASES = [
    ("somm257_k30", W.unit_subdomain(0, 0, 257, 30.0, W.AP_DIRX_SOMMY, 32), False, "Q"),
    ("somm257_k30_P", W.unit_subdomain(0, 0, 257, 30.0, W.AP_DIRX_SOMMY, 32), False, "P"),
    ("dir4_129_real", W.small_subdomain(129, 10.0, W.AP_DIRICHLET4, 4), False, "Q"),
    ("dir4_129_user", W.small_subdomain(129, 10.0, W.AP_DIRICHLET4, 4), True, "Q"),
    ("somm129_k20_user_P", W.small_subdomain(129, 20.0, W.AP_DIRX_SOMMY, 3), True, "P"),
    ("offcentre65", off_centre(65, 7.0, 4), False, "Q"),
    ("somm_paper65", W.small_subdomain(65, 11.0, W.AP_DIRX_SOMMY_PAPER, 2), False, "Q"),
]


@pytest.mark.parametrize("name,sub,user,kind", CASES, ids=[c[0] for c in CASES])
def test_tensor_core_columns_match_fp64_and_oracle(mdp, name, sub, user, kind):
    G = mdp.Plan([sub], host_only=True).layout(0)[0]
    nc = 8 * sub.n_modes
    xi = W.random_complex((nc, G), seed=51) if user else None
    got, prof = project(mdp, [sub], True, xi, kind)
    ref64, prof64 = project(mdp, [sub], False, xi, kind)
    assert prof.get("k_inv_cols_tc", (0, 0))[1] > 0 and "k_inv_cols" not in prof, prof
    assert prof64.get("k_inv_cols", (0, 0))[1] > 0 and "k_inv_cols_tc" not in prof64, prof64
    assert rel_col_err(got, ref64) < 1e-12
    cols = list(range(0, nc, max(1, nc // 16)))
    S = APSystem(sub)
    ref = S.columns(cols=cols, kind=kind) if xi is None else S.columns(xi=xi[cols], kind=kind)
    assert rel_col_err(got[cols], ref) < 1e-10


def test_tensor_core_columns_wide_dynamic_range(mdp):
    """User densities whose magnitudes span 24 decades over gamma: every matrix row of the
    contraction is scaled by its own largest exponent, and the result stays within 1e-10 of the
    oracle relative to each column's largest value."""
    sub = W.small_subdomain(129, 10.0, W.AP_DIRX_SOMMY, 2)
    G = mdp.Plan([sub], host_only=True).layout(0)[0]
    rng = np.random.default_rng(52)
    xi = W.random_complex((16, G), seed=53) * 10.0 ** rng.uniform(-12, 12, (16, G))
    got, prof = project(mdp, [sub], True, xi)
    assert prof.get("k_inv_cols_tc", (0, 0))[1] > 0
    ref = APSystem(sub).columns(xi=xi)
    assert rel_col_err(got, ref) < 1e-10


def test_tensor_core_columns_at_the_exactness_limit(mdp):
    """Nq = 2047 (2049^2 grid): each parity half of the modes has 1024 terms, the most that keep
    every digit-product sum within 2^24; equal to the FP64 sums."""
    sub = W.small_subdomain(2049, 60.0, W.AP_DIRX_SOMMY, 2)
    got, prof = project(mdp, [sub], True)
    ref64, _ = project(mdp, [sub], False)
    assert prof.get("k_inv_cols_tc", (0, 0))[1] > 0
    assert rel_col_err(got, ref64) < 1e-12


def test_off_centre_grids_at_and_beyond_the_limit(mdp):
    """Off-centre subdomains sum all modes into every output: Nq = 1023 is on the tensor cores
    (equal to the FP64 sums), Nq = 1100 > 1023 keeps the FP64 kernel."""
    sub = off_centre(1025, 40.0, 2)
    got, prof = project(mdp, [sub], True)
    ref64, _ = project(mdp, [sub], False)
    assert prof.get("k_inv_cols_tc", (0, 0))[1] > 0, prof
    assert rel_col_err(got, ref64) < 1e-12
    sub = off_centre(1101, 40.0, 2)
    got, prof = project(mdp, [sub], True)
    ref64, _ = project(mdp, [sub], False)
    assert prof.get("k_inv_cols", (0, 0))[1] > 0 and "k_inv_cols_tc" not in prof, prof
    assert np.array_equal(got, ref64)


def adjoint(mdp, subs, tc, cot, xi=None, kind="Q"):
    old = os.environ.get("MDP_TC_COLS")
    os.environ["MDP_TC_COLS"] = "1" if tc else "0"
    try:
        plan = mdp.Plan(subs)
    finally:
        if old is None:
            del os.environ["MDP_TC_COLS"]
        else:
            os.environ["MDP_TC_COLS"] = old
    plan.profile(True)
    gx, gk = plan.adjoint(torch.from_numpy(cot).cuda(), xi=None if xi is None else torch.from_numpy(xi).cuda(),
                          kind=kind)
    torch.cuda.synchronize()
    plan.status()
    prof = plan.profile_read()
    plan.profile(False)
    plan.close()
    return gx.cpu().numpy(), gk.cpu().numpy(), prof


@pytest.mark.parametrize("case", ["centred", "off_centre", "user_P"])
def test_adjoint_ring_sums_on_the_tensor_cores_match_fp64(mdp, case):
    """The adjoint's sums over the modes at the 4 ring columns of the inner middle rows
    (k_adj_ring_cols) on the tensor cores: grad_xi and dLoss/dk equal the FP64 sums' to 1e-11
    (the same split as the forward gamma columns, on the adjoint field's own per-column scale)."""
    if case == "centred":
        subs, user, kind = [W.unit_subdomain(0, 0, 257, 30.0, W.AP_DIRX_SOMMY, 8),
                            W.unit_subdomain(1, 0, 129, 12.0, W.AP_DIRICHLET4, 6)], False, "Q"
    elif case == "off_centre":
        subs, user, kind = [off_centre(65, 7.0, 4)], False, "Q"
    else:
        subs, user, kind = [W.small_subdomain(129, 20.0, W.AP_DIRX_SOMMY, 3)], True, "P"
    plan = mdp.Plan(subs)
    n = plan.output_size
    plan.close()
    rng = np.random.default_rng(17)
    cot = rng.standard_normal(n) + 1j * rng.standard_normal(n)
    xi = rng.standard_normal(n) + 1j * rng.standard_normal(n) if user else None
    gx_tc, gk_tc, prof = adjoint(mdp, subs, True, cot, xi, kind)
    gx_64, gk_64, prof64 = adjoint(mdp, subs, False, cot, xi, kind)
    assert "k_adj_ring_cols_tc" in prof and "k_adj_ring_cols" in prof64
    assert np.abs(gx_tc - gx_64).max() <= 1e-11 * np.abs(gx_64).max()
    assert np.abs(gk_tc - gk_64).max() <= 1e-11 * np.abs(gk_64).max()
