"""Factorisation on the GPU (mdp_plan_update_k on a device plan) against the host plan's
factorisation of the same wavenumbers, table by table, and the projection after a device
refactor against the oracle at the new k."""
import numpy as np
import pytest

import workloads as W
from oracle.projection import APSystem

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

CASES = [("somm_n65", W.small_subdomain(65, 11.0, W.AP_DIRX_SOMMY, 3), 14.5),
         ("dir4_n65", W.small_subdomain(65, 9.0, W.AP_DIRICHLET4, 3), 7.25),
         ("somm_n61", W.small_subdomain(61, 10.0, W.AP_DIRX_SOMMY, 2), 12.0),
         ("somm_n257_k30", W.dd2x2_257().subdomains[0], 31.5),
         ("somm_paper_n65", W.small_subdomain(65, 9.0, W.AP_DIRX_SOMMY_PAPER, 2), 10.5)]


def cols_close(dev, host, ncomplex):
    """max over table columns of max|dev - host| / max|host| (complex entries by modulus)."""
    dev = dev.reshape(-1, ncomplex, 2)
    host = host.reshape(-1, ncomplex, 2)
    num = np.hypot(*(dev - host).transpose(2, 0, 1)).max(axis=0)
    den = np.hypot(*host.transpose(2, 0, 1)).max(axis=0)
    return float((num / np.maximum(den, 1e-300)).max())


@pytest.mark.parametrize("name,sub,k1", CASES, ids=[c[0] for c in CASES])
def test_device_factorisation_matches_host(mdp, name, sub, k1):
    dplan = mdp.Plan([sub])
    dplan.update_k([k1])
    hplan = mdp.Plan([sub.with_k(k1)], host_only=True)
    td, pd = dplan.read_tables(True)
    th, ph = hplan.read_tables(False)
    info = hplan.sub_info(0)
    off = hplan.table_offsets(0)
    assert off == dplan.table_offsets(0)
    Nq, Nt, i0 = info["Nq"], info["Nt"], info["i0"]
    np.testing.assert_array_equal(pd[off["piv"]:off["piv"] + Nq * Nt], ph[off["piv"]:off["piv"] + Nq * Nt])
    seg_d = td[off["seg"]:off["seg"] + 5 * Nq].reshape(Nq, 5)
    seg_h = th[off["seg"]:off["seg"] + 5 * Nq].reshape(Nq, 5)
    np.testing.assert_array_equal(seg_d, seg_h)
    FW = 8 if info["cplx"] else 4
    fd = td[off["fact"]:off["fact"] + Nq * Nt * FW]
    fh = th[off["fact"]:off["fact"] + Nq * Nt * FW]
    if FW == 8:
        assert cols_close(fd, fh, 4) < 1e-12
    else:
        num = np.abs(fd - fh).reshape(-1, 4).max(0)
        assert (num / np.maximum(np.abs(fh).reshape(-1, 4).max(0), 1e-300)).max() < 1e-12
    assert cols_close(td[off["dT"]:off["dT"] + Nq * Nt * 6], th[off["dT"]:off["dT"] + Nq * Nt * 6], 3) < 1e-13
    # sweep rows i0 .. itop of every mode (rows above itop are never read); the sweep table
    # [Nq][NYf][24] is the last table of a one-subdomain plan (then 32-double alignment padding)
    NYf = (len(th) - off["fs"]) // (Nq * 24)
    worst = 0.0
    for q in range(Nq):
        itop = int(seg_h[q, 4])
        base = off["fs"] + q * NYf * 24
        blk_d = td[base:base + (itop - i0 + 1) * 24].reshape(-1, 24)
        blk_h = th[base:base + (itop - i0 + 1) * 24].reshape(-1, 24)
        np.testing.assert_array_equal(blk_d[:, 22], blk_h[:, 22])
        worst = max(worst, cols_close(blk_d[:, :22].ravel(), blk_h[:, :22].ravel(), 11))
    assert worst < 1e-12


@pytest.mark.parametrize("ap", [W.AP_DIRICHLET4, W.AP_DIRX_SOMMY, W.AP_DIRX_SOMMY_PAPER])
def test_projection_after_device_refactor_matches_oracle(mdp, ap):
    sub = W.small_subdomain(65, 9.0, ap, 3)
    plan = mdp.Plan([sub], tile_cols=16)
    plan.update_k([13.3])
    G, nc, _, _ = plan.layout(0)
    got = plan.project().cpu().numpy().reshape(nc, G)
    ref = APSystem(sub.with_k(13.3)).columns()
    err = (np.abs(got - ref).max(axis=1) / np.abs(ref).max(axis=1)).max()
    assert err < 1e-10
    # back to the first k: the same columns as a fresh plan
    plan.update_k([9.0])
    again = plan.project().cpu().numpy()
    fresh = mdp.Plan([sub], tile_cols=16).project().cpu().numpy()
    assert np.abs(again - fresh).max() <= 1e-12 * np.abs(fresh).max()


def test_device_refactor_reports_resonance_and_recovers(mdp):
    """k on a discrete Dirichlet eigenvalue: the device factorisation reports MDP_ERR_SINGULAR;
    a later update to a regular k succeeds and the columns are right again."""
    from paper_2103_12172_gb300 import MdpError
    n = 33
    nc = n - 1
    h = 1.2 / nc
    lp, lq = -4 * np.sin(np.pi * np.array([2, 3]) / (2 * nc)) ** 2
    k2 = -((lp + lq) / h**2 + lp * lq / (6 * h**2)) / (1 + (lp + lq) / 12)
    sub = W.small_subdomain(n, 5.0, W.AP_DIRICHLET4, 2)
    plan = mdp.Plan([sub])
    with pytest.raises(MdpError) as e:
        plan.update_k([np.sqrt(k2)])
    assert e.value.code == 4  # MDP_ERR_SINGULAR
    plan.update_k([6.0])
    G, ncol, _, _ = plan.layout(0)
    got = plan.project().cpu().numpy().reshape(ncol, G)
    ref = APSystem(sub.with_k(6.0)).columns()
    assert (np.abs(got - ref).max(axis=1) / np.abs(ref).max(axis=1)).max() < 1e-10


def test_factor_reciprocal_is_accurate_to_an_ulp(mdp):
    """The reciprocal of the device factorisation against the correctly rounded 1/x: within 2
    ulp over 60 decades, at the edges of the seed's range and on both sides of them."""
    import ctypes
    from paper_2103_12172_gb300 import _lib
    rng = np.random.default_rng(5)
    x = np.concatenate([10.0 ** rng.uniform(-30, 30, 200000),
                        rng.uniform(0.5, 2.0, 10000),
                        [2.0 ** -120, 2.0 ** 120, 2.0 ** -121, 2.0 ** 121, 1e-300, 1e300, 1.0, 3.0]])
    xd = torch.from_numpy(x).cuda()
    yd = torch.empty_like(xd)
    L = _lib.lib()
    _lib.check(L.mdp_probe_rcp(ctypes.c_void_p(xd.data_ptr()), ctypes.c_void_p(yd.data_ptr()), len(x),
                               ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)), "mdp_probe_rcp")
    y = yd.cpu().numpy()
    r = 1.0 / x                                   # correctly rounded
    ulps = np.abs(y - r) / np.spacing(r)
    assert ulps.max() <= 2.0, ulps.max()


@pytest.mark.parametrize("graph", [False, True])
def test_async_updates_overlap_and_match_synchronous_ones(mdp, graph):
    """mdp_plan_update_k_async: a sweep over k with each refactorisation queued on its own stream
    while the previous projection still runs on another (two table sets). Every step's columns
    equal those of a plan refactored synchronously to the same k, bit for bit; with a graph plan
    the captured graphs follow the table set in use; the gradient after an async update is that of
    the synchronous plan; a singular k shows in the status word."""
    from paper_2103_12172_gb300 import MdpError
    subs = [W.small_subdomain(65, 11.0, W.AP_DIRX_SOMMY, 3), W.small_subdomain(65, 9.0, W.AP_DIRICHLET4, 2)]
    ks = [[11.0, 9.0], [12.5, 9.75], [10.25, 8.5], [13.0, 10.5], [11.75, 9.25]]
    ref = mdp.Plan(subs, tile_cols=32)
    want = []
    for k in ks:
        ref.update_k(k)
        want.append(ref.project().cpu().numpy())
    plan = mdp.Plan(subs, tile_cols=32, graph=graph)
    fs, cs = torch.cuda.Stream(), torch.cuda.Stream()
    outs = [torch.empty(plan.output_size, dtype=torch.complex128, device="cuda") for _ in ks]
    for i, k in enumerate(ks):
        plan.update_k_async(k, stream=fs)          # queued behind nothing on fs: overlaps step i-1 on cs
        plan.project(out=outs[i], stream=cs)
    torch.cuda.synchronize()
    plan.status()
    for o, w in zip(outs, want):
        assert np.array_equal(o.cpu().numpy(), w)
    # a synchronous update after async ones, then the gradient equals the reference's
    plan.update_k(ks[2])
    ref.update_k(ks[2])
    cot = torch.from_numpy(W.random_complex(plan.output_size, seed=5)).cuda()
    g1, k1 = plan.adjoint(cot)
    g2, k2 = ref.adjoint(cot)
    assert torch.equal(g1, g2) and torch.equal(k1, k2)
    # a singular k (a discrete Dirichlet eigenvalue of the second subdomain) is reported late
    n, nc = 65, 64
    h = 1.2 / nc
    lp, lq = -4 * np.sin(np.pi * np.array([2, 3]) / (2 * nc)) ** 2
    kres = float(np.sqrt(-((lp + lq) / h**2 + lp * lq / (6 * h**2)) / (1 + (lp + lq) / 12)))
    plan.update_k_async([11.0, kres], stream=fs)
    torch.cuda.synchronize()
    with pytest.raises(MdpError) as e:
        plan.status()
    assert e.value.code == 4  # MDP_ERR_SINGULAR
    plan.update_k_async(ks[0], stream=fs)
    plan.project(out=outs[0], stream=cs)
    torch.cuda.synchronize()
    plan.status()
    assert np.array_equal(outs[0].cpu().numpy(), want[0])
