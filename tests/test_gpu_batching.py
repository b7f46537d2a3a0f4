"""Batching schedule: CUDA-graph replay, stream capture of the allocation-free
calls, multi-wave schedules with uneven subdomains, and the tile autotuner."""
import numpy as np
import pytest

import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def test_graph_mode_replays_and_recaptures(mdp):
    subs = [W.unit_subdomain(0, 0, 65, 9.0, W.AP_DIRX_SOMMY, 3), W.unit_subdomain(1, 0, 129, 17.0, W.AP_DIRX_SOMMY, 2)]
    ref = mdp.Plan(subs).project().cpu()
    plan = mdp.Plan(subs, graph=True, tile_cols=16)
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        out1 = torch.empty(plan.output_size, dtype=torch.complex128, device="cuda")
        out2 = torch.empty_like(out1)
        for _ in range(3):          # capture, then replays
            plan.project(out=out1)
        plan.project(out=out2)      # new output pointer: a second graph
    s.synchronize()
    assert torch.equal(out1.cpu(), ref) and torch.equal(out2.cpu(), ref)


def test_project_is_capturable_in_a_torch_cuda_graph(mdp):
    """The compute calls allocate nothing, so a caller can capture them in its own graph."""
    sub = W.small_subdomain(65, 11.0, W.AP_DIRX_SOMMY, 2)
    plan = mdp.Plan([sub])
    out = torch.empty(plan.output_size, dtype=torch.complex128, device="cuda")
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        plan.project(out=out)       # warm-up outside capture
    torch.cuda.current_stream().wait_stream(s)
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        plan.project(out=out)
    out.zero_()
    g.replay()
    torch.cuda.synchronize()
    assert torch.equal(out.cpu(), mdp.Plan([sub]).project().cpu())


def test_uneven_multi_wave_schedule_matches_single_items(mdp):
    """Subdomains of three grid sizes and wavenumbers packed into several waves by a small
    workspace budget give, column for column, the per-subdomain results."""
    subs = [W.unit_subdomain(0, 0, 129, 12.0, W.AP_DIRX_SOMMY, 3),
            W.unit_subdomain(1, 0, 257, 33.0, W.AP_DIRX_SOMMY, 2),
            W.unit_subdomain(2, 0, 65, 7.0, W.AP_DIRX_SOMMY, 4)]
    plan = mdp.Plan(subs, tile_cols=8, workspace_bytes=16 << 20)
    out = plan.project()
    for i, s in enumerate(subs):
        one = mdp.Plan([s]).project()
        assert torch.equal(plan.blocks(out)[i].reshape(-1), one)


def test_autotuner_picks_a_candidate_and_caches(mdp, tmp_path):
    from paper_2103_12172_gb300.autotune import tune_tile
    subs = [W.small_subdomain(129, 10.0, W.AP_DIRX_SOMMY, 4)]
    path = str(tmp_path / "tune.json")
    t = tune_tile(subs, candidates=(8, 16, 32), cache_path=path)
    assert t in (8, 16, 32)
    assert tune_tile(subs, candidates=(8, 16, 32), cache_path=path) == t


def test_dedupe_projection_adjoint_and_graph_match_the_plain_plan(mdp):
    """MDP_PLAN_DEDUPE on the 2 x 2 decomposition (four identical subdomains, 129^2): basis
    columns computed once and copied, user densities and the adjoint per subdomain on the shared
    tables, graph replay -- all equal to the plan without deduplication."""
    import numpy as np
    subs = [W.unit_subdomain(i, j, 129, 12.0, W.AP_DIRX_SOMMY, 6) for j in range(2) for i in range(2)]
    plain = mdp.Plan(subs, tile_cols=32)
    dd = mdp.Plan(subs, tile_cols=32, dedupe=True)
    assert dd.leaders() == [0, 0, 0, 0]
    ref = plain.project().cpu().numpy()
    got = dd.project().cpu().numpy()
    assert np.abs(got - ref).max() <= 1e-13 * np.abs(ref).max()
    blocks = dd.blocks(torch.from_numpy(got))
    assert all(torch.equal(b, blocks[0]) for b in blocks[1:])
    xi = torch.from_numpy(W.random_complex((plain.output_size,), seed=21)).cuda()
    r1 = plain.project(xi=xi).cpu().numpy()
    r2 = dd.project(xi=xi).cpu().numpy()
    assert np.abs(r2 - r1).max() <= 1e-13 * np.abs(r1).max()
    cot = torch.from_numpy(W.random_complex((plain.output_size,), seed=22)).cuda()
    g1, k1 = plain.adjoint(cot, xi=xi)
    g2, k2 = dd.adjoint(cot, xi=xi)
    assert torch.allclose(g2, g1, rtol=0, atol=1e-13 * g1.abs().max().item())
    assert torch.allclose(k2, k1, rtol=1e-11, atol=0)
    gplan = mdp.Plan(subs, tile_cols=32, dedupe=True, graph=True)
    s = torch.cuda.Stream()
    out = torch.empty(gplan.output_size, dtype=torch.complex128, device="cuda")
    with torch.cuda.stream(s):
        gplan.project(out=out)
        out.zero_()
        gplan.project(out=out)      # replay of the captured graph, copies included
    s.synchronize()
    assert np.abs(out.cpu().numpy() - ref).max() <= 1e-13 * np.abs(ref).max()


def test_qcache_stores_loads_and_fills_missing_blocks(mdp, tmp_path):
    """QCache: the first call computes and stores one file per distinct problem; the second loads
    them; a deleted entry is recomputed alone. Translated copies of a subdomain share one entry,
    so their blocks agree with their own computation to rounding (the placement differs in the
    last bits), and exactly with each other."""
    import os
    from paper_2103_12172_gb300.qcache import QCache
    subs = [W.unit_subdomain(i, 0, 65, 9.0, W.AP_DIRX_SOMMY, 4) for i in range(3)]
    subs.append(W.unit_subdomain(3, 0, 65, 11.0, W.AP_DIRX_SOMMY, 4))
    plan = mdp.Plan(subs, tile_cols=16)
    ref = plan.project().cpu().numpy()
    cache = QCache(str(tmp_path))
    first = cache.project(plan).cpu().numpy()
    assert np.array_equal(first, ref)
    files = sorted(os.listdir(tmp_path))
    assert len(files) == 2 and all(f.endswith(".npy") for f in files)
    tol = 1e-13 * np.abs(ref).max()
    second = cache.project(plan).cpu().numpy()
    assert np.abs(second - ref).max() <= tol
    b2 = plan.blocks(torch.from_numpy(second))
    assert torch.equal(b2[1], b2[0]) and torch.equal(b2[2], b2[0]) and torch.equal(b2[3], plan.blocks(torch.from_numpy(ref))[3])
    os.remove(os.path.join(tmp_path, files[0]))
    third = cache.project(plan).cpu().numpy()
    assert np.abs(third - ref).max() <= tol and len(os.listdir(tmp_path)) == 2


def test_plan_variants_agree_and_the_tuner_picks_one(mdp, tmp_path):
    """Every kernel variant the autotuner searches (FP64 or tensor-core gamma columns, FFT or
    direct dense rows, FFT block sizes, 2 or 4 staged sweep rows) gives the same columns to
    rounding (1e-12 per column; the oracle pins the default), and tune_plan returns one of them
    and caches it."""
    from paper_2103_12172_gb300.autotune import plan_kwargs, tune_plan
    subs = [W.unit_subdomain(0, 0, 129, 12.0, W.AP_DIRX_SOMMY, 3), W.unit_subdomain(1, 0, 65, 9.0, W.AP_DIRICHLET4, 3)]
    ref = mdp.Plan(subs).project().cpu().numpy()
    variants = [dict(fp64_cols=True), dict(direct_rows=True), dict(fft_block_points=2048),
                dict(fft_block_points=4096), dict(tri_stages=4), dict(tile_cols=8, tri_stages=4, fp64_cols=True)]
    for v in variants:
        got = mdp.Plan(subs, **v).project().cpu().numpy()
        assert np.abs(got - ref).max() <= 1e-12 * np.abs(ref).max(), v
    path = str(tmp_path / "tune.json")
    t = tune_plan(subs, tiles=(16, 64), cache_path=path)
    assert t["tile_cols"] in (16, 24) and t["tri_stages"] in (2, 4) and t["fft_block_points"] in (1024, 2048, 4096)
    assert plan_kwargs(tune_plan(subs, tiles=(16, 64), cache_path=path)) == plan_kwargs(t)
    got = mdp.Plan(subs, **plan_kwargs(t)).project().cpu().numpy()
    assert np.abs(got - ref).max() <= 1e-12 * np.abs(ref).max()
