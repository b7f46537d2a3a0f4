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
