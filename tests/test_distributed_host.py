"""Multi-rank host logic on CPU (gloo, world size 2): LPT partition of the column units and the
gather of Q blocks, with the oracle computing each rank's columns."""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

import workloads as W
from paper_2103_12172_gb300.distributed import assemble, gather_blocks, lpt_partition, make_units


def test_lpt_partition_covers_every_column_once_and_balances():
    wl = W.dd8x8_mixed()
    subs = list(wl.subdomains)
    for world in (1, 2, 3, 8):
        parts, load = lpt_partition(subs, world, tile_cols=128)
        seen = {}
        for r, lst in enumerate(parts):
            for sub, c0, nc in lst:
                for c in range(c0, c0 + nc):
                    assert (sub, c) not in seen
                    seen[(sub, c)] = r
        assert len(seen) == sum(8 * s.n_modes for s in subs)
        biggest = max(u[3] for u in make_units(subs, 128))
        assert max(load) - min(load) <= 2 * biggest + 1e-9   # LPT bound with one unit of slack
    with pytest.raises(ValueError):
        lpt_partition(subs, 0)


def test_identical_subdomains_share_a_rank_when_balanced():
    subs = [W.unit_subdomain(i, 0, 65, 10.0, 1, 2) for i in range(2)] + \
           [W.unit_subdomain(i, 1, 65, 20.0, 1, 2) for i in range(2)]
    parts, _ = lpt_partition(subs, 2, tile_cols=16)
    ks = [{subs[s].k for s, _, _ in lst} for lst in parts]
    assert all(len(k) == 1 for k in ks)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, result_path):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    from oracle.projection import APSystem
    subs = [W.small_subdomain(33, 5.0, W.AP_DIRX_SOMMY, 2), W.unit_subdomain(1, 0, 33, 7.0, W.AP_DIRX_SOMMY, 1)]
    parts, _ = lpt_partition(subs, world, tile_cols=4)
    systems = {}
    blocks = {}
    for sub, c0, nc in parts[rank]:
        S = systems.setdefault(sub, APSystem(subs[sub]))
        blocks[(sub, c0, nc)] = torch.from_numpy(S.columns(cols=range(c0, c0 + nc)))
    merged = gather_blocks(blocks)
    if rank == 0:
        full = assemble(subs, merged, lambda i: systems.get(i, APSystem(subs[i])).n_gamma)
        ok = all(np.allclose(full[i].numpy(), APSystem(s).columns()) for i, s in enumerate(subs))
        with open(result_path, "w") as f:
            f.write("ok" if ok else "mismatch")
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_gather_reassembles_q(tmp_path):
    path = str(tmp_path / "res.txt")
    mp.spawn(_worker, args=(2, _free_port(), path), nprocs=2, join=True)
    assert open(path).read() == "ok"
