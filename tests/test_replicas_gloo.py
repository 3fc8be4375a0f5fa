"""Multi-rank host logic on CPU ranks (gloo, world size 2): item sharding
covers every work item exactly once with balanced shares, and the histogram
all-reduce / timing combine give the whole-job result."""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

from paper_1805_04463_gb300.replicas import combine_timing, shard_chunks


def test_shard_chunks_cover_each_item_once():
    for total in (1, 7, 128, 1000, 266240):
        for world in (1, 2, 3, 8):
            seen = []
            for r in range(world):
                for b, e in shard_chunks(total, world, r):
                    seen.extend(range(b, e))
            assert sorted(seen) == list(range(total))
            sizes = [sum(e - b for b, e in shard_chunks(total, world, r)) for r in range(world)]
            assert max(sizes) - min(sizes) <= 16  # at most one item per round


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, out):
    import torch
    import torch.distributed as dist
    from paper_1805_04463_gb300.replicas import allreduce_hist, combine_timing, shard_chunks
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    # a fake per-item histogram contribution: item t adds 1 to bin t % 17
    total = 1000
    h = torch.zeros(17, dtype=torch.int64)
    for b, e in shard_chunks(total, world, rank):
        for t in range(b, e):
            h[t % 17] += 1
    allreduce_hist(h, dist)
    ms, work = combine_timing(10.0 + rank, 100.0 * (rank + 1), dist)
    out[rank] = (h.tolist(), ms, work)
    dist.destroy_process_group()


@pytest.mark.timeout(120)
def test_gloo_two_ranks_allreduce_and_timing():
    world = 2
    mgr = mp.get_context("spawn").Manager()
    out = mgr.dict()
    port = _free_port()
    mp.spawn(_worker, args=(world, port, out), nprocs=world, join=True)
    want = np.bincount(np.arange(1000) % 17, minlength=17).tolist()
    for r in range(world):
        h, ms, work = out[r]
        assert h == want
        assert ms == 11.0 and work == 300.0


def test_combine_timing_without_group():
    assert combine_timing(5.0, 7.0, None) == (5.0, 7.0)
