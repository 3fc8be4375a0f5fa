"""Multi-rank host logic on CPU ranks (gloo, world size 2): item sharding
covers every work item exactly once with balanced shares, the histogram
all-reduce / timing combine give the whole-job result, and the loss of a rank
(one that leaves, one that falls silent, one gone during a collective) is
detected on the host within a bounded time instead of hanging the others."""
import os
import socket
import time

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
    import oracle
    from paper_1805_04463_gb300.replicas import allreduce_hist, combine_timing, shard_chunks
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    # Every rank rebuilds the same seeded 2D order and counts only its share
    # of the work items -- here the oracle's rows i (each row contributes the
    # intervals of every pair (i, j > i)), taken in the interleaved ranges
    # shard_chunks assigns -- and the one sum all-reduce gives every rank
    # the whole set's N_k.
    n, seed = 700, 0xC5E70011
    bits = oracle.causal_matrix(0, oracle.sprinkle(0, n, seed))
    h = torch.zeros(oracle.hist_len(n), dtype=torch.int64)
    for b, e in shard_chunks(n, world, rank):
        h += torch.from_numpy(oracle.interval_abundance(bits, threads=1, rows=(b, e, 1)))
    mine = int(h.sum())
    allreduce_hist(h, dist)
    ms, work = combine_timing(10.0 + rank, 100.0 * (rank + 1), dist)
    out[rank] = (h.tolist(), mine, ms, work)
    dist.destroy_process_group()


@pytest.mark.timeout(120)
def test_gloo_two_ranks_allreduce_and_timing(oracle):
    world = 2
    mgr = mp.get_context("spawn").Manager()
    out = mgr.dict()
    port = _free_port()
    mp.spawn(_worker, args=(world, port, out), nprocs=world, join=True)
    n, seed = 700, 0xC5E70011
    want = oracle.interval_abundance(oracle.causal_matrix(0, oracle.sprinkle(0, n, seed)))
    for r in range(world):
        h, mine, ms, work = out[r]
        assert h == want.tolist()
        # each rank counted a real, non-trivial part of the pairs, not all of them
        assert 0 < mine < int(want.sum())
        assert ms == 11.0 and work == 300.0
    assert out[0][1] + out[1][1] == int(want.sum())


def test_combine_timing_without_group():
    assert combine_timing(5.0, 7.0, None) == (5.0, 7.0)


def _worker_failure(rank, world, port, out, mode):
    import datetime

    import torch
    import torch.distributed as dist
    from paper_1805_04463_gb300.replicas import PeerLost, allreduce_hist, check_peers, heartbeat, leave
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    store = dist.TCPStore("127.0.0.1", port + 1, world, rank == 0, timeout=datetime.timedelta(seconds=30))
    dist.init_process_group("gloo", rank=rank, world_size=world, timeout=datetime.timedelta(seconds=5))
    h = torch.ones(5, dtype=torch.int64)
    for step in range(3):
        if rank == 1 and step == 2:
            # rank 1 stops between steps, with nothing in flight
            if mode == "leave":
                leave(store, rank)
            elif mode == "silent":
                time.sleep(3.0)      # alive, but posts nothing for step 2
            out[rank] = "stopped"
            return
        heartbeat(store, rank, step)
        t0 = time.monotonic()
        try:
            if mode == "collective" and step == 2:
                allreduce_hist(h, dist)     # the peer is gone: must fail, not hang
            else:
                check_peers(store, world, rank, step, timeout_s=1.0)
                allreduce_hist(h, dist)
        except PeerLost as e:
            out[rank] = ("peer_lost", e.rank, step, time.monotonic() - t0)
            return
        except RuntimeError as e:       # gloo: the process-group timeout or a closed peer
            out[rank] = ("collective_failed", step, time.monotonic() - t0, type(e).__name__)
            return
    out[rank] = ("finished",)


@pytest.mark.timeout(120)
@pytest.mark.parametrize("mode", ["leave", "silent", "collective"])
def test_gloo_rank_loss_detected_on_host(mode):
    world = 2
    mgr = mp.get_context("spawn").Manager()
    out = mgr.dict()
    port = _free_port()
    while port >= 65535:
        port = _free_port()
    mp.spawn(_worker_failure, args=(world, port, out, mode), nprocs=world, join=True)
    assert out[1] == "stopped"
    r0 = out[0]
    if mode == "collective":
        assert r0[0] == "collective_failed" and r0[1] == 2 and r0[2] < 30.0
    else:
        assert r0[0] == "peer_lost" and r0[1] == 1 and r0[2] == 2
        assert r0[3] < (0.5 if mode == "leave" else 5.0)
