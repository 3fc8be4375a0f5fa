"""Multi-rank host logic: replicas and item sharding.

Two ways to use several GPUs (one process per GPU):

- Replicas (weak scaling): every rank evaluates its own sets; nothing is
  exchanged on the data path.  Only the timing is combined: the job's time
  is the slowest rank's, its work the sum over ranks (`combine_timing`).
- Item sharding (one large set): the interval count of a set is a fixed list
  of independent work items (`cs_count_items`).  Every rank rebuilds the set
  from its seed (O(n^2), cheap next to the O(n^3) count), counts an
  interleaved share of the items (`shard_chunks` + `cs_count_jobs`), and one
  sum all-reduce of the int64 histogram gives every rank the full N_k
  (`allreduce_hist`).  Interleaving many small chunks balances the ranks
  because the items of a set are ordered by decreasing cost.

The thesis distributes its pair loop across computers with MPI (Section
"MPI Optimization"); here the unit is a tile of the count, and the only
exchange is the final histogram.

Failure detection between ranks is host-side: each rank posts a heartbeat
(its step number) to the process group's key-value store before every
launch, and `check_peers` confirms, with a time limit, that every other rank
has reached the same step -- or raises `PeerLost` naming the rank that left
or fell silent -- so no rank launches work whose exchange would wait on a
dead peer.  Ranks leave only between steps (`leave`).
"""
from __future__ import annotations

import time


class PeerLost(RuntimeError):
    """Another rank left the job or stopped posting heartbeats."""

    def __init__(self, rank, why):
        self.rank = rank
        super().__init__(f"rank {rank} {why}")


def _hb_key(rank):
    return f"cs_hb/{rank}"


def heartbeat(store, rank: int, step: int):
    """Post that `rank` is about to run step `step`."""
    store.set(_hb_key(rank), str(step))


def leave(store, rank: int):
    """Post that `rank` leaves the job (call between steps only)."""
    store.set(_hb_key(rank), "left")


def check_peers(store, world: int, rank: int, step: int, timeout_s: float = 2.0, poll_s: float = 0.005):
    """Wait until every other rank has posted a heartbeat for a step >= `step`.
    Raises PeerLost for a rank that posted `leave` or did not reach `step`
    within `timeout_s` seconds."""
    deadline = time.monotonic() + timeout_s
    pending = [r for r in range(world) if r != rank]
    while pending:
        still = []
        for r in pending:
            key = _hb_key(r)
            if store.check([key]):
                v = store.get(key).decode()
                if v == "left":
                    raise PeerLost(r, "left the job")
                if int(v) >= step:
                    continue
            still.append(r)
        pending = still
        if pending:
            if time.monotonic() > deadline:
                raise PeerLost(pending[0], f"posted no heartbeat for step {step} within {timeout_s} s")
            time.sleep(poll_s)


def shard_chunks(total_items: int, world: int, rank: int, rounds: int = 16):
    """Contiguous item ranges [b, e) assigned to `rank`.  The items are cut into
    `rounds` consecutive rounds, each round into `world` nearly equal pieces;
    ranks take pieces in snake order (0..W-1, then W-1..0, ...), so every rank
    gets items from every cost level and the shares differ by at most one item
    per round."""
    if total_items <= 0:
        return []
    rounds = max(1, min(rounds, total_items))
    out = []
    for k in range(rounds):
        lo, hi = total_items * k // rounds, total_items * (k + 1) // rounds
        p = rank if k % 2 == 0 else world - 1 - rank
        b, e = lo + (hi - lo) * p // world, lo + (hi - lo) * (p + 1) // world
        if e > b:
            out.append((b, e))
    return out


def combine_timing(elapsed_ms: float, work: float, dist=None):
    """(max elapsed over ranks, total work over ranks); identity without a process group."""
    if dist is None or not dist.is_initialized():
        return elapsed_ms, work
    import torch
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([elapsed_ms], dtype=torch.float64, device=dev)
    w = torch.tensor([work], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.all_reduce(w, op=dist.ReduceOp.SUM)
    return float(t[0]), float(w[0])


def allreduce_hist(hist, dist=None):
    """Sum an int64 histogram tensor over ranks in place (the single exchange of
    the sharded count)."""
    if dist is not None and dist.is_initialized():
        dist.all_reduce(hist, op=dist.ReduceOp.SUM)
    return hist


def count_sharded(cs, buf, path, world, rank, dist=None, operands_ptr=None, stream=None):
    """Count this rank's share of the items of the set in `buf` (bits built),
    then all-reduce the histogram.  Returns the histogram tensor."""
    import torch
    total = cs.count_items(buf.n, path)
    ranges = shard_chunks(total, world, rank)
    buf.hist.zero_()
    if ranges:
        L = cs.lib()
        tb = L.cs_count_jobs_table_bytes(len(ranges), path)
        wb = L.cs_count_jobs_workspace_bytes(len(ranges), path)
        table = torch.empty(tb + 128, dtype=torch.uint8, pin_memory=True)
        ws = torch.empty(wb, dtype=torch.uint8, device=buf.bits.device)
        jobs = [cs.CountJob(buf.bits.data_ptr(), buf.n, buf.rw, buf.hist.data_ptr(), operands_ptr, b, e)
                for b, e in ranges]
        cs.count_jobs(jobs, path, (table.data_ptr() + 127) // 128 * 128, ws.data_ptr(), wb, stream)
        torch.cuda.synchronize()
    return allreduce_hist(buf.hist, dist)
