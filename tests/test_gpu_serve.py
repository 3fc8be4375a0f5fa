"""Serving loop on the GPU: requests that overlap on the device (admitted
while others are counting, their tiles sharing count launches) must give
exactly the histogram and actions each gives alone."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

EPS = (0.0, 0.05, 0.1, 0.2)


@pytest.fixture(scope="module")
def cs():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1805_04463_gb300 import build
    build.build()
    import paper_1805_04463_gb300 as m
    return m


@pytest.mark.parametrize("path", [1, 2, 3], ids=["popc", "mma", "mma4"])
def test_results_same_alone_and_in_the_mix(cs, path):
    import torch
    from paper_1805_04463_gb300 import serve, workloads
    # a dense burst: 40 requests in 20 ms, N log-uniform in [2^10, 2^13]
    reqs = workloads.serving_requests(rate=2000.0, duration_s=0.02, log2_min=10, log2_max=13, seed=77)
    assert len(reqs) >= 20
    srv = serve.Server(path=path, tick_macs=2e8 if path == 1 else 2e9)  # small ticks: many shared launches
    stats, res = srv.run(reqs)
    assert stats["requests"] == len(reqs) and stats["ticks"] > len(reqs) // 4
    for rid, (t, kind, n, seed) in enumerate(reqs):
        buf = cs.allocate(kind, n, path=1)
        cs.run(buf, seed, eps=EPS)
        torch.cuda.synchronize()
        hist, acts = res[rid]
        assert (hist == buf.hist.cpu().numpy()).all(), rid
        assert (acts == buf.actions.cpu().numpy()[:len(EPS)]).all(), rid


def test_sliced_counting_matches_single_call(cs, oracle):
    # cs_count_jobs with uneven slices of three sets in shared launches
    import torch
    sets = [(0, 3000, 1), (2, 2049, 2), (1, 1500, 3)]
    for path in (1, 2, 3):
        bufs = [cs.allocate(k, n, path=1) for k, n, _ in sets]
        ops = []
        for (k, n, sd), b in zip(sets, bufs):
            cs.sprinkle(k, n, sd, b.coords, b.workspace)
            cs.causal_matrix(k, n, b.coords, b.bits)
            b.hist.zero_()
            if path != 1:
                nb = cs.operands_bytes(n, path)
                t = torch.empty(nb + 1024, dtype=torch.uint8, device="cuda")
                ptr = (t.data_ptr() + 1023) // 1024 * 1024
                cs.prepare_operands(n, b.bits, ptr, nb, path=path)
                ops.append((t, ptr))
            else:
                ops.append((None, None))
        totals = [cs.count_items(n, path) for _, n, _ in sets]
        cuts = [np.unique(np.r_[0, np.sort(np.random.default_rng(s).integers(0, t + 1, 3)), t]) for s, t in
                enumerate(totals)]
        L = cs.lib()
        tb = L.cs_count_jobs_table_bytes(len(sets), path)
        wb = L.cs_count_jobs_workspace_bytes(len(sets), path)
        table = torch.empty(tb + 128, dtype=torch.uint8, pin_memory=True)
        ws = torch.empty(wb, dtype=torch.uint8, device="cuda")
        for step in range(max(len(c) for c in cuts) - 1):
            jobs = []
            for s, ((k, n, sd), b) in enumerate(zip(sets, bufs)):
                c = cuts[s]
                lo, hi = (int(c[step]), int(c[step + 1])) if step + 1 < len(c) else (int(c[-1]), int(c[-1]))
                jobs.append(cs.CountJob(b.bits.data_ptr(), n, b.rw, b.hist.data_ptr(), ops[s][1], lo, hi))
            cs.count_jobs(jobs, path, (table.data_ptr() + 127) // 128 * 128, ws.data_ptr(), wb)
            torch.cuda.synchronize()
        for (k, n, sd), b in zip(sets, bufs):
            want = oracle.interval_abundance(oracle.causal_matrix(k, oracle.sprinkle(k, n, sd)))
            assert (b.hist.cpu().numpy() == want).all(), (path, k, n)


@pytest.mark.parametrize("path", [1, 2, 3], ids=["popc", "mma", "mma4"])
def test_item_shards_sum_to_the_full_count(cs, path):
    # Each of three ranks' shares counted separately (as three GPUs would),
    # summed on the host: the sharded count's single exchange.
    import torch
    from paper_1805_04463_gb300 import replicas
    kind, n, seed = 0, 5000, 31
    full = cs.allocate(kind, n, path=path)
    cs.run(full, seed, eps=())
    torch.cuda.synchronize()
    total = torch.zeros_like(full.hist)
    for rank in range(3):
        b = cs.allocate(kind, n, path=1)
        cs.sprinkle(kind, n, seed, b.coords, b.workspace)
        cs.causal_matrix(kind, n, b.coords, b.bits)
        ptr = None
        if path != 1:
            nb = cs.operands_bytes(n, path)
            ops = torch.empty(nb + 1024, dtype=torch.uint8, device="cuda")
            ptr = (ops.data_ptr() + 1023) // 1024 * 1024
            cs.prepare_operands(n, b.bits, ptr, nb, path=path)
        total += replicas.count_sharded(cs, b, path, 3, rank, dist=None, operands_ptr=ptr)
    assert torch.equal(total, full.hist)


def test_autotuner_installs_a_measured_table(cs, tmp_path):
    # The tuner measures the path per size, the raster side of the tensor
    # counts per size and the multi-set path and run length, installs them,
    # persists them, and a later load installs the same choices; results do
    # not depend on any of them.
    import torch
    from paper_1805_04463_gb300 import tune
    old = (cs.get_auto_paths(), cs.get_auto_tiles(), cs.get_batch_tuning())
    f = str(tmp_path / "tune.json")
    try:
        r = tune.autotune(sizes=(1024, 4096, 16384), tile_sizes=(4096, 16384), rasters=(4, 8, 16),
                          runs=(4, 16), batch_sample=(12, 6), path=f)
        assert cs.get_auto_paths() == [tuple(x) for x in r["paths"]]
        assert [x[0] for x in r["measurements"]] == [1024, 4096, 16384]
        assert all(x[1] > 0 and x[2] > 0 for x in r["measurements"])
        # tile order: every candidate raster side was timed at each tensor-path size
        assert [n for n, _ in r["tile_measurements"]] == [4096, 16384]
        assert all(set(ts) == {"4", "8", "16"} and min(ts.values()) > 0 for _, ts in r["tile_measurements"])
        assert cs.get_auto_tiles() == [tuple(x) for x in r["tiles"]]
        assert all(rs in (4, 8, 16) for _, rs in r["tiles"])
        # multi-set tuning: both tensor paths and both run lengths timed
        assert {(p, run) for p, run, _ in r["batch_measurements"]} == {(2, 4), (2, 16), (3, 4), (3, 16)}
        assert cs.get_batch_tuning() == r["batch"]
        cs.set_auto_paths(old[0])
        cs.set_auto_tiles(old[1])
        cs.set_batch_tuning(*old[2])
        loaded = tune.load(f)
        assert loaded["tiles"] == r["tiles"] and cs.get_auto_tiles() == [tuple(x) for x in r["tiles"]]
        assert loaded["batch"] == r["batch"] and cs.get_batch_tuning() == r["batch"]
        assert loaded["paths"] == r["paths"] and cs.get_auto_paths() == r["paths"]
        # AUTO under the tuned choices gives the same counts as every explicit path
        for n in (1024, 16384):
            hs = []
            for p in (0, 1, 2, 3):
                b = cs.allocate(0, n, path=p)
                cs.run(b, 5, eps=())
                torch.cuda.synchronize()
                hs.append(b.hist.clone())
            assert all(torch.equal(hs[0], h) for h in hs[1:])
    finally:
        cs.set_auto_paths(old[0])
        cs.set_auto_tiles(old[1])
        cs.set_batch_tuning(*old[2])


def test_auto_server_counts_on_the_fp4_pair_path(cs):
    # On a tcgen05 device the server's AUTO choice is the FP4 pair job kernel.
    from paper_1805_04463_gb300 import serve
    assert cs.resolved_path(1 << 16) == cs.PATH_MMA4
    assert serve.Server().count_path == cs.PATH_MMA4
