"""Batched ensembles on the GPU: every set of a batch must give exactly the
same coordinates-derived histogram, bracket and actions as the oracle (and
as the single-set entry points), on every count path, also when the batch
launch is captured into a CUDA graph and replayed."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

EPS = (0.0, 0.05, 0.1, 0.2)
TOL = 1e-12

MIXED = [(0, 1, 11), (0, 2, 12), (2, 3, 13), (1, 127, 14), (0, 129, 15), (2, 1000, 16), (1, 2049, 17),
         (0, 4096, 18), (2, 2048, 19), (1, 8192, 20), (0, 300, 21), (2, 4133, 22), (3, 2, 23), (3, 1500, 24),
         (3, 4099, 25), (4, 3, 26), (4, 2222, 27), (4, 8000, 28), (5, 1, 29), (5, 1777, 30), (6, 2, 31),
         (6, 3001, 32)]


@pytest.fixture(scope="module")
def cs():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1805_04463_gb300 import build
    build.build()
    import paper_1805_04463_gb300 as m
    return m


def _check_against_oracle(cs, oracle, b):
    hist = b.hist.cpu().numpy()
    acts = b.actions.cpu().numpy()
    brs = b.brackets.cpu().numpy()
    for s, (kind, n, seed) in enumerate(b.sets):
        c = oracle.sprinkle(kind, n, seed)
        want = oracle.interval_abundance(oracle.causal_matrix(kind, c))
        got = hist[b.hist_offsets[s]:b.hist_offsets[s] + want.size]
        assert (got == want).all(), (s, kind, n)
        d = oracle.dim(kind)
        for e, eps in enumerate(EPS):
            so, bo = oracle.action(d, n, want, eps)
            assert abs(acts[s, e] - so) <= TOL * max(1.0, abs(so)), (s, eps, acts[s, e], so)
            assert brs[s] == bo


@pytest.mark.parametrize("path", [1, 2, 3], ids=["popc", "mma", "mma4"])
def test_mixed_batch_matches_oracle(cs, oracle, path):
    import torch
    b = cs.Batch(MIXED, path=path)
    assert b.path == path
    b.launch(EPS)
    torch.cuda.synchronize()
    assert b.status() == 0
    _check_against_oracle(cs, oracle, b)


@pytest.mark.parametrize("path", [1, 2, 3], ids=["popc", "mma", "mma4"])
def test_batch_equals_single_set_calls(cs, path):
    import torch
    sets = [(1, 4000 + 37 * s, 500 + s) for s in range(6)] + [(2, 2000 + 53 * s, 600 + s) for s in range(4)]
    b = cs.Batch(sets, path=path)
    b.launch(EPS)
    torch.cuda.synchronize()
    for s, (kind, n, seed) in enumerate(sets):
        buf = cs.allocate(kind, n, path=path)
        cs.run(buf, seed, eps=EPS)
        torch.cuda.synchronize()
        assert torch.equal(buf.hist, b.set_hist(s))
        assert torch.equal(buf.actions[:len(EPS)].cpu(), b.actions[s].cpu())


def test_brackets_without_eps(cs, oracle):
    """A batch with no eps still writes every set's exact bracket (one CTA per set)."""
    import torch
    sets = [(1, 900 + 41 * s, 700 + s) for s in range(3)] + [(2, 600, 710), (0, 1024, 711)]
    b = cs.Batch(sets, path=3, n_eps=0)
    b.launch(())
    torch.cuda.synchronize()
    assert b.status() == 0
    brs = b.brackets.cpu().numpy()
    for s, (kind, n, seed) in enumerate(sets):
        want = oracle.interval_abundance(oracle.causal_matrix(kind, oracle.sprinkle(kind, n, seed)))
        assert brs[s] == oracle.action(oracle.dim(kind), n, want, 0.0)[1], s


@pytest.mark.parametrize("path", [0, 3], ids=["auto", "mma4"])
def test_batch_graph_replay(cs, oracle, path):
    import torch
    sets = [(1, 1500 + 100 * s, 900 + s) for s in range(5)] + [(2, 777, 950), (0, 1024, 951)]
    b = cs.Batch(sets, path=path)
    b.launch(EPS)  # warm-up outside capture (sets kernel attributes)
    torch.cuda.synchronize()
    ref = b.hist.clone()
    b.hist.zero_()
    g = torch.cuda.CUDAGraph()
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        with torch.cuda.graph(g, stream=s):
            b.launch(EPS, stream=s)
    for _ in range(3):
        b.hist.zero_()
        g.replay()
        torch.cuda.synchronize()
        assert torch.equal(b.hist, ref)
    _check_against_oracle(cs, oracle, b)


def test_ensemble_workload_sample(cs, oracle):
    # The benchmark ensemble's first and last sets through the batch path.
    import torch
    from paper_1805_04463_gb300 import workloads
    e = workloads.ensemble()
    sets = e[:3] + e[-3:]
    b = cs.Batch(sets, path=0)
    b.launch(EPS)
    torch.cuda.synchronize()
    _check_against_oracle(cs, oracle, b)


def test_ensemble_driver_resumes_on_the_gpu(cs, oracle, tmp_path):
    from paper_1805_04463_gb300 import ensemble
    sets = [(1, 700 + 13 * s, 3100 + s) for s in range(5)] + [(4, 900, 3200), (0, 9000, 3300)]
    out = tmp_path / "ens.jsonl"
    first = ensemble.run(sets[:3], str(out), eps=(0.0, 0.1), chunk=2)
    recs = ensemble.run(sets, str(out), eps=(0.0, 0.1), chunk=2)   # resumes: only the last four run
    assert recs[:3] == first
    for (kind, n, seed), r in zip(sets, recs):
        c = oracle.sprinkle(kind, n, seed)
        want = oracle.interval_abundance(oracle.causal_matrix(kind, c))
        assert r["pairs"] == int(want.sum()) and r["hist_head"] == want[:64].tolist()
        s_or, br = oracle.action(oracle.dim(kind), n, want, 0.1)
        assert r["bracket"] == br and abs(r["actions"]["0.1"] - s_or) <= 1e-12 * max(1.0, abs(s_or))


def test_batch_poll_reports_pending_then_status(cs):
    # cs_batch_poll never waits: while the stream is held by a bounded
    # self-test wait (0.5 s) the launch behind it is still pending; after a
    # synchronise the poll reads the launch's status word (0).  The same
    # holds for a CUDA-graph replay of the launch.
    import torch
    sets = [(1, 1200 + 50 * s, 700 + s) for s in range(4)] + [(2, 900, 760)]
    b = cs.Batch(sets, path=0)
    assert b.poll() == 0                         # nothing launched yet
    s = torch.cuda.Stream()
    hold = torch.zeros(1 << 16, dtype=torch.uint8, device="cuda")
    with torch.cuda.stream(s):
        cs.selftest_wait(hold, 0.5, complete=False, stream=s)
        b.launch(EPS, stream=s)
    assert b.poll() == cs.PENDING
    s.synchronize()
    assert b.poll() == 0
    ref = b.hist.clone()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.stream(s):
        with torch.cuda.graph(g, stream=s):
            b.launch(EPS, stream=s)
    s.synchronize()
    with torch.cuda.stream(s):
        cs.selftest_wait(hold, 0.5, complete=False, stream=s)
        g.replay()
    assert b.poll() == cs.PENDING
    s.synchronize()
    assert b.poll() == 0 and torch.equal(b.hist, ref)
    assert cs.workspace_status(hold) == -4       # the hold itself timed out, as intended
