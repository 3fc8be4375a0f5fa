"""GPU parity: the CUDA path through the C ABI against the CPU oracle.

Integer results (coordinates, causal-matrix bits, every N_k, the action
bracket) must match bit for bit; actions within 1e-12 relative.  Sizes span
several 128-row tiles with ragged tails; the full-size workloads (N = 1024
2D order, N = 16384 4D diamond, N = 131072 2D order) run in the launch
configuration the benchmark times.
"""
import functools
import math

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

EPS = (0.0, 0.05, 0.1, 0.2, 2.0 ** -6)
TOL = 1e-12


@pytest.fixture(scope="module")
def cs():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1805_04463_gb300 import build
    build.build()
    import paper_1805_04463_gb300 as m
    return m


def _run(cs, kind, n, seed, path=1, coords=None):
    import torch
    b = cs.allocate(kind, n, path=path)
    if coords is None:
        cs.sprinkle(kind, n, seed, b.coords, b.workspace)
        assert cs.workspace_status(b.workspace) == 0
    else:
        b.coords.copy_(torch.from_numpy(np.ascontiguousarray(coords, dtype=np.int32)))
    cs.causal_matrix(kind, n, b.coords, b.bits)
    cs.interval_abundance(n, b.bits, b.hist, path, b.workspace)
    assert cs.workspace_status(b.workspace) == 0
    torch.cuda.synchronize()
    return b


def _np_bits(b):
    return b.bits.cpu().numpy().view(np.uint64)


@pytest.mark.parametrize("kind", [0, 1, 2, 3, 4, 5, 6])
@pytest.mark.parametrize("n", [1, 2, 3, 63, 64, 65, 129, 1000, 4097])
def test_sprinkle_and_relate_bit_exact(cs, oracle, kind, n):
    seed = 0xC5E70000 + 31 * n + kind
    b = _run(cs, kind, n, seed)
    want = oracle.sprinkle(kind, n, seed)
    assert (b.coords.cpu().numpy() == want).all()
    assert (_np_bits(b) == oracle.causal_matrix(kind, want)).all()


@pytest.mark.parametrize("kind", [0, 1, 5])
@pytest.mark.parametrize("n", [12876, 12877, 16384, 20011])
def test_relate_light_cone_large_bit_exact(cs, oracle, kind, n):
    """Light-cone sets above the sizes of the all-kinds test, several row
    tiles of relate chunks and mirror super-tiles deep, ragged and exact
    multiples of 64: every bit, both triangles, against the oracle."""
    seed = 0xC5E72000 + n + kind
    b = _run(cs, kind, n, seed)
    want = oracle.sprinkle(kind, n, seed)
    assert (b.coords.cpu().numpy() == want).all()
    assert (_np_bits(b) == oracle.causal_matrix(kind, want)).all()


@pytest.mark.parametrize("n", [12877, 16384])
def test_relate_chain_antichain_large(cs, oracle, n):
    """Extreme relations at size: a chain (every pair related, every word
    after the diagonal all ones) and an antichain (none)."""
    chain = np.stack([np.arange(n), np.arange(n)]).astype(np.int32)
    anti = np.stack([np.arange(n), np.arange(n)[::-1]]).astype(np.int32)
    for coords in (chain, anti):
        b = _run(cs, 0, n, 0, coords=coords)
        assert (_np_bits(b) == oracle.causal_matrix(0, coords)).all()


@pytest.mark.parametrize("path", [1, 2, 3], ids=["popc", "mma", "mma4"])
@pytest.mark.parametrize("kind,n", [(0, 2), (0, 3), (0, 127), (0, 128), (0, 129), (0, 255), (0, 256), (0, 257),
                                    (0, 300), (0, 511), (0, 1000), (0, 1024), (0, 2049), (0, 4133), (1, 129),
                                    (1, 1500), (1, 3001), (2, 200), (2, 1111), (2, 4096), (2, 5000),
                                    (3, 250), (3, 1777), (3, 4096), (3, 6000), (4, 255), (4, 2500), (4, 5003)])
def test_interval_abundance_bit_exact(cs, oracle, kind, n, path):
    seed = 0xC5E71000 + n + kind
    b = _run(cs, kind, n, seed, path=path)
    bits = _np_bits(b)
    # the bitset the count read is the oracle's for this (kind, n, seed)
    assert (bits == oracle.causal_matrix(kind, oracle.sprinkle(kind, n, seed))).all()
    want = oracle.interval_abundance(bits)
    assert (b.hist.cpu().numpy() == want).all()
    if n <= 256:
        assert (want == oracle.interval_abundance_naive(kind, b.coords.cpu().numpy())).all()


@pytest.mark.parametrize("path", [1, 2, 3], ids=["popc", "mma", "mma4"])
@pytest.mark.parametrize("n", [4, 130, 1000, 3000])
def test_chain_antichain_structures(cs, oracle, n, path):
    chain = np.stack([np.arange(n), np.arange(n)]).astype(np.int32)
    anti = np.stack([np.arange(n), np.arange(n)[::-1]]).astype(np.int32)
    hc = _run(cs, 0, n, 0, coords=chain, path=path).hist.cpu().numpy()
    ha = _run(cs, 0, n, 0, coords=anti, path=path).hist.cpu().numpy()
    assert hc.tolist() == [n - 1 - k for k in range(n - 1)]
    assert not ha.any()
    t = (np.arange(n) * 3).astype(np.int32)
    z = np.zeros(n, np.int32)
    h4 = _run(cs, 2, n, 0, coords=np.stack([t, z, z, z]), path=path).hist.cpu().numpy()
    assert h4.tolist() == hc.tolist()
    h3 = _run(cs, 3, n, 0, coords=np.stack([t, z, z]), path=path).hist.cpu().numpy()
    assert h3.tolist() == hc.tolist()
    h3a = _run(cs, 3, n, 0, coords=np.stack([z + 7, np.arange(n, dtype=np.int32), z]), path=path)
    assert not h3a.hist.cpu().numpy().any()


@pytest.mark.parametrize("path", [1, 2, 3], ids=["popc", "mma", "mma4"])
def test_full_chain_131072_counts_exact(cs, path):
    # Every pair related: |A_ij| = j - i - 1 reaches N - 2 = 131070, the
    # largest count the N = 131072 workload can produce (exactness of the
    # tensor-core FP32 accumulation at the top of its range).
    n = 131072
    chain = np.stack([np.arange(n), np.arange(n)]).astype(np.int32)
    h = _run(cs, 0, n, 0, coords=chain, path=path).hist.cpu().numpy()
    assert (h == np.arange(n - 1, 0, -1)).all()


@pytest.mark.parametrize("kind,n", [(0, 1024), (2, 3000), (1, 2500), (3, 3000), (4, 4000), (5, 3500), (6, 3500)])
def test_action_device_and_host(cs, oracle, kind, n):
    import torch
    seed = 77 + n
    b = _run(cs, kind, n, seed)
    h = b.hist.cpu().numpy()
    d = cs.dim(kind)
    cs.action_device(d, n, b.hist, list(EPS), b.actions, b.bracket, b.workspace)
    torch.cuda.synchronize()
    acts = b.actions.cpu().numpy()
    for e, eps in enumerate(EPS):
        s_or, br_or = oracle.action(d, n, h, eps)
        assert abs(acts[e] - s_or) <= TOL * max(1.0, abs(s_or)), (eps, acts[e], s_or)
        s_h, br_h = cs.action(d, n, h, eps)
        assert abs(s_h - s_or) <= TOL * max(1.0, abs(s_or))
        assert br_h == br_or
    assert int(b.bracket.item()) == oracle.action(d, n, h, 0.0)[1]


@pytest.mark.parametrize("kind,n", [(0, 1024), (2, 700), (3, 900), (4, 800)])
def test_evaluate_host_buffers(cs, oracle, kind, n):
    seed = 4242
    coords = oracle.sprinkle(kind, n, seed)
    want = oracle.interval_abundance(oracle.causal_matrix(kind, coords))
    d = cs.dim(kind)
    h1, a1, br1 = cs.evaluate(kind, n, seed, None, 1, EPS)          # sprinkled on the device
    h2, a2, br2 = cs.evaluate(kind, n, 0, coords, 1, EPS)           # coordinates from the host
    h3, a3, br3 = cs.evaluate(kind, n, seed, None, 3, EPS)          # FP4 tensor path
    assert (h1 == want).all() and (h2 == want).all() and br1 == br2
    assert (h3 == want).all() and br3 == br1 and list(a3) == list(a1)
    for e, eps in enumerate(EPS):
        s_or, _ = oracle.action(d, n, want, eps)
        assert abs(a1[e] - s_or) <= TOL * max(1.0, abs(s_or))
        assert a1[e] == a2[e]


def _light_ray_points(kind, n, seed, scale):
    """Time-sorted 2+1 / 3+1 points, half on light rays x = t + e (e in
    {-1, 0, 1}, other spatial coordinates 0): pairs on one ray are exactly
    null or within a few 2^21 of it; half uniform in the diamond's box."""
    rng = np.random.default_rng(seed)
    d = 3 if kind == 3 else 4
    t = np.sort(rng.integers(0, 1 << 20, n))
    c = np.zeros((d, n), dtype=np.int64)
    c[0] = t
    ray = rng.random(n) < 0.5
    c[1] = np.where(ray, t - (1 << 19) + rng.integers(-1, 2, n), rng.integers(-(1 << 19), 1 << 19, n))
    for k in range(2, d):
        c[k] = np.where(ray, 0, rng.integers(-(1 << 19), 1 << 19, n))
    return (c * scale).astype(np.int32)


@pytest.mark.parametrize("kind", [2, 3], ids=["3+1", "2+1"])
@pytest.mark.parametrize("scale", [1, 1 << 8], ids=["in_fp32_range", "beyond"])
def test_relate_near_light_cone(cs, oracle, kind, scale):
    # The 2+1 and 3+1 relate decides most pairs in FP32 and the ones within
    # its error bound of the light cone exactly; coordinates beyond 2^20 take
    # the exact path throughout.  Null pairs must stay unrelated.
    n = 1500
    c = _light_ray_points(kind, n, 99 + kind, scale)
    b = _run(cs, kind, n, 0, coords=c)
    want = oracle.causal_matrix(kind, c)
    assert (_np_bits(b) == want).all()
    assert (b.hist.cpu().numpy() == oracle.interval_abundance(want)).all()


@pytest.mark.parametrize("kind", [0, 1, 5], ids=["2d_order", "diamond", "square"])
def test_relate_light_cone_coordinate_extremes(cs, oracle, kind):
    # Light-cone coordinates anywhere in [0, 2^31): values at both ends of
    # the range (differences up to 2^31 - 1 either way), many equal values
    # (null pairs) and a ragged tail; labels in time order (u + v, ties by
    # index; for the 2D order u is the label itself).
    rng = np.random.default_rng(7 + kind)
    n = 2000
    top = (1 << 31) - 1
    pool = np.concatenate([np.arange(4), top - np.arange(4), rng.integers(0, 1 << 31, 64)])
    v = rng.choice(pool, n)
    if kind == 0:
        c = np.stack([np.arange(n), v])
    else:
        u = rng.choice(pool, n)
        order = np.lexsort((np.arange(n), u + v))
        c = np.stack([u[order], v[order]])
    c = c.astype(np.int64).astype(np.int32)
    b = _run(cs, kind, n, 0, coords=c)
    want = oracle.causal_matrix(kind, c)
    assert (_np_bits(b) == want).all()
    assert (b.hist.cpu().numpy() == oracle.interval_abundance(want)).all()


def test_invalid_arguments_rejected(cs):
    import torch
    b = cs.allocate(0, 100)
    L = cs.lib()
    st = torch.cuda.current_stream().cuda_stream
    ws = b.workspace
    assert L.cs_interval_abundance(0, b.bits.data_ptr(), b.rw, b.hist.data_ptr(), 1, ws.data_ptr(), ws.numel(), st) == -1
    assert L.cs_interval_abundance(100, b.bits.data_ptr(), 8, b.hist.data_ptr(), 1, ws.data_ptr(), ws.numel(), st) == -1
    assert L.cs_interval_abundance(100, b.bits.data_ptr(), b.rw, b.hist.data_ptr(), 1, ws.data_ptr(), 16, st) == -2
    assert L.cs_sprinkle(9, 100, 1, b.coords.data_ptr(), ws.data_ptr(), ws.numel(), st) == -1
    assert L.cs_causal_matrix(0, 100, b.coords.data_ptr(), None, b.rw, st) == -1


# ------------------------------------------------- full-size workloads

def _check_actions(cs, oracle, kind, n, seed, b, want_hist, path):
    """Local and smeared actions of a full-size set through every entry point
    that forms them -- cs_action_device on the GPU histogram, cs_action on the
    host, and cs_evaluate from host buffers -- against the oracle's action on
    the oracle's own histogram (binary128): within 1e-12 relative, and the
    integer bracket exact.  At these sizes the smeared sum cancels by orders
    of magnitude (Eq. s2d_smeared, s4d_smeared), and the device sum's
    truncation bound, derived from R <= n(n-1)/2, is exercised in full."""
    import torch
    d = cs.dim(kind)
    cs.action_device(d, n, b.hist, list(EPS), b.actions, b.bracket, b.workspace)
    torch.cuda.synchronize()
    acts = b.actions.cpu().numpy()
    _, ev_acts, ev_br = cs.evaluate(kind, n, seed, None, path, EPS)
    br_or = oracle.action(d, n, want_hist, 0.0)[1]
    assert int(b.bracket.item()) == br_or and ev_br == br_or
    for e, eps in enumerate(EPS):
        s_or, br = oracle.action(d, n, want_hist, eps)
        tol = TOL * max(1.0, abs(s_or))
        assert abs(acts[e] - s_or) <= tol, ("device", eps, acts[e], s_or)
        s_h, br_h = cs.action(d, n, want_hist, eps)
        assert abs(s_h - s_or) <= tol and br_h == br, ("host", eps, s_h, s_or)
        assert abs(ev_acts[e] - s_or) <= tol, ("evaluate", eps, ev_acts[e], s_or)


def test_full_2d_order_1024_exact(cs, oracle):
    n, seed = 1024, 0xC5E70001
    b = _run(cs, 0, n, seed)
    c = oracle.sprinkle(0, n, seed)
    assert (b.coords.cpu().numpy() == c).all()
    h = b.hist.cpu().numpy()
    assert (h == oracle.interval_abundance_naive(0, c)).all()
    assert (h == oracle.interval_abundance_dominance2d(c[1])).all()


@pytest.mark.parametrize("path", [1, 2, 3], ids=["popc", "mma", "mma4"])
def test_full_4d_diamond_16384_exact(cs, oracle, path):
    n, seed = 16384, 0xC5E70002
    b = _run(cs, 2, n, seed, path=path)
    c = oracle.sprinkle(2, n, seed)
    assert (b.coords.cpu().numpy() == c).all()
    bits = oracle.causal_matrix(2, c)
    assert (_np_bits(b) == bits).all()
    want = oracle.interval_abundance(bits)
    assert (b.hist.cpu().numpy() == want).all()
    _check_actions(cs, oracle, 2, n, seed, b, want, path)


def _past_counts(v):
    """past[m] = #{i < m : v_i < v_m} by a Fenwick tree over v."""
    n = v.size
    fen = np.zeros(n + 1, dtype=np.int64)
    past = np.zeros(n, dtype=np.int64)
    for m in range(n):
        p, s = int(v[m]), 0
        while p > 0:
            s += fen[p]
            p -= p & -p
        past[m] = s
        p = int(v[m]) + 1
        while p <= n:
            fen[p] += 1
            p += p & -p
    return past


@functools.lru_cache(maxsize=None)
def _oracle_2d_full(n, seed):
    """Oracle sprinkle, bitset-free N_k, links and chain counts of a 2D order (cached)."""
    import oracle as o
    c = o.sprinkle(0, n, seed)
    v = c[1].astype(np.int64)
    past = _past_counts(v)
    future = (n - 1 - v) - (np.arange(n) - past)
    return c, o.interval_abundance_dominance2d(c[1]), o.links_2d(c[1]), int(past.sum()), int((past * future).sum())


@pytest.mark.parametrize("path", [1, 2, 3], ids=["popc", "mma", "mma4"])
def test_full_2d_order_131072(cs, oracle, path):
    # Full size, bench launch configuration: every N_k against the bitset-free
    # dominance count; also sum_k N_k = R, N_0 = links, and the first moment
    # sum_k k N_k = sum_m |past(m)| |future(m)| (chains of three through m).
    n, seed = 131072, 0xC5E70003
    b = _run(cs, 0, n, seed, path=path)
    c, h_dom, links, r, chains3 = _oracle_2d_full(n, seed)
    assert (b.coords.cpu().numpy() == c).all()
    h = b.hist.cpu().numpy()
    assert int(h.sum()) == r
    assert int((np.arange(h.size) * h).sum()) == chains3
    assert int(h[0]) == links
    # the GPU bitset on sampled rows, from the definition (v_i < v_j for i < j)
    v = c[1].astype(np.int64)
    bits = _np_bits(b)
    idx = np.arange(n)
    for i in range(0, n, 997):
        rel = ((v > v[i]) & (idx > i)) | ((v < v[i]) & (idx < i))
        want = np.zeros(b.rw, dtype=np.uint64)
        packed = np.packbits(rel.astype(np.uint8), bitorder="little")
        want[:packed.size // 8] = packed.view(np.uint64)
        assert (bits[i] == want).all(), i
    assert (h == h_dom).all()
    _check_actions(cs, oracle, 0, n, seed, b, h_dom, path)


@functools.lru_cache(maxsize=None)
def _dominance(n, seed):
    import oracle as o
    return o.interval_abundance_dominance2d(o.sprinkle(0, n, seed)[1])


@pytest.mark.parametrize("path", [2, 3], ids=["mma", "mma4"])
def test_largest_set_262144(cs, oracle, path):
    # n = 2^18, the largest 2D order whose FP8 tensor-core operands (137 GB)
    # fit beside its bitset on one GPU: every N_k against the bitset-free
    # dominance count, the total and the first moment of N_k from the
    # coordinates (sum_k N_k = R, sum_k k N_k = chains of three), sampled
    # bitset rows from the definition, and a full chain at this size, whose
    # counts run up to n - 2 = 262142.
    import torch
    n, seed = 1 << 18, 0xC5E70007
    b = _run(cs, 0, n, seed, path=path)
    c = oracle.sprinkle(0, n, seed)
    assert (b.coords.cpu().numpy() == c).all()
    v = c[1].astype(np.int64)
    past = _past_counts(v)
    future = (n - 1 - v) - (np.arange(n) - past)
    h = b.hist.cpu().numpy()
    assert int(h.sum()) == int(past.sum())
    assert int((np.arange(h.size) * h).sum()) == int((past * future).sum())
    # every N_k against the bitset-free dominance count
    assert (h == _dominance(n, seed)).all()
    bits = b.bits.cpu().numpy().view(np.uint64)
    idx = np.arange(n)
    for i in range(0, n, 8191):
        rel = ((v > v[i]) & (idx > i)) | ((v < v[i]) & (idx < i))
        packed = np.packbits(rel.astype(np.uint8), bitorder="little").view(np.uint64)
        assert (bits[i, :packed.size] == packed).all() and not bits[i, packed.size:].any(), i
    del b, bits
    torch.cuda.empty_cache()
    chain = np.stack([np.arange(n), np.arange(n)]).astype(np.int32)
    hc = _run(cs, 0, n, 0, coords=chain, path=path).hist.cpu().numpy()
    assert (hc == np.arange(n - 1, 0, -1)).all()


@pytest.mark.parametrize("path", [1, 2, 3], ids=["popc", "mma", "mma4"])
def test_random_kinds_and_sizes(cs, oracle, path):
    # 40 seeded random (kind, n) pairs, n from 1 to 3000: coordinates,
    # bitsets, every N_k and the actions against the oracle.
    import torch
    rng = np.random.default_rng(20261203 + path)
    for t in range(40):
        kind = int(rng.integers(0, 7))
        n = int(rng.integers(1, 3001))
        seed = int(rng.integers(0, 2 ** 62))
        b = _run(cs, kind, n, seed, path=path)
        c = oracle.sprinkle(kind, n, seed)
        assert (b.coords.cpu().numpy() == c).all(), (kind, n, seed)
        bits = oracle.causal_matrix(kind, c)
        assert (_np_bits(b) == bits).all(), (kind, n, seed)
        want = oracle.interval_abundance(bits)
        assert (b.hist.cpu().numpy() == want).all(), (kind, n, seed)
        d = cs.dim(kind)
        cs.action_device(d, n, b.hist, list(EPS), b.actions, b.bracket, b.workspace)
        torch.cuda.synchronize()
        acts = b.actions.cpu().numpy()
        for e, eps in enumerate(EPS):
            s_or, _ = oracle.action(d, n, want, eps)
            assert abs(acts[e] - s_or) <= TOL * max(1.0, abs(s_or)), (kind, n, seed, eps)
