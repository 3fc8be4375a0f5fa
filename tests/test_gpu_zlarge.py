"""The largest sets, run after the other GPU tests (this file is collected
after them): CS_PATH_AUTO's memory rule and random 2D orders of 2^19 and
2^20 elements evaluated end to end through cs_evaluate from host buffers.

At n = 2^19 the bitset takes 34 GB and the FP4 pair path's operands (one
unmasked matrix of n^2 / 2 bytes plus the masked diagonal blocks) 137 GB, so
AUTO keeps the tensor path with the whole matrix; at 2^20 the matrix would
take 550 GB beside a 137 GB bitset, and the FP4 path runs in bands of
supertile rows re-expanded from the bitset (cs_mma4_band_panels) within the
AUTO memory limit.  The thesis links sets of N ~ 2^20 on its GPU (Chapter
"Causal Set Action", Section "Summary").
"""
import functools

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

POPC, MMA, MMA4 = 1, 2, 3


@pytest.fixture(scope="module")
def cs():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1805_04463_gb300 import build
    build.build()
    import paper_1805_04463_gb300 as m
    yield m
    m.set_auto_memory_limit(0)


def test_auto_memory_rule(cs):
    total = cs.get_auto_memory_limit()
    assert total > 200e9                                  # 90% of a GB300's memory
    assert cs.resolved_path(1 << 17, 0) == MMA4
    assert cs.resolved_path(1 << 19, 0) == MMA4           # 34 + 137 GB fit
    ws19 = cs.interval_abundance_workspace(1 << 19, 0)
    assert cs.mma4_band_panels(1 << 19, ws19) == 2048     # the whole matrix
    # 137 + 550 GB do not: bands of g supertile rows within the limit
    assert cs.resolved_path(1 << 20, 0) == MMA4
    ws20 = cs.interval_abundance_workspace(1 << 20, 0)
    assert cs.bitset_bytes(1 << 20) + ws20 <= total
    g = cs.mma4_band_panels(1 << 20, ws20)
    assert 32 <= g < 4096 and cs.mma4_band_panels(1 << 20, ws20 - 1) == g - 1
    # a caller's lower limit: at 2^17 the whole FP4 matrix needs 2.1 + 8.6 GB;
    # below that AUTO keeps the FP4 path in bands down to 32 supertile rows,
    # then takes the POPC path
    n = 1 << 17
    full = cs.interval_abundance_workspace(n, MMA4)
    cs.set_auto_memory_limit(cs.bitset_bytes(n) + full)
    assert cs.resolved_path(n, 0) == MMA4 and cs.mma4_band_panels(n, full) == 512
    cs.set_auto_memory_limit(cs.bitset_bytes(n) + full - 1)
    assert cs.resolved_path(n, 0) == MMA4
    assert cs.mma4_band_panels(n, cs.interval_abundance_workspace(n, 0)) == 255
    lo, hi = 1, full
    while lo < hi:                                        # the smallest workspace of 32-panel bands
        mid = (lo + hi) // 2
        lo, hi = (lo, mid) if cs.mma4_band_panels(n, mid) >= 32 else (mid + 1, hi)
    cs.set_auto_memory_limit(cs.bitset_bytes(n) + lo)
    assert cs.resolved_path(n, 0) == MMA4 and cs.interval_abundance_workspace(n, 0) == lo
    cs.set_auto_memory_limit(cs.bitset_bytes(n) + lo - 1)
    assert cs.resolved_path(n, 0) == POPC
    # an FP8 table entry falls back to the smaller FP4 workspace first
    cs.set_auto_paths([(0, MMA)])
    try:
        assert cs.resolved_path(4096, 0) == MMA
        cs.set_auto_memory_limit(cs.bitset_bytes(4096) + cs.interval_abundance_workspace(4096, MMA4))
        assert cs.resolved_path(4096, 0) == MMA4
    finally:
        cs.set_auto_paths([(0, POPC), (1024, MMA), (4096, MMA4)])
        cs.set_auto_memory_limit(0)
    assert cs.get_auto_memory_limit() == total


@functools.lru_cache(maxsize=None)
def _dominance(n, seed):
    import oracle as o
    c = o.sprinkle(0, n, seed)
    return c, o.interval_abundance_dominance2d(c[1])


def test_evaluate_2d_order_524288_auto(cs, oracle):
    # n = 2^19 through the host-buffer entry point on CS_PATH_AUTO (the FP4
    # pair path at this size): every N_k against the bitset-free dominance
    # count, the bracket and the smeared actions against the oracle's.
    import torch
    torch.cuda.empty_cache()
    n, seed = 1 << 19, 0xC5E70013
    assert cs.resolved_path(n, 0) == MMA4
    eps = (0.0, 0.05, 0.1)
    h, acts, br = cs.evaluate(0, n, seed, None, 0, eps)
    c, want = _dominance(n, seed)
    assert int(h.sum()) == int(want.sum())
    assert (h == want).all()
    s0, br0 = oracle.action(2, n, want, 0.0)
    assert br == br0
    for e, x in enumerate(eps):
        s, _ = oracle.action(2, n, want, x)
        assert abs(acts[e] - s) <= 1e-12 * max(1.0, abs(s)), (x, acts[e], s)


def _past_counts(v):
    """For each j, the number of i < j with v_i < v_j: merge levels of width
    w = 1, 2, 4, ..., each right half searching its block's sorted left half."""
    v = np.asarray(v, dtype=np.int64)
    n = v.size
    idx = np.arange(n)
    past = np.zeros(n, dtype=np.int64)
    w = 1
    while w < n:
        blk, right = idx // (2 * w), (idx % (2 * w)) >= w
        lk = np.sort(blk[~right] * n + v[~right])
        base = blk[right] * n
        past[right] += np.searchsorted(lk, base + v[right]) - np.searchsorted(lk, base)
        w *= 2
    return past


def test_past_counts_helper():
    rng = np.random.default_rng(5)
    v = rng.permutation(1000)
    want = np.array([(v[:j] < v[j]).sum() for j in range(v.size)])
    assert (_past_counts(v) == want).all()


def test_evaluate_2d_order_1048576_bands(cs, oracle):
    # n = 2^20 through cs_evaluate on CS_PATH_AUTO: the FP4 path in bands.
    # The total and the first moment of N_k against the coordinates (sum_k
    # N_k = related pairs, sum_k k N_k = chains of three; every band of
    # supertiles counts pairs and chains of its own), and the bracket and
    # actions as the oracle forms them from this histogram.  Element by
    # element the bands are checked at smaller sizes (test_gpu_bands).
    import torch
    torch.cuda.empty_cache()
    n, seed = 1 << 20, 0xC5E70014
    assert cs.resolved_path(n, 0) == MMA4
    assert cs.mma4_band_panels(n, cs.interval_abundance_workspace(n, 0)) < 4096
    eps = (0.0, 0.05, 0.1)
    h, acts, br = cs.evaluate(0, n, seed, None, 0, eps)
    c = oracle.sprinkle(0, n, seed)
    v = c[1].astype(np.int64)
    past = _past_counts(v)
    future = (n - 1 - v) - (np.arange(n) - past)
    assert int(h.sum()) == int(past.sum())
    assert int((np.arange(h.size) * h).sum()) == int((past * future).sum())
    s0, br0 = oracle.action(2, n, h, 0.0)
    assert br == br0
    for e, x in enumerate(eps):
        s, _ = oracle.action(2, n, h, x)
        assert abs(acts[e] - s) <= 1e-12 * max(1.0, abs(s)), (x, acts[e], s)
