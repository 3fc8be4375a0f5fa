"""The largest sets, run after the other GPU tests (this file is collected
after them): CS_PATH_AUTO's memory rule and a 2^19-element random 2D order
evaluated end to end through cs_evaluate from host buffers.

At n = 2^19 the bitset takes 34 GB and the FP4 pair path's operands (one
unmasked matrix of n^2 / 2 bytes plus the masked diagonal blocks) 137 GB, so
AUTO keeps the tensor path; at 2^20 they would take 550 GB and AUTO falls
back to the POPC path, which needs no operands.  The thesis links sets of
N ~ 2^20 on its GPU (Chapter "Causal Set Action", Section "Summary").
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
    assert cs.resolved_path(1 << 20, 0) == POPC           # 137 + 550 GB do not
    assert cs.interval_abundance_workspace(1 << 20, 0) == cs.interval_abundance_workspace(1 << 20, POPC)
    # a caller's lower limit: at 2^17 the FP4 path needs 2.1 + 8.6 GB
    need = cs.bitset_bytes(1 << 17) + cs.interval_abundance_workspace(1 << 17, MMA4)
    cs.set_auto_memory_limit(need)
    assert cs.resolved_path(1 << 17, 0) == MMA4
    cs.set_auto_memory_limit(need - 1)
    assert cs.resolved_path(1 << 17, 0) == POPC
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
