"""cs_sprinkle_noalloc: the sprinkle entry point for callers that cannot
allocate device memory (for example code running under CUDA-graph stream
capture, or a plugin restricted to memory its host hands it).  Its scratch is
a fixed device array inside the library instead of a caller workspace; its
output must equal cs_sprinkle's for the same arguments.

This file is named to be collected last, so a run that stops at the first
failure has run every other test before reaching it.  It also passes when
run alone in a fresh process.
"""
import ctypes

import pytest

pytestmark = pytest.mark.gpu

MAX_N = 262144  # CS_SPRINKLE_NOALLOC_MAX_N in include/cs.h


@pytest.fixture(scope="module")
def cs():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1805_04463_gb300 import build
    build.build()
    import paper_1805_04463_gb300 as m
    return m


def _with_workspace(cs, kind, n, seed):
    import torch
    coords = torch.empty((cs.dim(kind), n), dtype=torch.int32, device="cuda")
    ws = torch.empty(cs.sprinkle_workspace_bytes(kind, n), dtype=torch.uint8, device="cuda")
    cs.sprinkle(kind, n, seed, coords, ws)
    assert cs.workspace_status(ws) == 0
    return coords


def _no_alloc(cs, kind, n, seed):
    import torch
    coords = torch.full((cs.dim(kind), n), -7, dtype=torch.int32, device="cuda")
    L = cs.lib()
    st = torch.cuda.current_stream().cuda_stream
    assert L.cs_sprinkle_noalloc(kind, n, seed, ctypes.c_void_p(coords.data_ptr()), ctypes.c_void_p(st)) == 0
    torch.cuda.synchronize()
    return coords


@pytest.mark.parametrize("kind", [0, 1, 2, 3, 4, 5, 6])
def test_no_alloc_matches_workspace_entry_point_twice(cs, kind):
    import torch
    # Two calls in a row through the C ABI; the second is smaller, so stale
    # scratch left by the first must not leak into it.
    for n, seed in [(5000, 11 + kind), (1500, 12 + kind)]:
        got = _no_alloc(cs, kind, n, seed)
        want = _with_workspace(cs, kind, n, seed)
        assert torch.equal(got, want), (kind, n)


@pytest.mark.parametrize("kind", [0, 2, 3, 4], ids=["2d_order", "4d_diamond", "3d_diamond", "ds_slab"])
def test_no_alloc_at_its_size_limit_and_beyond(cs, kind):
    # The largest accepted n for the permutation kind, both rejection-sampled
    # diamonds (their attempt counters share the scratch) and the de Sitter
    # slab (its table lookups), then one element more, which is refused.
    import torch
    got = _no_alloc(cs, kind, MAX_N, 99 + kind)
    want = _with_workspace(cs, kind, MAX_N, 99 + kind)
    assert torch.equal(got, want)
    coords = torch.empty((cs.dim(kind), MAX_N + 1), dtype=torch.int32, device="cuda")
    st = torch.cuda.current_stream().cuda_stream
    assert cs.lib().cs_sprinkle_noalloc(kind, MAX_N + 1, 1, ctypes.c_void_p(coords.data_ptr()),
                                        ctypes.c_void_p(st)) == -1  # CS_EINVAL
