"""Longest chains and greedy maximal antichains on the GPU against the
oracle (exact), and at the full N = 131072 2D order against the longest
increasing subsequence (the height) and the antichain's defining properties,
checked from the coordinates."""
import bisect

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def cs():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1805_04463_gb300 import build
    build.build()
    import paper_1805_04463_gb300 as m
    return m


def _set(cs, kind, n, seed):
    import torch
    b = cs.allocate(kind, n, path=1)
    cs.sprinkle(kind, n, seed, b.coords, b.workspace)
    cs.causal_matrix(kind, n, b.coords, b.bits)
    torch.cuda.synchronize()
    return b


def _lis(seq):
    tails = []
    for x in seq:
        k = bisect.bisect_left(tails, x)
        if k == len(tails):
            tails.append(x)
        else:
            tails[k] = x
    return len(tails)


@pytest.mark.parametrize("kind,n", [(0, 1), (0, 2), (0, 65), (0, 700), (1, 500), (2, 900), (3, 640), (4, 1500),
                                    (5, 800), (6, 900)])
def test_chains_and_antichains_match_oracle(cs, oracle, kind, n):
    b = _set(cs, kind, n, 900 + n + kind)
    bits = b.bits.cpu().numpy().view(np.uint64)
    assert cs.longest_chain(n, b.bits) == oracle.longest_chain(bits)
    rng = np.random.default_rng(n)
    for _ in range(12 if n > 1 else 0):
        i, j = sorted(rng.integers(0, n, 2).tolist())
        assert cs.longest_chain(n, b.bits, i, j) == oracle.longest_chain(bits, i, j), (i, j)
    for s in sorted({0, n // 3, n - 1}):
        size, members = cs.greedy_antichain(n, b.bits, s)
        w_size, w_members = oracle.greedy_antichain(bits, s)
        assert size == w_size
        assert (members.cpu().numpy().view(np.uint64) == w_members).all()


def test_full_size_2d_order(cs):
    n = 131072
    b = _set(cs, 0, n, 0xC5E70003)
    v = b.coords[1].cpu().numpy().astype(np.int64)
    assert cs.longest_chain(n, b.bits) == _lis(v.tolist())
    size, members = cs.greedy_antichain(n, b.bits, 12345)
    a = np.unpackbits(members.cpu().numpy().view(np.uint8), bitorder="little")[:n].astype(bool)
    idx = np.nonzero(a)[0]
    assert a[12345] and idx.size == size
    assert (np.diff(v[idx]) < 0).all()           # pairwise unrelated: v decreases along u
    assert size <= _lis((-v).tolist())           # at most the width
    # maximal: every other element is related to a member
    out = np.nonzero(~a)[0]
    for lo in range(0, out.size, 4096):
        k = out[lo:lo + 4096][:, None]
        rel = ((idx[None, :] > k) & (v[idx][None, :] > v[k])) | ((idx[None, :] < k) & (v[idx][None, :] < v[k]))
        assert rel.any(axis=1).all()
