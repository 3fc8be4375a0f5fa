"""Property-based checks (hypothesis, CPU only): for arbitrary small 2D
orders the bitset count, the brute-force count and the bitset-free dominance
count agree and satisfy the interval identities; the library's host action
agrees with the oracle for arbitrary histograms."""
import numpy as np
import pytest

hyp = pytest.importorskip("hypothesis")
from hypothesis import given, settings, strategies as st  # noqa: E402


def _coords(v):
    v = np.asarray(v, dtype=np.int32)
    return np.stack([np.arange(v.size, dtype=np.int32), v])


perms = st.integers(min_value=1, max_value=90).flatmap(
    lambda n: st.permutations(list(range(n))))


@settings(max_examples=60, deadline=None)
@given(perms)
def test_three_counts_agree_on_any_2d_order(oracle, v):
    c = _coords(v)
    n = c.shape[1]
    bits = oracle.causal_matrix(0, c)
    h = oracle.interval_abundance(bits)
    assert (h == oracle.interval_abundance_naive(0, c)).all()
    assert (h == oracle.interval_abundance_dominance2d(c[1])).all()
    va = np.asarray(v)
    # sum_k N_k = related pairs; sum_k k N_k = chains of three i < m < j
    R = sum(1 for i in range(n) for j in range(i + 1, n) if va[i] < va[j])
    assert int(h.sum()) == R
    past = np.array([np.sum(va[:m] < va[m]) for m in range(n)])
    future = np.array([np.sum(va[m + 1:] > va[m]) for m in range(n)])
    assert int((np.arange(h.size) * h).sum()) == int((past * future).sum())
    assert int(h[0]) == oracle.links_2d(c[1])


@settings(max_examples=80, deadline=None)
@given(st.integers(min_value=1, max_value=400), st.sampled_from([2, 3, 4]),
       st.floats(min_value=1e-3, max_value=0.999), st.integers(min_value=0, max_value=2 ** 31))
def test_host_action_matches_oracle_on_any_histogram(oracle, n, dim, eps, seed):
    from paper_1805_04463_gb300 import build
    build.build()
    import paper_1805_04463_gb300 as cs
    rng = np.random.default_rng(seed)
    h = rng.integers(0, 1000, max(n - 1, 1)).astype(np.int64)
    for e in (0.0, eps, 1.0):
        s_lib, b_lib = cs.action(dim, n, h, e)
        s_or, b_or = oracle.action(dim, n, h, e)
        assert b_lib == b_or
        assert abs(s_lib - s_or) <= 1e-12 * max(1.0, abs(s_or))
