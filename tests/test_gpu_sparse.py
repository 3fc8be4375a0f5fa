"""Degree vectors and past/future sparse relation lists on the GPU against
the oracle (bit-exact), across kinds and ragged sizes, and at the full
N = 131072 2D order on sampled rows checked from the coordinates."""
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


@pytest.mark.parametrize("kind,n", [(0, 1), (0, 2), (0, 63), (0, 64), (0, 65), (0, 1000), (1, 129), (2, 3001),
                                    (3, 2049), (4, 4100), (0, 5000), (5, 2000), (6, 2100)])
def test_degrees_and_lists_match_oracle(cs, oracle, kind, n):
    import torch
    b = _set(cs, kind, n, 700 + n + kind)
    bits = b.bits.cpu().numpy().view(np.uint64)
    kin = torch.empty(n, dtype=torch.int32, device="cuda")
    kout = torch.empty(n, dtype=torch.int32, device="cuda")
    cs.degrees(n, b.bits, kin, kout)
    want_in, want_out = oracle.degrees(bits)
    assert (kin.cpu().numpy() == want_in).all() and (kout.cpu().numpy() == want_out).all()
    for direction in (0, 1):
        off, cols = cs.sparse_relations(n, b.bits, direction)
        w_off, w_cols = oracle.sparse_relations(bits, direction)
        assert (off.cpu().numpy() == w_off).all()
        assert (cols.cpu().numpy() == w_cols).all()


def test_too_small_column_buffer_is_reported(cs):
    import torch
    n = 3000
    b = _set(cs, 0, n, 5)
    L = cs.lib()
    ws = torch.empty(L.cs_sparse_workspace_bytes(n), dtype=torch.uint8, device="cuda")
    off = torch.empty(n + 1, dtype=torch.int64, device="cuda")
    assert L.cs_sparse_offsets(n, b.bits.data_ptr(), b.rw, 1, off.data_ptr(), ws.data_ptr(), ws.numel(), None) == 0
    total = int(off[n].item())
    cols = torch.full((total,), -7, dtype=torch.int32, device="cuda")
    cap = total // 2
    assert L.cs_sparse_columns(n, b.bits.data_ptr(), b.rw, 1, off.data_ptr(), cols.data_ptr(), cap,
                               ws.data_ptr(), ws.numel(), None) == 0
    assert cs.workspace_status(ws) == -2          # CS_ENOMEM recorded
    assert (cols[cap:] == -7).all()               # nothing written past the capacity


def test_full_size_2d_order_sampled_rows(cs):
    import torch
    n = 131072
    b = _set(cs, 0, n, 0xC5E70003)
    v = b.coords[1].cpu().numpy().astype(np.int64)
    kin = torch.empty(n, dtype=torch.int32, device="cuda")
    kout = torch.empty(n, dtype=torch.int32, device="cuda")
    cs.degrees(n, b.bits, kin, kout)
    off, cols = cs.sparse_relations(n, b.bits, 1)
    kout_h = kout.cpu().numpy()
    # sum of degrees = related pairs = n(n-1)/2 - inversions of v
    inv = 0
    bit = np.zeros(n + 1, dtype=np.int64)
    for x in v[::-1]:  # Fenwick count of smaller values to the right
        k = x
        s = 0
        while k > 0:
            s += bit[k]
            k -= k & -k
        inv += s
        k = x + 1
        while k <= n:
            bit[k] += 1
            k += k & -k
    R = n * (n - 1) // 2 - inv
    assert int(kin.sum().item()) == int(kout.sum().item()) == R == int(off[n].item())
    off_h = off.cpu().numpy()
    rng = np.random.default_rng(4)
    for i in list(rng.integers(0, n, 24)) + [0, n - 1]:
        want = np.nonzero(v[i + 1:] > v[i])[0] + i + 1
        got = cols[int(off_h[i]):int(off_h[i + 1])].cpu().numpy()
        assert kout_h[i] == want.size and (got == want).all()
