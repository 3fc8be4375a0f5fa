"""The FP4 pair count in bands (cs_mma4_band_panels): when the whole operand
matrix E does not fit the workspace, the supertile rows fall into groups of g
panels and each pair of groups is counted from a band buffer re-expanded
from the bitset.  Every band width must give exactly the oracle's N_k (and
layer sums), on ragged sizes, several groups deep, with one-panel groups and
with a last group of one panel."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

MMA4 = 3


@pytest.fixture(scope="module")
def cs():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1805_04463_gb300 import build
    build.build()
    import paper_1805_04463_gb300 as m
    return m


def _band_bytes(cs, n, g):
    """The smallest workspace whose FP4 count runs in bands of g panels."""
    lo, hi = 1, 1 << 40
    while lo < hi:
        mid = (lo + hi) // 2
        if cs.mma4_band_panels(n, mid) >= g:
            hi = mid
        else:
            lo = mid + 1
    assert cs.mma4_band_panels(n, lo) == g
    return lo


def _bits(cs, kind, n, seed, coords=None):
    import torch
    b = cs.allocate(kind, n, path=1)
    if coords is None:
        cs.sprinkle(kind, n, seed, b.coords, b.workspace)
        assert cs.workspace_status(b.workspace) == 0
    else:
        b.coords.copy_(torch.from_numpy(np.ascontiguousarray(coords, dtype=np.int32)))
    cs.causal_matrix(kind, n, b.coords, b.bits)
    return b


def _count_banded(cs, b, g, kmax=None):
    import torch
    n = b.n
    ws = torch.empty(_band_bytes(cs, n, g), dtype=torch.uint8, device="cuda")
    hist = torch.empty(cs.hist_len(n), dtype=torch.int64, device="cuda")
    if kmax is None:
        cs.interval_abundance(n, b.bits, hist, MMA4, ws)
        layer = None
    else:
        layer = torch.empty((kmax + 1, n), dtype=torch.float64, device="cuda")
        cs.layer_sums(n, b.bits, hist, layer, kmax, path=MMA4, workspace=ws)
    assert cs.workspace_status(ws) == 0
    torch.cuda.synchronize()
    return hist.cpu().numpy(), (None if layer is None else layer.cpu().numpy())


@pytest.mark.parametrize("kind,n,g", [(0, 2000, 1), (0, 2000, 3), (0, 2304, 4), (1, 3001, 2), (2, 4133, 5),
                                      (3, 1777, 1), (4, 5003, 4), (5, 2500, 3), (6, 3000, 2), (0, 769, 1)])
def test_bands_match_oracle(cs, oracle, kind, n, g):
    seed = 0xBA4D0000 + 97 * n + kind
    b = _bits(cs, kind, n, seed)
    nsb = (n + 255) // 256
    assert 1 <= g < nsb
    got, _ = _count_banded(cs, b, g)
    bits = b.bits.cpu().numpy().view(np.uint64)
    assert (bits == oracle.causal_matrix(kind, oracle.sprinkle(kind, n, seed))).all()
    assert (got == oracle.interval_abundance(bits)).all()


@pytest.mark.parametrize("g", [7, 13, 39])
def test_bands_2d_order_20011(cs, oracle, g):
    # 79 supertile rows: 12, 7 and 3 groups (the last of one panel for g = 39),
    # against the bitset-free dominance count
    n, seed = 20011, 0xBA4D2011
    b = _bits(cs, 0, n, seed)
    got, _ = _count_banded(cs, b, g)
    c = oracle.sprinkle(0, n, seed)
    assert (b.coords.cpu().numpy() == c).all()
    assert (got == oracle.interval_abundance_dominance2d(c[1])).all()


def test_bands_chain(cs):
    # every pair related: N_k = n - 1 - k, each band's K range at its longest
    n = 4096
    chain = np.stack([np.arange(n), np.arange(n)]).astype(np.int32)
    b = _bits(cs, 0, n, 0, coords=chain)
    got, _ = _count_banded(cs, b, 2)
    assert (got == np.arange(n - 1, 0, -1)).all()


def test_bands_equal_whole_set_and_layer_sums(cs, oracle):
    # banded and whole-set counts of one bitset agree, and so do the layer
    # sums (phi = 1: exact element counts), against the oracle's
    import torch
    kind, n, seed, kmax = 2, 3001, 0xBA4D3001, 3
    b = _bits(cs, kind, n, seed)
    whole = torch.empty(cs.hist_len(n), dtype=torch.int64, device="cuda")
    ws = torch.empty(cs.interval_abundance_workspace(n, MMA4), dtype=torch.uint8, device="cuda")
    assert cs.mma4_band_panels(n, ws.numel()) == (n + 255) // 256
    cs.interval_abundance(n, b.bits, whole, MMA4, ws)
    for g in (1, 2, 5):
        got, layer = _count_banded(cs, b, g, kmax=kmax)
        assert (got == whole.cpu().numpy()).all(), g
        bits = b.bits.cpu().numpy().view(np.uint64)
        want = oracle.layer_sums(bits, kmax)
        assert (layer == want).all(), g
