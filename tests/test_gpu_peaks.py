"""Peak probes on the GPU: the innermost operation of each count path alone
on every SM (cs_peak_probe), the figures beside the roofline denominators."""
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


def test_peak_probes(cs):
    # Rates in the range the device's unit counts allow (about 16 POPC per SM
    # per clock; FP8 and FP4 tensor rates in PFLOP/s), the count kernels'
    # MMA shapes running without a status error.
    popc = cs.peak_probe(cs.PATH_POPC, 1 << 12)
    fp8 = cs.peak_probe(cs.PATH_MMA, 1 << 12)
    fp4 = cs.peak_probe(cs.PATH_MMA4, 1 << 12)
    assert 1e12 < popc < 1e13
    assert 1e15 < fp8 < 1e16
    assert 1.5 * fp8 < fp4 < 4 * fp8


def test_peak_probe_after_counts_leaves_them_exact(cs, oracle):
    # A probe between two counts on the same context changes nothing.
    import numpy as np
    import torch
    n = 5000
    b = cs.allocate(0, n)
    cs.run(b, 11, eps=())
    torch.cuda.synchronize()
    h1 = b.hist.clone()
    cs.peak_probe(cs.PATH_MMA4, 1 << 10)
    cs.run(b, 11, eps=())
    torch.cuda.synchronize()
    assert torch.equal(h1, b.hist)
    bits = b.bits.cpu().numpy().view(np.uint64)
    assert (b.hist.cpu().numpy() == oracle.interval_abundance(bits)).all()
