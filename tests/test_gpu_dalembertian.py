"""Per-element discrete d'Alembertian on the GPU (Eqs. b2d_local, b4d_local):
the layer sums ride in the interval-count epilogue.  With phi = 1 they are
exact element counts and must match the oracle bit for bit; with a general
field they are double sums in atomic order (tolerance 1e-12 of the summed
magnitudes)."""
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


def _layers(cs, kind, n, seed, path, kmax, phi=None):
    import torch
    b = cs.allocate(kind, n, path=path)
    cs.sprinkle(kind, n, seed, b.coords, b.workspace)
    cs.causal_matrix(kind, n, b.coords, b.bits)
    layer = torch.empty((kmax + 1, n), dtype=torch.float64, device="cuda")
    ph = None if phi is None else torch.from_numpy(phi).cuda()
    cs.layer_sums(n, b.bits, b.hist, layer, kmax, ph, path, b.workspace)
    assert cs.workspace_status(b.workspace) == 0
    torch.cuda.synchronize()
    return b, layer, ph


@pytest.mark.parametrize("path", [1, 2, 3], ids=["popc", "mma", "mma4"])
@pytest.mark.parametrize("kind,n", [(0, 300), (0, 2049), (2, 1500), (1, 4096), (3, 2500)])
def test_layer_sums_exact_for_unit_field(cs, oracle, kind, n, path):
    import torch
    b, layer, _ = _layers(cs, kind, n, 40 + n, path, 4)
    bits = b.bits.cpu().numpy().view(np.uint64)
    want = oracle.layer_sums(bits, 4)
    got = layer.cpu().numpy()
    assert (got == want).all()
    assert (got.sum(axis=1) == b.hist.cpu().numpy()[:5]).all()
    d = cs.dim(kind)
    out = torch.empty(n, dtype=torch.float64, device="cuda")
    cs.dalembertian(d, n, layer, out, ell=0.75)
    torch.cuda.synchronize()
    ref = oracle.dalembertian(d, want, 0.75)
    assert np.allclose(out.cpu().numpy(), ref, rtol=1e-14, atol=0)


@pytest.mark.parametrize("path", [1, 2, 3], ids=["popc", "mma", "mma4"])
def test_layer_sums_general_field(cs, oracle, path):
    import torch
    kind, n = 2, 3000
    phi = np.random.default_rng(3).normal(size=n)
    b, layer, ph = _layers(cs, kind, n, 77, path, 3, phi)
    bits = b.bits.cpu().numpy().view(np.uint64)
    want = oracle.layer_sums(bits, 3, phi)
    mag = oracle.layer_sums(bits, 3, np.abs(phi))
    got = layer.cpu().numpy()
    assert (np.abs(got - want) <= 1e-12 * np.maximum(mag, 1e-300)).all()
    out = torch.empty(n, dtype=torch.float64, device="cuda")
    cs.dalembertian(4, n, layer, out, ell=1.0, phi=ph)
    torch.cuda.synchronize()
    ref = oracle.dalembertian(4, want, 1.0, phi)
    scale = np.abs(phi) + mag[0] + 9 * mag[1] + 16 * mag[2] + 8 * mag[3]
    assert (np.abs(out.cpu().numpy() - ref) <= 1e-12 * 4 / np.sqrt(6) * scale + 1e-300).all()


def test_layer_sums_chain(cs):
    import torch
    n = 1000
    b = cs.allocate(0, n, path=2)
    b.coords.copy_(torch.from_numpy(np.stack([np.arange(n), np.arange(n)]).astype(np.int32)))
    cs.causal_matrix(0, n, b.coords, b.bits)
    phi = torch.arange(n, dtype=torch.float64, device="cuda") * 0.5
    layer = torch.empty((3, n), dtype=torch.float64, device="cuda")
    cs.layer_sums(n, b.bits, b.hist, layer, 2, phi, 2, b.workspace)
    torch.cuda.synchronize()
    for m in range(3):
        want = torch.zeros(n, dtype=torch.float64, device="cuda")
        want[m + 1:] = phi[:n - m - 1]
        assert torch.equal(layer[m], want)
