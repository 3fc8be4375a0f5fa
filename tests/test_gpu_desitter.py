"""The thesis's validation experiment on the GPU path (Section "Convergence
and Running Times", Figure "The action in (1+1)-dimensional de Sitter
spacetime"): on the 1+1 de Sitter slab |eta| <= 0.5 the smeared action with
eps = 2^-6, averaged over sprinklings, approaches the Einstein-Hilbert value
S_EH = 4 pi tan(eta_0) = 6.865 once N is large (the thesis sees convergence
set in around N = 2^14 and studies N up to 2^17).

This is a statistical check of the whole pipeline -- sprinkling density,
relation, counts and action together -- against a number the thesis prints,
not a parity test: parity with the oracle is in test_gpu_parity.py.  It is
sensitive: with eta and theta on a grid of 2 pi / 2^20 rad instead of
2 pi / 2^32, grid-null pairs (angle = conformal time difference exactly,
hence unrelated) removed enough near-null links at N = 2^17 to pull the mean
to -0.6.
"""
import math

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

EPS = 2.0 ** -6
ETA0 = (83443 + 0.5) * 2 * math.pi / 2 ** 20     # the slab edge on the grid, 0.4999998 rad
S_EH = 4 * math.pi * math.tan(ETA0)              # 6.8651


@pytest.fixture(scope="module")
def cs():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1805_04463_gb300 import build
    build.build()
    import paper_1805_04463_gb300 as m
    return m


def _actions(cs, n, seeds):
    import torch
    b = cs.allocate(cs.KIND_2D_DS_SLAB, n)
    out = []
    for s in seeds:
        cs.run(b, s, eps=(EPS,))
        torch.cuda.synchronize()
        assert cs.workspace_status(b.workspace) == 0
        out.append(float(b.actions[0].item()))
    return np.array(out)


@pytest.mark.parametrize("log2n,graphs", [(16, 40), (17, 24)])
def test_smeared_action_converges_to_einstein_hilbert(cs, log2n, graphs):
    assert abs(S_EH - 6.865) < 1e-3
    n = 1 << log2n
    s = _actions(cs, n, range(0xD5000000 + 1000 * log2n, 0xD5000000 + 1000 * log2n + graphs))
    se = s.std(ddof=1) / math.sqrt(s.size)
    assert abs(s.mean() - S_EH) < 4 * se, (s.mean(), se)
    # the terms of the sum are orders of magnitude larger than S
    assert s.std(ddof=1) < 0.1 * n * EPS
