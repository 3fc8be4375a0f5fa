"""Failure detection without a GPU fault.

- A bounded in-kernel wait on an mbarrier that nothing completes gives up
  after its limit, records CS_ETIMEOUT in the workspace status word and
  returns; the context stays usable (the next count still matches the oracle).
- Host-side fault injection makes the device allocation or the count launch
  fail as if the CUDA call had failed; the error comes back as a status, the
  library frees what it had allocated, and the next call succeeds.
"""
import time

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

CS_ENOMEM, CS_ECUDA, CS_ETIMEOUT = -2, -3, -4


@pytest.fixture(scope="module")
def cs():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1805_04463_gb300 import build
    build.build()
    import paper_1805_04463_gb300 as m
    yield m
    m.inject_fault(m.FAULT_ALLOC | m.FAULT_LAUNCH, 0)


def _count_matches_oracle(cs, oracle, n=1500, seed=99):
    b = cs.allocate(0, n)
    cs.run(b, seed)
    bits = b.bits.cpu().numpy().view(np.uint64)
    assert (b.hist.cpu().numpy() == oracle.interval_abundance(bits)).all()


def test_bounded_wait_times_out_and_context_survives(cs, oracle):
    import torch
    ws = torch.zeros(256, dtype=torch.uint8, device="cuda")
    t0 = time.perf_counter()
    cs.selftest_wait(ws, 0.05, complete=False)
    assert cs.workspace_status(ws) == CS_ETIMEOUT
    assert time.perf_counter() - t0 < 5.0
    waited_ns = int(ws[16:24].cpu().numpy().view(np.uint64)[0])   # aux[0]
    assert 0.05e9 <= waited_ns < 2e9
    assert torch.cuda.synchronize() is None
    _count_matches_oracle(cs, oracle)


def test_bounded_wait_completes_when_released(cs):
    import torch
    ws = torch.zeros(256, dtype=torch.uint8, device="cuda")
    cs.selftest_wait(ws, 1.0, complete=True)
    assert cs.workspace_status(ws) == 0
    assert int(ws[16:24].cpu().numpy().view(np.uint64)[0]) < 1e9


def test_injected_allocation_failure(cs, oracle):
    cs.inject_fault(cs.FAULT_ALLOC, 1)
    with pytest.raises(cs.CsError) as e:
        cs.evaluate(0, 2000, seed=5, eps=(0.0,))
    assert e.value.status == CS_ENOMEM
    hist, acts, br = cs.evaluate(0, 2000, seed=5, eps=(0.0,))  # next call is clean
    c = oracle.sprinkle(0, 2000, 5)
    assert (hist == oracle.interval_abundance(oracle.causal_matrix(0, c))).all()


@pytest.mark.parametrize("path", [1, 2, 3], ids=["popc", "mma", "mma4"])
def test_injected_launch_failure(cs, oracle, path):
    import torch
    n = 1200
    b = cs.allocate(2, n, path=path)
    cs.sprinkle(2, n, 8, b.coords, b.workspace)
    cs.causal_matrix(2, n, b.coords, b.bits)
    cs.inject_fault(cs.FAULT_LAUNCH, 2)
    for _ in range(2):
        with pytest.raises(cs.CsError) as e:
            cs.interval_abundance(n, b.bits, b.hist, path, b.workspace)
        assert e.value.status == CS_ECUDA
    cs.interval_abundance(n, b.bits, b.hist, path, b.workspace)
    torch.cuda.synchronize()
    assert cs.workspace_status(b.workspace) == 0
    bits = b.bits.cpu().numpy().view(np.uint64)
    assert (b.hist.cpu().numpy() == oracle.interval_abundance(bits)).all()
