"""C-ABI checks that need no GPU: the library builds, loads and exports every
symbol include/cs.h declares; layout helpers; host-side action vs the oracle."""
import math
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def cslib():
    from paper_1805_04463_gb300 import build
    build.build()
    import paper_1805_04463_gb300 as cs
    return cs


def _declared_functions():
    names = []
    for h in os.listdir(os.path.join(ROOT, "include")):
        if not h.endswith(".h"):
            continue
        text = open(os.path.join(ROOT, "include", h)).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"^[A-Za-z_][\w \*]*?\b(cs_\w+)\s*\(", text, flags=re.M):
            names.append(m.group(1))
    return sorted(set(names))


def test_header_declares_the_entry_points():
    names = _declared_functions()
    for want in ("cs_sprinkle", "cs_causal_matrix", "cs_interval_abundance", "cs_action", "cs_action_device",
                 "cs_evaluate", "cs_workspace_status", "cs_strerror"):
        assert want in names


def test_library_exports_every_declared_symbol(cslib):
    L = cslib.lib()
    missing = [n for n in _declared_functions() if not hasattr(L, n)]
    assert not missing, missing


def test_layout_helpers(cslib):
    assert cslib.dim(0) == 2 and cslib.dim(1) == 2 and cslib.dim(2) == 4 and cslib.dim(7) == 0
    for n, w in [(1, 16), (64, 16), (1024, 16), (1025, 32), (16384, 256), (131072, 2048), (131073, 2064)]:
        assert cslib.row_words(n) == w
        assert cslib.bitset_bytes(n) == n * w * 8
    assert cslib.hist_len(1) == 1 and cslib.hist_len(1024) == 1023
    assert cslib.coords_bytes(2, 10) == 160 and cslib.coords_bytes(0, 10) == 80
    assert cslib.sprinkle_workspace_bytes(0, 0) == 0       # invalid n
    assert cslib.sprinkle_workspace_bytes(7, 10) == 0      # invalid kind
    assert cslib.interval_abundance_workspace(1000, 9) == 0


def test_fp4_band_planner(cslib):
    """The FP4 count's band width for a workspace size (host arithmetic only):
    the whole matrix E (n rows of ceil(n/256)*128 bytes) plus the masked
    diagonal blocks (256 bytes a row) when it fits; else groups of g
    supertile rows whose band buffer (2 g * 256 rows of E) fits beside the
    diagonal blocks; 0 below one-panel bands."""
    band = cslib.mma4_band_panels
    for n in (256, 1000, 20011, 131072, 1 << 20):
        nsb = (n + 255) // 256
        row = nsb * 128
        up = lambda x, a: -(-x // a) * a
        diag = up(n * 128, 1024) + n * 128              # DU, then DL at a 1024-byte aligned offset
        full = up(1024 + up(n * row, 1024) + diag, 256)
        assert band(n, full + 4096) == nsb
        assert band(n, 1 << 62) == nsb
        assert band(n, 0) == 0 and band(n, 1024 + diag) == 0
        if nsb < 2:
            continue
        one = up(1024 + 512 * row + diag, 256)          # bands of one panel: 512 rows of E
        assert band(n, one) == 1 and band(n, one - 1) == 0
        for g in (1, 2, 3, 7, 32, 100):
            if 2 * g >= nsb:
                continue
            need = up(1024 + 2 * g * 256 * row + diag, 256)
            assert band(n, need) == g and band(n, need - 1) == g - 1, (n, g)
            if need + 2 * 256 * row - 1 < full:
                assert band(n, need + 2 * 256 * row - 1) == g, (n, g)
        # wider workspaces never give narrower bands
        sizes = np.linspace(one, full + 1, 40).astype(np.int64)
        gs = [band(n, int(b)) for b in sizes]
        assert gs == sorted(gs) and gs[-1] == nsb
    assert band(0, 1 << 40) == -1


def test_fp4_band_plan_covers_every_supertile_once(cslib):
    """The band list and the work-item decode of the FP4 count, run on the
    host: over all bands every supertile (si, sj), si <= sj, is counted by
    exactly one work item and none below the diagonal is -- for ragged sizes,
    one-panel groups, a last group of one panel, raster sides that do not
    divide the groups, and the whole set as one band."""
    for n in (256, 257, 2000, 2304, 20011, 65536):
        nsb = (n + 255) // 256
        upper, lower = np.triu_indices(nsb), np.tril_indices(nsb, -1)
        for g in sorted({1, 2, 3, 7, 13, 39, max(1, nsb - 1), nsb, nsb + 5}):
            for raster in (1, 3, 8):
                items, c = cslib.mma4_band_cover(n, g, raster)
                assert items == nsb * (nsb + 1) // 2, (n, g, raster)
                assert (c[upper] == 1).all() and (c[lower] == 0).all(), (n, g, raster)
    L = cslib.lib()
    assert L.cs_mma4_band_cover(1000, 0, 8, None) == -1 and L.cs_mma4_band_cover((1 << 20) + 1, 4, 8, None) == -1


def test_strerror_and_version(cslib):
    L = cslib.lib()
    assert L.cs_strerror(0) == b"ok"
    assert L.cs_strerror(-4).startswith(b"bounded")
    assert b"sm_103a" in L.cs_version()


def test_host_action_matches_oracle(cslib, oracle):
    rng = np.random.default_rng(7)
    for dim in (2, 3, 4):
        for n in (1, 2, 3, 50, 1000, 20000):
            for _ in range(3):
                hl = max(n - 1, 1)
                h = rng.integers(0, 10 ** 6, hl).astype(np.int64)
                for eps in (0.0, -1.0, 1.0, 0.05, 0.1, 0.2, 0.5, 0.9, 1e-3):
                    s_lib, b_lib = cslib.action(dim, n, h, eps)
                    s_or, b_or = oracle.action(dim, n, h, eps)
                    assert b_lib == b_or
                    assert abs(s_lib - s_or) <= 1e-12 * max(1.0, abs(s_or)), (dim, n, eps, s_lib, s_or)


def test_host_action_on_real_abundances(cslib, oracle):
    # Abundances of an actual 2D order: the smeared sum cancels strongly.
    c = oracle.sprinkle(0, 3000, 11)
    h = oracle.interval_abundance(oracle.causal_matrix(0, c))
    for eps in (0.05, 0.1, 0.2, 2.0 ** -6):
        s_lib, _ = cslib.action(2, 3000, h, eps)
        s_or, _ = oracle.action(2, 3000, h, eps)
        assert abs(s_lib - s_or) <= 1e-12 * max(1.0, abs(s_or))
    s_lib, b_lib = cslib.action(2, 3000, h, 0.0)
    assert s_lib == 2 * b_lib


def test_host_action_rejects_bad_arguments(cslib):
    for args in [(1, 10, np.zeros(9, np.int64), 0.0), (5, 10, np.zeros(9, np.int64), 0.0),
                 (2, 10, np.zeros(9, np.int64), 1.5),
                 (2, -1, np.zeros(9, np.int64), 0.0), (2, 10, np.zeros(9, np.int64), float("nan"))]:
        with pytest.raises(cslib.CsError):
            cslib.action(*args)


def test_chain_local_action_closed_form(cslib):
    for n in (3, 10, 1000):
        h = np.array([n - 1 - k for k in range(n - 1)], dtype=np.int64)
        assert cslib.action(2, n, h) == (2.0 * n, n)
        if n >= 4:
            s, b = cslib.action(4, n, h)
            assert b == n - 1 and abs(s - 4 / math.sqrt(6) * (n - 1)) <= 1e-15 * s
        # 2+1: N - n1 + 27/8 n2 - 9/4 n3 = 1 + 9N/8 (bracket reported times 8)
        c3 = (math.pi / (3 * math.sqrt(2))) ** (2 / 3) / math.gamma(5 / 3)
        s, b = cslib.action(3, n, h)
        assert b == 8 + 9 * n and abs(s - c3 * (1 + 9 * n / 8)) <= 1e-14 * s


def test_batch_sizes_on_host(cslib):
    L = cslib.lib()
    arr = cslib._desc_array([(1, 4096, 1), (2, 2048, 2), (0, 1, 3)])
    assert L.cs_batch_hist_len(arr, 3) == 4095 + 2047 + 1
    assert L.cs_batch_workspace_bytes(arr, 3, 1) > 0
    assert L.cs_batch_workspace_bytes(arr, 3, 2) > L.cs_batch_workspace_bytes(arr, 3, 3) > \
        L.cs_batch_workspace_bytes(arr, 3, 1)
    assert L.cs_batch_workspace_bytes(arr, 3, 4) == 0                # no such path
    bad = cslib._desc_array([(1, 8193, 1)])                      # n beyond CS_BATCH_MAX_N
    assert L.cs_batch_workspace_bytes(bad, 1, 1) == 0 and L.cs_batch_hist_len(bad, 1) == -1
    bad = cslib._desc_array([(7, 100, 1)])                       # unknown kind
    assert L.cs_batch_workspace_bytes(bad, 1, 1) == 0


def test_workload_generators_are_seeded():
    from paper_1805_04463_gb300 import workloads
    a, b = workloads.ensemble(), workloads.ensemble()
    assert a == b and len(a) == 768
    assert all(k == 1 for k, _, _ in a[:512]) and all(k == 2 for k, _, _ in a[512:])
    assert abs(np.mean([n for _, n, _ in a[:512]]) - 4096) < 5 * 64 / np.sqrt(512)
    r = workloads.serving_requests(duration_s=2.0)
    assert r == workloads.serving_requests(duration_s=2.0)
    assert all(1024 <= n < 65536 for _, _, n, _ in r)
    assert abs(len(r) - 400) < 5 * 20


def test_auto_path_table_round_trip(cslib):
    old = cslib.get_auto_paths()
    assert old[0][0] == 0
    try:
        cslib.set_auto_paths([(0, 1), (3000, 2), (50000, 1)])
        assert cslib.get_auto_paths() == [(0, 1), (3000, 2), (50000, 1)]
        for bad in ([(1, 1)], [(0, 1), (0, 2)], [(0, 4)], [(0, 1), (10, 2), (5, 1)]):
            with pytest.raises(cslib.CsError):
                cslib.set_auto_paths(bad)
        assert cslib.get_auto_paths() == [(0, 1), (3000, 2), (50000, 1)]
    finally:
        cslib.set_auto_paths(old)


def test_tuner_choice_logic():
    from paper_1805_04463_gb300 import tune
    m = [(1024, 0.1, 0.3), (2048, 0.3, 0.35), (4096, 1.0, 0.5), (8192, 6.0, 1.0), (65536, 900.0, 60.0)]
    assert tune.choose(m) == [(0, 1), (4096, 2)]
    assert tune.choose([(1024, 0.1, None)]) == [(0, 1)]
    assert tune.choose([(1024, 0.5, 0.1), (2048, 0.4, 0.5), (4096, 2.0, 1.0)]) == [(0, 2), (2048, 1), (4096, 2)]
    # with the FP4 path: the fastest of three, None where a path was not run
    assert tune.choose([(1024, 0.1, 0.3, 0.4), (8192, 6.0, 1.0, 1.2), (32768, 90.0, 4.0, 2.0)]) == \
        [(0, 1), (8192, 2), (32768, 3)]
    assert tune.choose([(1024, 0.5, None, 0.2), (2048, 0.4, 0.3, None)]) == [(0, 3), (2048, 2)]


def test_tuner_tile_choice_logic():
    from paper_1805_04463_gb300 import tune
    # the fastest raster side per size; the default side (8) wins within 1%
    m = [(4096, {4: 1.00, 8: 1.005, 16: 1.2}), (16384, {4: 9.0, 8: 8.0, 16: 7.0}), (65536, {4: 50, 8: 40, 16: 45})]
    assert tune.choose_tiles(m) == [(0, 8), (16384, 16), (65536, 8)]
    assert tune.choose_tiles([(4096, {4: 1.0, 8: 2.0})]) == [(0, 4)]
    assert tune.choose_tiles([]) == [(0, 8)]
    # batches: the fastest (path, run) pair
    assert tune.choose_batch([(2, 4, 9.0), (2, 16, 8.0), (3, 4, 7.5), (3, 16, 7.9)]) == (3, 4)


def test_tile_and_batch_tuning_entry_points(cslib):
    L = cslib.lib()
    old_tiles, old_batch = cslib.get_auto_tiles(), cslib.get_batch_tuning()
    assert old_tiles == [(0, 8)] and old_batch == (0, 16)
    try:
        cslib.set_auto_tiles([(0, 8), (32768, 16)])
        assert cslib.get_auto_tiles() == [(0, 8), (32768, 16)]
        cslib.set_batch_tuning(2, 4)
        assert cslib.get_batch_tuning() == (2, 4)
        with pytest.raises(cslib.CsError):
            cslib.set_auto_tiles([(1, 8)])            # must start at 0
        with pytest.raises(cslib.CsError):
            cslib.set_auto_tiles([(0, 8), (0, 4)])    # must increase
        with pytest.raises(cslib.CsError):
            cslib.set_auto_tiles([(0, 33)])           # raster side 1..32
        with pytest.raises(cslib.CsError):
            cslib.set_batch_tuning(4, 16)             # no such path
        with pytest.raises(cslib.CsError):
            cslib.set_batch_tuning(0, 65)             # run 1..64
        assert L.cs_get_batch_tuning(None, None) == -1
    finally:
        cslib.set_auto_tiles(old_tiles)
        cslib.set_batch_tuning(*old_batch)


def test_peak_probe_rejects_bad_arguments(cslib):
    import ctypes
    L = cslib.lib()
    out = ctypes.c_double(0.0)
    assert L.cs_peak_probe(0, 10, 256, ctypes.byref(out)) == -1          # AUTO is not a probe
    assert L.cs_peak_probe(4, 10, 256, ctypes.byref(out)) == -1          # no such path
    assert L.cs_peak_probe(1, 0, 256, ctypes.byref(out)) == -1           # at least one repetition
    assert L.cs_peak_probe(1, (1 << 22) + 1, 256, ctypes.byref(out)) == -1   # at most 2^22
    assert L.cs_peak_probe(1, 10, 257, ctypes.byref(out)) == -1          # 256-byte aligned workspace
    assert L.cs_peak_probe(1, 10, 256, None) == -1


def test_failure_detection_entry_points_reject_bad_arguments(cslib):
    L = cslib.lib()
    assert L.cs_selftest_wait(None, 0.1, 0, None) == -1        # no workspace
    assert L.cs_selftest_wait(256, 0.0, 0, None) == -1         # limit must be > 0
    assert L.cs_selftest_wait(256, 11.0, 0, None) == -1        # and at most 10 s
    assert L.cs_selftest_wait(257, 0.1, 0, None) == -1         # 256-byte aligned
    assert L.cs_inject_fault(-1, 1) == -1
    assert L.cs_inject_fault(cslib.FAULT_ALLOC, -1) == -1
    assert L.cs_inject_fault(cslib.FAULT_ALLOC, 0) == 0


def test_job_items_and_operand_sizes_on_host(cslib):
    # The FP4 pair path counts in 256 x 256 supertiles (half the FP8 tile
    # slots) and keeps one K-padded-to-256 nibble matrix E plus two 128-byte
    # diagonal-block rows per element (DU, DL): a quarter of the FP8 bytes
    # and more.
    L = cslib.lib()
    up = lambda x: (x + 1023) // 1024 * 1024
    for n in (1, 255, 256, 257, 4096, 100000):
        assert L.cs_count_items(n, 2) == 2 * L.cs_count_items(n, 3) > 0
        kp8, kp4 = (n + 127) // 128 * 128, (n + 255) // 256 * 256
        b8, e4, d4 = n * kp8, n * (kp4 // 2), up(n * 128) + n * 128
        assert L.cs_operands_bytes(n, 2) == up(b8) + b8
        assert L.cs_operands_bytes(n, 3) == up(e4) + d4
        assert L.cs_operands_bytes(n, 1) == 0
    assert L.cs_count_items(100, 4) == -1 and L.cs_operands_bytes(100, 4) == 0
    assert L.cs_count_jobs_table_bytes(3, 3) == L.cs_count_jobs_table_bytes(3, 2) > 0
