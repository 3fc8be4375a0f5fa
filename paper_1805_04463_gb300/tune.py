"""Autotuner: which interval-count path to run for which set size.

For each size bucket the tuner builds a random 2D order on the device, times
cs_interval_abundance on both paths (CUDA events on the launching stream,
after a warm-up), checks that the two histograms agree, and keeps the faster
path.  The resulting table (n_min -> path) is installed as the library's
CS_PATH_AUTO policy (cs_set_auto_paths) and persisted as JSON keyed by the
device name, so a later process can load it instead of measuring again.

    python -m paper_1805_04463_gb300.tune          # measure, install, save
"""
from __future__ import annotations

import json
import os

import paper_1805_04463_gb300 as cs

DEFAULT_SIZES = (1024, 2048, 4096, 8192, 16384, 32768, 65536)
DEFAULT_FILE = os.path.join(os.path.expanduser("~"), ".cache", "causet_gb300", "tune.json")


def choose(measurements):
    """Measurements [(n, popc_ms, mma_ms)] -> AUTO table [(n_min, path)]: the
    faster path per size, runs of equal choices merged, the first entry at 0."""
    ms = sorted(measurements)
    table = []
    for n, popc_ms, mma_ms in ms:
        path = cs.PATH_MMA if (mma_ms is not None and mma_ms < popc_ms) else cs.PATH_POPC
        if not table:
            table.append((0, path))
        elif table[-1][1] != path:
            table.append((n, path))
    return table or [(0, cs.PATH_POPC)]


def measure(sizes=DEFAULT_SIZES, reps=3, seed=0x7E57):
    """Time both count paths on a random 2D order of each size."""
    import torch
    out = []
    for n in sizes:
        buf = cs.allocate(cs.KIND_2D_ORDER, n, path=cs.PATH_POPC)
        cs.sprinkle(cs.KIND_2D_ORDER, n, seed, buf.coords, buf.workspace)
        cs.causal_matrix(cs.KIND_2D_ORDER, n, buf.coords, buf.bits)
        times, hists = {}, {}
        for path in (cs.PATH_POPC, cs.PATH_MMA):
            if cs.resolved_path(n, path) != path:
                times[path] = None
                continue
            ws = torch.empty(cs.interval_abundance_workspace(n, path), dtype=torch.uint8, device="cuda")
            hist = torch.empty_like(buf.hist)
            cs.interval_abundance(n, buf.bits, hist, path, ws)  # warm-up
            best = None
            for _ in range(reps):
                a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                a.record()
                cs.interval_abundance(n, buf.bits, hist, path, ws)
                b.record()
                torch.cuda.synchronize()
                t = a.elapsed_time(b)
                best = t if best is None else min(best, t)
            times[path], hists[path] = best, hist
            del ws
        if len(hists) == 2 and not torch.equal(hists[cs.PATH_POPC], hists[cs.PATH_MMA]):
            raise RuntimeError(f"paths disagree at n={n}")
        out.append((n, times[cs.PATH_POPC], times[cs.PATH_MMA]))
    return out


def device_key():
    import torch
    p = torch.cuda.get_device_properties(torch.cuda.current_device())
    return f"{p.name} sm_{p.major}{p.minor} x{p.multi_processor_count}"


def save(table, measurements, path=DEFAULT_FILE):
    os.makedirs(os.path.dirname(path), exist_ok=True)
    data = {}
    if os.path.exists(path):
        with open(path) as f:
            data = json.load(f)
    data[device_key()] = {"table": table, "measurements": measurements}
    with open(path, "w") as f:
        json.dump(data, f, indent=1)


def load(path=DEFAULT_FILE):
    """Install a saved table for this device; returns it, or None if there is none."""
    if not os.path.exists(path):
        return None
    with open(path) as f:
        entry = json.load(f).get(device_key())
    if not entry:
        return None
    table = [tuple(x) for x in entry["table"]]
    cs.set_auto_paths(table)
    return table


def autotune(sizes=DEFAULT_SIZES, install=True, persist=True, path=DEFAULT_FILE):
    m = measure(sizes)
    table = choose(m)
    if install:
        cs.set_auto_paths(table)
    if persist:
        save(table, m, path)
    return table, m


if __name__ == "__main__":
    t, m = autotune()
    for n, a, b in m:
        print(f"n={n:7d}  popc {a:9.3f} ms  mma {b if b is None else round(b, 3)} ms")
    print("AUTO table:", t)
