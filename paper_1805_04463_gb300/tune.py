"""Autotuner: which interval-count path to run for which set size.

For each size bucket the tuner builds a random 2D order on the device, times
cs_interval_abundance on every path (POPC, FP8 tensor, FP4 tensor; CUDA
events on the launching stream, after a warm-up), checks that the
histograms agree, and keeps the fastest path.  The resulting table
(n_min -> path) is installed as the library's CS_PATH_AUTO policy
(cs_set_auto_paths) and persisted as JSON keyed by the device name, so a
later process can load it instead of measuring again.

    python -m paper_1805_04463_gb300.tune          # measure, install, save
"""
from __future__ import annotations

import json
import os

import paper_1805_04463_gb300 as cs

DEFAULT_SIZES = (1024, 2048, 4096, 8192, 16384, 32768, 65536)
DEFAULT_FILE = os.path.join(os.path.expanduser("~"), ".cache", "causet_gb300", "tune.json")
PATHS = (cs.PATH_POPC, cs.PATH_MMA, cs.PATH_MMA4)


def choose(measurements):
    """Measurements [(n, popc_ms, mma_ms[, mma4_ms])] (None = path not run) ->
    AUTO table [(n_min, path)]: the fastest path per size (POPC on ties), runs
    of equal choices merged, the first entry at 0."""
    ms = sorted(measurements, key=lambda m: m[0])
    table = []
    for m in ms:
        n = m[0]
        times = [(t, p) for p, t in zip(PATHS, m[1:]) if t is not None]
        path = min(times, key=lambda x: (x[0], x[1]))[1] if times else cs.PATH_POPC
        if not table:
            table.append((0, path))
        elif table[-1][1] != path:
            table.append((n, path))
    return table or [(0, cs.PATH_POPC)]


def measure(sizes=DEFAULT_SIZES, reps=3, seed=0x7E57):
    """Time every count path on a random 2D order of each size."""
    import torch
    out = []
    for n in sizes:
        buf = cs.allocate(cs.KIND_2D_ORDER, n, path=cs.PATH_POPC)
        cs.sprinkle(cs.KIND_2D_ORDER, n, seed, buf.coords, buf.workspace)
        cs.causal_matrix(cs.KIND_2D_ORDER, n, buf.coords, buf.bits)
        times, hists = {}, {}
        for path in PATHS:
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
        ref = next(iter(hists.values()))
        if any(not torch.equal(ref, h) for h in hists.values()):
            raise RuntimeError(f"paths disagree at n={n}")
        out.append((n,) + tuple(times[p] for p in PATHS))
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
    for n, *ts in m:
        print(f"n={n:7d}  " + "  ".join(f"{name} {t if t is None else round(t, 3)} ms"
                                        for name, t in zip(("popc", "mma", "mma4"), ts)))
    print("AUTO table:", t)
