"""Autotuner: which interval-count path, and which tile order, for which size.

Three measured choices, each timed on the running GPU (CUDA events on the
launching stream, after a warm-up; the histograms of every candidate must
agree):

- the CS_PATH_AUTO path table: for each size bucket a random 2D order is
  counted on every path (POPC, FP8 tensor, FP4 tensor pairs) and the fastest
  path kept (cs_set_auto_paths);
- the raster side of the single-set tensor counts: for each size bucket the
  count on the path AUTO now picks is timed with each candidate raster side
  (the supertiles are handed out in raster blocks of side R so that the CTAs
  running at one time share operand panels in L2) and the fastest kept
  (cs_set_auto_tiles);
- the multi-set counts: a sample of the ensemble workload (1+1 and 3+1
  diamonds of Poisson sizes) is run as one batch on each tensor path with
  each candidate queue run length, and the fastest pair kept
  (cs_set_batch_tuning).

The choices are installed in the library and persisted as JSON keyed by the
device name, so a later process can load them instead of measuring again.

    python -m paper_1805_04463_gb300.tune          # measure, install, save
"""
from __future__ import annotations

import json
import os

import paper_1805_04463_gb300 as cs

DEFAULT_SIZES = (1024, 2048, 4096, 8192, 16384, 32768, 65536)
DEFAULT_TILE_SIZES = (4096, 16384, 65536, 131072)
DEFAULT_RASTERS = (4, 8, 16)
DEFAULT_RUNS = (4, 8, 16, 32)
DEFAULT_FILE = os.path.join(os.path.expanduser("~"), ".cache", "causet_gb300", "tune.json")
PATHS = (cs.PATH_POPC, cs.PATH_MMA, cs.PATH_MMA4)
RASTER_DEFAULT = 8


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


def choose_tiles(measurements, tolerance=0.01):
    """Measurements [(n, {raster: ms})] -> tile table [(n_min, raster)]: per size the
    fastest raster side, unless the default side is within `tolerance` of it
    (timing noise does not move the choice); equal neighbours merged, the
    first entry at 0."""
    table = []
    for n, times in sorted(measurements, key=lambda m: m[0]):
        times = {int(r): t for r, t in times.items() if t is not None}
        if not times:
            continue
        best = min(times, key=lambda r: (times[r], r))
        if RASTER_DEFAULT in times and times[RASTER_DEFAULT] <= times[best] * (1.0 + tolerance):
            best = RASTER_DEFAULT
        if not table:
            table.append((0, best))
        elif table[-1][1] != best:
            table.append((n, best))
    return table or [(0, RASTER_DEFAULT)]


def choose_batch(measurements):
    """Measurements [(path, run, ms)] -> (path, run) of the fastest batch launch."""
    path, run, _ = min(measurements, key=lambda m: (m[2], m[0], m[1]))
    return int(path), int(run)


def _time(fn, reps, stream=None):
    import torch
    fn()  # warm-up
    best = None
    for _ in range(reps):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        fn()
        b.record(stream)
        torch.cuda.synchronize()
        t = a.elapsed_time(b)
        best = t if best is None else min(best, t)
    return best


def _order(n, seed):
    buf = cs.allocate(cs.KIND_2D_ORDER, n, path=cs.PATH_POPC)
    cs.sprinkle(cs.KIND_2D_ORDER, n, seed, buf.coords, buf.workspace)
    cs.causal_matrix(cs.KIND_2D_ORDER, n, buf.coords, buf.bits)
    return buf


def measure(sizes=DEFAULT_SIZES, reps=3, seed=0x7E57):
    """Time every count path on a random 2D order of each size."""
    import torch
    out = []
    for n in sizes:
        buf = _order(n, seed)
        times, hists = {}, {}
        for path in PATHS:
            if cs.resolved_path(n, path) != path:
                times[path] = None
                continue
            ws = torch.empty(cs.interval_abundance_workspace(n, path), dtype=torch.uint8, device="cuda")
            hist = torch.empty_like(buf.hist)
            times[path] = _time(lambda: cs.interval_abundance(n, buf.bits, hist, path, ws), reps)
            hists[path] = hist
            del ws
        ref = next(iter(hists.values()))
        if any(not torch.equal(ref, h) for h in hists.values()):
            raise RuntimeError(f"paths disagree at n={n}")
        out.append((n,) + tuple(times[p] for p in PATHS))
    return out


def measure_tiles(sizes=DEFAULT_TILE_SIZES, rasters=DEFAULT_RASTERS, reps=3, seed=0x7E58):
    """Time the single-set count on the path AUTO picks, for each raster side."""
    import torch
    old = cs.get_auto_tiles()
    out = []
    try:
        for n in sizes:
            path = cs.resolved_path(n, cs.PATH_AUTO)
            if path not in (cs.PATH_MMA, cs.PATH_MMA4):
                continue
            buf = _order(n, seed)
            ws = torch.empty(cs.interval_abundance_workspace(n, path), dtype=torch.uint8, device="cuda")
            times, ref = {}, None
            for r in rasters:
                cs.set_auto_tiles([(0, r)])
                hist = torch.empty_like(buf.hist)
                times[r] = _time(lambda: cs.interval_abundance(n, buf.bits, hist, path, ws), reps)
                if ref is None:
                    ref = hist
                elif not torch.equal(ref, hist):
                    raise RuntimeError(f"raster {r} changes the counts at n={n}")
            out.append((n, times))
            del ws, buf
    finally:
        cs.set_auto_tiles(old)
    return out


def measure_batch(n2d=64, n4d=32, runs=DEFAULT_RUNS, reps=3):
    """Time one batch launch of an ensemble sample on each tensor path and run length."""
    import torch
    from paper_1805_04463_gb300 import workloads
    sets = workloads.ensemble(n2d=n2d, n4d=n4d)
    old = cs.get_batch_tuning()
    out, ref = [], None
    try:
        for path in (cs.PATH_MMA, cs.PATH_MMA4):
            b = cs.Batch(sets, path=path, n_eps=1)
            for run in runs:
                cs.set_batch_tuning(old[0], run)
                out.append((path, run, _time(lambda: b.launch((0.0,)), reps)))
                if ref is None:
                    ref = b.hist.clone()
                elif not torch.equal(ref, b.hist):
                    raise RuntimeError(f"batch path {path}, run {run} changes the counts")
            del b
    finally:
        cs.set_batch_tuning(*old)
    return out


def device_key():
    import torch
    p = torch.cuda.get_device_properties(torch.cuda.current_device())
    return f"{p.name} sm_{p.major}{p.minor} x{p.multi_processor_count}"


def save(result, path=DEFAULT_FILE):
    os.makedirs(os.path.dirname(path), exist_ok=True)
    data = {}
    if os.path.exists(path):
        with open(path) as f:
            data = json.load(f)
    data[device_key()] = result
    with open(path, "w") as f:
        json.dump(data, f, indent=1)


def install(result):
    cs.set_auto_paths([tuple(x) for x in result["paths"]])
    if result.get("tiles"):
        cs.set_auto_tiles([tuple(x) for x in result["tiles"]])
    if result.get("batch"):
        cs.set_batch_tuning(*result["batch"])


def load(path=DEFAULT_FILE):
    """Install the saved choices for this device; returns them, or None if there are none."""
    if not os.path.exists(path):
        return None
    with open(path) as f:
        entry = json.load(f).get(device_key())
    if not entry:
        return None
    # JSON keeps lists; the choices are (n_min, value) pairs and a (path, run) pair
    entry["paths"] = [tuple(x) for x in entry["paths"]]
    entry["tiles"] = [tuple(x) for x in entry.get("tiles") or []]
    if entry.get("batch"):
        entry["batch"] = tuple(entry["batch"])
    install(entry)
    return entry


def autotune(sizes=DEFAULT_SIZES, tile_sizes=DEFAULT_TILE_SIZES, rasters=DEFAULT_RASTERS, runs=DEFAULT_RUNS,
             batch_sample=(64, 32), install_=True, persist=True, path=DEFAULT_FILE):
    """Measure the three choices (paths, then tiles under the new path table,
    then the multi-set tuning), install and persist them; returns the result."""
    old_paths = cs.get_auto_paths()
    m = measure(sizes)
    paths = choose(m)
    cs.set_auto_paths(paths)
    try:
        tm = measure_tiles(tile_sizes, rasters)
        bm = measure_batch(*batch_sample, runs=runs)
    finally:
        if not install_:
            cs.set_auto_paths(old_paths)
    result = {"paths": paths, "measurements": m,
              "tiles": choose_tiles(tm), "tile_measurements": [(n, {str(r): t for r, t in ts.items()}) for n, ts in tm],
              "batch": choose_batch(bm), "batch_measurements": bm}
    if install_:
        install(result)
    if persist:
        save(result, path)
    return result


if __name__ == "__main__":
    r = autotune()
    for n, *ts in r["measurements"]:
        print(f"n={n:7d}  " + "  ".join(f"{name} {t if t is None else round(t, 3)} ms"
                                        for name, t in zip(("popc", "mma", "mma4"), ts)))
    print("AUTO table:", r["paths"])
    print("tiles:", r["tiles"], r["tile_measurements"])
    print("batch (path, run):", r["batch"], r["batch_measurements"])
