"""Benchmark: interval-count throughput of the GB300 causal-set path.

One step = one pass of the whole hot path over one causal set, all on the
device: sprinkle -> causal matrix -> interval abundances -> BD actions
(local + smeared at eps = 0.05, 0.1, 0.2).  The default workload is the
large random 2D order, N = 131072 (2.1 GB bitset, larger than L2).

Prints one JSON line (rank 0).  value = related pairs counted per second
(Gpairs/s) over the whole job; e2e = the same metric through the host-buffer
entry point cs_evaluate (coordinates copied from pinned host memory, the
histogram and actions copied back, every step); roofline = the count
kernel's achieved rate against the POPC (or tensor) peak; cpu_baseline = the
CPU oracle on a bounded sample of the same workload.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--workload NAME] [--path auto|popc|mma|mma4]
  python bench.py --impl reference ...   # the CPU oracle as the reference arm
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOADS = {
    # name: (kind, n, seed, description)
    "2d_order_131072": (0, 131072, 0xC5E70003, "random 2D order, N=131072 (2.1 GB bitset)"),
    "4d_diamond_16384": (2, 16384, 0xC5E70002, "4D Minkowski diamond, N=16384, int32 grid 2^20"),
    "2d_order_1024": (0, 1024, 0xC5E70001, "random 2D order, N=1024"),
    # a mid-size order for profiling captures (operands 1 GB in FP4, above L2)
    "2d_order_32768": (0, 32768, 0xC5E70009, "random 2D order, N=32768"),
}
EPS = (0.0, 0.05, 0.1, 0.2)
PATHS = {"auto": 0, "popc": 1, "mma": 2, "mma4": 3}
PATH_NAMES = {1: "popc", 2: "mma", 3: "mma4"}
POPC_PER_SM_PER_CLK = 16  # 32-bit population count, per SM per clock


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except OSError:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0,
                "sm_max_mhz": 2070.0}, "fallback"


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


class ClockSampler:
    """nvidia-smi clock/throttle samples during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def __enter__(self):
        fd, self.path = tempfile.mkstemp(prefix="clocks_", suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + self.Q, "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        try:
            for line in open(self.path):
                f = [x.strip() for x in line.split(",")]
                if len(f) < 9:
                    continue
                try:
                    sm.append(float(f[1]))
                    mx.append(float(f[2]))
                except ValueError:
                    continue
                for nm, v in zip(names, f[5:9]):
                    if v.lower() == "active":
                        reasons.add(nm)
        except OSError:
            pass
        finally:
            try:
                os.unlink(self.path)
            except OSError:
                pass
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def roofline_for(resolved, n, count_s, peaks, src, sm_count):
    """Achieved vs peak for the count call (algorithmic work: every pair i<j over the
    columns strictly between them, C(n,3) bit-AND/popcount terms = MACs).

    The tensor paths' peak is the measured bf16 BURST figure times the nominal
    ratio of the path's operand type to bf16: the count is a ~0.1 s kernel
    timed on its own stream, which runs at the full SM clock without a power
    cap (the clocks record of the run shows it), not a seconds-long loop.  The
    fraction of the sustained-derived peak is reported beside it."""
    terms = n * (n - 1) * (n - 2) / 6.0
    if resolved in (2, 3):
        ratio, kind, kern = ((6.0, "FP4 kind::mxf4", "k_count_mma4 (+ k_expand_f4)") if resolved == 3 else
                             (2.0, "FP8 kind::f8f6f4", "k_count_mma (+ k_expand_f8)"))
        burst = peaks.get("bf16_tflops")
        sustained = peaks.get("bf16_tflops_sustained", burst)
        peak = ratio * burst
        achieved = 2.0 * terms / count_s / 1e12
        return {"bound": "tensor", "kernel": kern, "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                "frac": achieved / peak, "frac_burst": achieved / peak,
                "frac_sustained": achieved / (ratio * sustained), "peak_sustained": ratio * sustained,
                "traffic": None, "algorithmic_macs": terms,
                "peak_source": f"{ratio:g} x bf16_tflops (burst, {src}; nominal {kind}/BF16 ratio); "
                               f"2 FLOP per MAC"}
    peak = sm_count * POPC_PER_SM_PER_CLK * peaks.get("sm_max_mhz", 2070.0) * 1e6 / 1e12  # T popc32/s
    achieved = terms / 32.0 / count_s / 1e12
    return {"bound": "alu", "kernel": "k_count_popc", "achieved": achieved, "peak": peak, "unit": "T popc32/s",
            "frac": achieved / peak, "traffic": None, "algorithmic_bit_ands": terms,
            "peak_source": f"{sm_count} SMs x {POPC_PER_SM_PER_CLK} POPC/clk x {peaks.get('sm_max_mhz')} MHz "
                           f"(sm_max_mhz, {src})"}


TRAFFIC_RECORDS = {2: "k_count_mma__2d_order_131072__dram.md", 3: "k_count_mma4__2d_order_131072__dram.md"}
MMA_SOURCES = [os.path.join(ROOT, "paper_1805_04463_gb300", "csrc", f)
               for f in ("cs_count_mma.cu", "cs_internal.cuh", "cs_kernels.cuh")]


def recorded_traffic(resolved):
    """DRAM bytes per full-size count launch (k_count_mma or k_count_mma4) from the
    committed ncu record, or None when the kernel sources changed since it was captured."""
    import hashlib
    try:
        path = os.path.join(ROOT, "profiles", TRAFFIC_RECORDS[resolved])
        rec = dict(line.split(":", 1) for line in open(path) if line.startswith(("traffic_", "kernel_")))
        h = hashlib.sha256(b"".join(open(f, "rb").read() for f in MMA_SOURCES)).hexdigest()[:16]
    except (OSError, ValueError, KeyError):
        return None
    if rec.get("kernel_sources_sha256_16", "").strip() != h:
        return None
    return float(rec["traffic_bytes_per_launch"])


def compare_paths(cs, torch, buf, n, stream):
    """Count-call time of each path on the same bitset (1 warm-up + 1 timed, CUDA events)."""
    out = {}
    for name, p in (("popc", 1), ("mma", 2), ("mma4", 3)):
        ws = torch.empty(cs.interval_abundance_workspace(n, p), dtype=torch.uint8, device="cuda")
        hist = torch.empty_like(buf.hist)
        cs.interval_abundance(n, buf.bits, hist, p, ws, stream)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        cs.interval_abundance(n, buf.bits, hist, p, ws, stream)
        b.record(stream)
        torch.cuda.synchronize()
        if not torch.equal(hist, buf.hist):
            raise RuntimeError(f"path {name} disagrees with the timed path")
        out[name] = a.elapsed_time(b)
        del ws
    return out


def ensemble_bench(cs, torch, path, steps=5, warmup=3, n2d=512, n4d=256):
    """Batched ensemble (one CUDA-graph replay of cs_batch_launch per step) vs the
    same sets as one-at-a-time plain launches, on this GPU."""
    from paper_1805_04463_gb300 import workloads
    sets = workloads.ensemble(n2d=n2d, n4d=n4d)
    stream = torch.cuda.Stream()
    b = cs.Batch(sets, path=path, n_eps=len(EPS))
    with torch.cuda.stream(stream):
        b.launch(EPS, stream=stream)
        stream.synchronize()
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g, stream=stream):
            b.launch(EPS, stream=stream)
        for _ in range(warmup):
            g.replay()
        a, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        for _ in range(steps):
            g.replay()
        e.record(stream)
    torch.cuda.synchronize()
    batched_ms = a.elapsed_time(e) / steps
    if b.status() != 0:
        raise cs.CsError(b.status(), "ensemble")
    pairs = int(b.hist.sum().item())
    # one-at-a-time: the same sets through the single-set entry points
    bufs = [cs.allocate(k, n, path=b.path) for k, n, _ in sets]
    def plain():
        for (k, n, sd), buf in zip(sets, bufs):
            cs.run(buf, sd, eps=EPS, stream=stream)
    with torch.cuda.stream(stream):
        plain()
        stream.synchronize()
        a2, e2 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a2.record(stream)
        plain()
        e2.record(stream)
    torch.cuda.synchronize()
    plain_ms = a2.elapsed_time(e2)
    same = all(torch.equal(buf.hist, b.set_hist(s)) for s, buf in enumerate(bufs))
    terms = sum(n * (n - 1) * (n - 2) / 6.0 for _, n, _ in sets)
    return {"workload": f"{n2d} 2D diamonds N~Poisson(4096) + {n4d} 4D diamonds N~Poisson(2048)",
            "sets": len(sets), "pairs": pairs, "path": PATH_NAMES[b.path],
            "batched_graph_ms": batched_ms, "plain_ms": plain_ms,
            "batched_gpairs_s": pairs / batched_ms / 1e6, "plain_gpairs_s": pairs / plain_ms / 1e6,
            "batched_actions_s": len(sets) / batched_ms * 1e3, "plain_actions_s": len(sets) / plain_ms * 1e3,
            "speedup": plain_ms / batched_ms, "identical_results": bool(same),
            "algorithmic_macs": terms, "achieved_tflops_whole_step": 2 * terms / batched_ms / 1e9}


def extras_bench(cs, torch, buf, kind, n, path, stream, peaks):
    """The next-row outputs on the bench set, each timed with CUDA events on the
    launching stream after a warm-up: degree vectors and the future sparse
    relation list (HBM-bound row scans: roofline against the copy bandwidth),
    and the d'Alembertian layer sums (the count with the per-element epilogue)."""
    def timed(fn, reps=3):
        fn()
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        for _ in range(reps):
            fn()
        b.record(stream)
        torch.cuda.synchronize()
        return a.elapsed_time(b) / reps
    out = {}
    L = cs.lib()
    words = (n + 63) // 64
    kin = torch.empty(n, dtype=torch.int32, device="cuda")
    kout = torch.empty(n, dtype=torch.int32, device="cuda")
    deg_ms = timed(lambda: cs.degrees(n, buf.bits, kin, kout, stream))
    deg_bytes = n * words * 8 + 8 * n
    ws = torch.empty(L.cs_sparse_workspace_bytes(n), dtype=torch.uint8, device="cuda")
    off = torch.empty(n + 1, dtype=torch.int64, device="cuda")
    L.cs_sparse_offsets(n, buf.bits.data_ptr(), buf.rw, 1, off.data_ptr(), ws.data_ptr(), ws.numel(), stream.cuda_stream)
    total = int(off[n].item())
    cols = torch.empty(max(total, 1), dtype=torch.int32, device="cuda")

    def csr():
        L.cs_sparse_offsets(n, buf.bits.data_ptr(), buf.rw, 1, off.data_ptr(), ws.data_ptr(), ws.numel(),
                            stream.cuda_stream)
        L.cs_sparse_columns(n, buf.bits.data_ptr(), buf.rw, 1, off.data_ptr(), cols.data_ptr(), total,
                            ws.data_ptr(), ws.numel(), stream.cuda_stream)
    csr_ms = timed(csr)
    if cs.workspace_status(ws) != 0 or int(kout.sum().item()) != total:
        raise RuntimeError("sparse lists disagree with the degrees")
    csr_bytes = n * words * 4 + 4 * total + 8 * (n + 1)  # upper half of the bitset read once, lists written
    hbm = peaks.get("hbm_gbs")
    out["sparse"] = {
        "degrees_ms": deg_ms, "degrees_gbs": deg_bytes / deg_ms / 1e6,
        "future_csr_ms": csr_ms, "future_relations": total, "future_csr_gbs": csr_bytes / csr_ms / 1e6,
        "roofline": {"bound": "hbm", "peak": hbm, "unit": "GB/s",
                     "frac_degrees": deg_bytes / deg_ms / 1e6 / hbm if hbm else None,
                     "frac_future_csr": csr_bytes / csr_ms / 1e6 / hbm if hbm else None,
                     "bytes": {"degrees": deg_bytes, "future_csr": csr_bytes}},
    }
    del cols
    # d'Alembertian layer sums (phi = 1, kmax = 3) against the plain count
    layer = torch.empty((4, n), dtype=torch.float64, device="cuda")
    lay_ms = timed(lambda: cs.layer_sums(n, buf.bits, buf.hist, layer, 3, None, path, buf.workspace, stream), reps=1)
    cnt_ms = timed(lambda: cs.interval_abundance(n, buf.bits, buf.hist, path, buf.workspace, stream), reps=1)
    out["dalembertian"] = {"layer_sums_ms": lay_ms, "count_only_ms": cnt_ms, "overhead": lay_ms / cnt_ms - 1.0,
                           "kmax": 3}
    # chains and antichains (synchronous entry points: wall time around the call)
    def wall(fn):
        fn()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        r = fn()
        return r, (time.perf_counter() - t0) * 1e3
    height, h_ms = wall(lambda: cs.longest_chain(n, buf.bits))
    (asize, _), a_ms = wall(lambda: cs.greedy_antichain(n, buf.bits, n // 2))
    out["chains"] = {"height": height, "height_ms": h_ms, "antichain_seed": n // 2, "antichain_size": asize,
                     "antichain_ms": a_ms}
    return out


def serving_bench(path, rate=200.0, duration_s=5.0):
    """The continuous-batching server on a Poisson trace (real time): throughput
    and latency percentiles under a 60 GB bitset budget."""
    from paper_1805_04463_gb300 import serve, workloads
    srv = serve.Server(path=path)
    srv.run(workloads.serving_requests(rate=rate, duration_s=0.1, seed=workloads.SEED_BASE + 55))  # warm-up
    reqs = workloads.serving_requests(rate=rate, duration_s=duration_s)
    stats, _ = srv.run(reqs)
    total_macs = sum(n * (n - 1) * (n - 2) / 6.0 for _, _, n, _ in reqs)
    offered = total_macs / duration_s
    # every request is served (the server queues what its budgets cannot
    # hold yet), so the admitted load is the work over the run's wall time
    # (arrivals and drain included, at least the trace's duration)
    served = (total_macs / max(stats["wall_s"], duration_s)) if stats.get("requests") == len(reqs) else None
    stats.update({"workload": f"Poisson arrivals {rate:g}/s for {duration_s:g} s, N = floor(2^U[10,16]), "
                              "50/50 2D order / 4D diamond, 60 GB bitset budget",
                  "offered_requests": len(reqs), "offered_macs_per_s": offered, "served_macs_per_s": served,
                  "admitted_load_fraction": None if served is None else served / offered})
    return stats


PROBE_REPS = {1: 1 << 16, 2: 1 << 16, 3: 1 << 16}
PROBE_WHAT = {1: "independent popc.b32 chains in registers, all SMs",
              2: "back-to-back tcgen05.mma kind::f8f6f4 M128 N256 K32, operands in shared memory, one CTA per SM",
              3: "back-to-back tcgen05.mma cta_group::2 kind::mxf4 M256 N256 K64, operands in shared memory, "
                 "CTA pairs on all SMs"}


def batch_path(name):
    """The path the batch and serving entry points take for --path (their own
    AUTO choice for --path auto)."""
    return PATHS[name]


def launches_per_step(kind, path):
    """Kernels of this library launched by one step: sprinkle (keys, 4 bucket-rank
    kernels per key stream, scatter), relate (upper part, mirror), count
    (operand expansion first on the tensor paths) and actions (partial, final)."""
    sprinkle = 1 + (2 if kind == 0 else 1) * 4 + 1
    count = 1 if path == 1 else 2
    return sprinkle + 2 + count + 2


def cpu_baseline(kind, n, seed, target_s=15.0, max_rows=None):
    """The oracle on a bounded sample of rows of the same workload (pairs/s)."""
    import numpy as np
    import oracle
    coords = oracle.sprinkle(kind, n, seed)
    bits = oracle.causal_matrix(kind, coords)
    # calibrate on a short sample, then size the sample to ~target_s seconds
    step = max(1, n // 64)
    t0 = time.perf_counter()
    h, threads = oracle.interval_abundance_threads(bits, rows=(0, n, step))
    dt = max(time.perf_counter() - t0, 1e-3)
    rows_done = len(range(0, n, step))
    rows_wanted = int(rows_done * target_s / dt)
    if max_rows:
        rows_wanted = min(rows_wanted, max_rows)
    step = max(1, n // max(rows_wanted, 1))
    t0 = time.perf_counter()
    h, threads = oracle.interval_abundance_threads(bits, rows=(0, n, step))
    dt = time.perf_counter() - t0
    pairs = int(np.asarray(h).sum())
    # one thread on a sample of the same rows sized to about half the time
    step1 = max(1, int(step * max(1.0, 2.0 * threads)))
    t0 = time.perf_counter()
    h1, _ = oracle.interval_abundance_threads(bits, threads=1, rows=(0, n, step1))
    dt1 = max(time.perf_counter() - t0, 1e-9)
    pairs1 = int(np.asarray(h1).sum())
    return {"value": pairs / dt / 1e9, "unit": "Gpairs/s", "cores": threads, "kind": "oracle",
            "sample": f"rows i = 0, {step}, {2 * step}, ... of the same set ({len(range(0, n, step))} of {n} rows, "
                      f"{pairs} related pairs, {dt:.1f} s)", "seconds": dt, "pairs": pairs,
            "single_thread": {"value": pairs1 / dt1 / 1e9, "unit": "Gpairs/s",
                              "sample": f"every {step1}th row ({pairs1} related pairs, {dt1:.1f} s)"}}


def run_reference(args):
    ws, rank, _ = _dist()
    kind, n, seed, desc = WORKLOADS[args.workload]
    if rank != 0:
        return 0
    # Each step = one bounded sample of the workload, timed on the host cores.
    import numpy as np
    import oracle
    coords = oracle.sprinkle(kind, n, seed)
    bits = oracle.causal_matrix(kind, coords)
    step = max(1, n // 256) if n > 4096 else 1
    rows = (0, n, step)
    for _ in range(args.warmup):
        oracle.interval_abundance(bits, rows=rows)
    times, pairs, threads = [], 0, 0
    for _ in range(args.steps):
        t0 = time.perf_counter()
        h, threads = oracle.interval_abundance_threads(bits, rows=rows)
        times.append(time.perf_counter() - t0)
        pairs = int(np.asarray(h).sum())
    total = sum(times)
    value = pairs * args.steps / total / 1e9
    sample = f"rows i = 0, {step}, ... ({len(range(*rows))} of {n} rows, {pairs} related pairs per step)"
    line = {
        "impl": "reference", "metric": f"interval-count Gpairs/s ({desc})", "value": value, "unit": "Gpairs/s",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000 * total / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u64", "data": "synthetic",
        "config": {"workload": args.workload, "kind": ["2d_order", "2d_diamond", "4d_diamond", "3d_diamond", "2d_ds_slab"][kind], "n": n,
                   "seed": seed, "path": "cpu oracle", "eps": list(EPS),
                   "l2": "inputs larger than L2" if n * ((n + 63) // 64) * 8 > 129e6 else "inputs smaller than L2",
                   "parallelism": "replicas1"},
        "cpu_baseline": {"value": value, "unit": "Gpairs/s", "cores": threads, "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": "Gpairs/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="2d_order_131072", choices=sorted(WORKLOADS))
    ap.add_argument("--path", default="auto", choices=sorted(PATHS))
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--e2e-steps", type=int, default=None)
    ap.add_argument("--compare-paths", action="store_true",
                    help="also time the other count path once on the same bitset")
    ap.add_argument("--no-ensemble", action="store_true", help="skip the batched-ensemble measurement")
    ap.add_argument("--no-serve", action="store_true", help="skip the serving-loop measurement")
    ap.add_argument("--no-extras", action="store_true",
                    help="skip the degree / sparse-list / d'Alembertian measurements")
    ap.add_argument("--no-tune", action="store_true",
                    help="skip the autotuner and keep the library's built-in path, tile and batch choices")
    ap.add_argument("--ensemble-sets", default="512,256",
                    help="ensemble size: number of 2D diamonds, number of 4D diamonds (profiling runs use a sample)")
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)

    import numpy as np
    import torch

    import paper_1805_04463_gb300 as cs
    from paper_1805_04463_gb300 import build as csbuild
    from paper_1805_04463_gb300 import replicas

    ws, rank, local = _dist()
    torch.cuda.set_device(local)
    dist = None
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    csbuild.build()
    tuning = None
    if not args.no_tune:
        # measured path table, raster sides and multi-set tuning on this GPU,
        # installed before anything is timed (not persisted)
        from paper_1805_04463_gb300 import tune
        r = tune.autotune(persist=False)
        tuning = {"paths": r["paths"], "tiles": r["tiles"], "batch_path_run": r["batch"],
                  "tile_measurements_ms": r["tile_measurements"],
                  "batch_measurements_ms": r["batch_measurements"]}
    kind, n, seed0, desc = WORKLOADS[args.workload]
    seed = seed0 + rank  # weak scaling: one independent set per rank
    path = PATHS[args.path]
    buf = cs.allocate(kind, n, path=path)
    stream = torch.cuda.current_stream()

    # count-kernel timing: events on the launching stream around each count call
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]

    def step(i=None):
        cs.sprinkle(kind, n, seed, buf.coords, buf.workspace, stream)
        cs.causal_matrix(kind, n, buf.coords, buf.bits, stream)
        if i is not None:
            ev[i][0].record(stream)
        cs.interval_abundance(n, buf.bits, buf.hist, path, buf.workspace, stream)
        if i is not None:
            ev[i][1].record(stream)
        cs.action_device(cs.dim(kind), n, buf.hist, list(EPS), buf.actions, buf.bracket, buf.workspace, stream)

    for _ in range(max(args.warmup, 0)):
        step()
    torch.cuda.synchronize()
    status = cs.workspace_status(buf.workspace)
    if status != 0:
        raise cs.CsError(status, "warm-up")

    start, stop = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    with ClockSampler(local) as clk:
        start.record(stream)
        for i in range(args.steps):
            step(i)
        stop.record(stream)
        torch.cuda.synchronize()
    if dist:
        dist.barrier()
    elapsed_ms = start.elapsed_time(stop)
    count_ms = [a.elapsed_time(b) for a, b in ev]

    # per-stage times of one more step (events between the stages, outside the timed region)
    se = [torch.cuda.Event(enable_timing=True) for _ in range(5)]
    se[0].record(stream)
    cs.sprinkle(kind, n, seed, buf.coords, buf.workspace, stream)
    se[1].record(stream)
    cs.causal_matrix(kind, n, buf.coords, buf.bits, stream)
    se[2].record(stream)
    cs.interval_abundance(n, buf.bits, buf.hist, path, buf.workspace, stream)
    se[3].record(stream)
    cs.action_device(cs.dim(kind), n, buf.hist, list(EPS), buf.actions, buf.bracket, buf.workspace, stream)
    se[4].record(stream)
    torch.cuda.synchronize()
    stages_ms = {name: se[k].elapsed_time(se[k + 1])
                 for k, name in enumerate(("sprinkle", "relate", "count", "action"))}
    hist = buf.hist.cpu().numpy()
    pairs = int(hist.sum())
    actions = buf.actions.cpu().numpy()[:len(EPS)].tolist()
    elapsed_ms, total_pairs = replicas.combine_timing(elapsed_ms, float(pairs), dist)
    value = total_pairs * args.steps / (elapsed_ms / 1e3) / 1e9

    # e2e through the host-buffer entry point: pinned coordinates in, histogram out
    coords_pinned = torch.empty((cs.dim(kind), n), dtype=torch.int32, pin_memory=True)
    coords_pinned.copy_(buf.coords.cpu())
    cp = coords_pinned.numpy()
    hist_pinned = torch.empty(cs.hist_len(n), dtype=torch.int64, pin_memory=True).numpy()
    e2e_steps = args.e2e_steps if args.e2e_steps is not None else args.steps
    h2, _, _ = cs.evaluate(kind, n, 0, cp, path, EPS, stream=stream, hist_out=hist_pinned)  # warm the pool
    if int(h2.sum()) != pairs:
        raise RuntimeError("host-buffer evaluation disagrees with the device pass")
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        h2, _, _ = cs.evaluate(kind, n, 0, cp, path, EPS, stream=stream, hist_out=hist_pinned)
    e2e_s = max(time.perf_counter() - t0, 1e-9)
    e2e_s, _ = replicas.combine_timing(e2e_s, 0.0, dist)
    e2e_value = total_pairs * e2e_steps / e2e_s / 1e9 if e2e_steps > 0 else None

    if rank != 0:
        if dist:
            dist.destroy_process_group()
        return 0

    peaks, src = _peaks()
    clocks = clk.summary()
    roofline = roofline_for(cs.resolved_path(n, path), n, statistics.mean(count_ms) / 1e3, peaks, src,
                            torch.cuda.get_device_properties(local).multi_processor_count)
    roofline["count_ms"] = statistics.mean(count_ms)
    resolved = cs.resolved_path(n, path)
    if roofline["bound"] == "tensor" and args.workload == "2d_order_131072":
        tr = recorded_traffic(resolved)
        roofline["traffic"] = tr
        roofline["traffic_source"] = (f"profiles/{TRAFFIC_RECORDS[resolved]} (dram__bytes_read.sum + "
                                      "dram__bytes_write.sum, one full-size launch)" if tr else
                                      "no capture for the current kernel sources")
    if args.compare_paths:
        roofline["paths_ms"] = compare_paths(cs, torch, buf, n, stream)
    # context beside the contract's peak: the path's innermost operation timed
    # alone on every SM (cs_peak_probe), and the count's fraction of it
    probe = cs.peak_probe(resolved, PROBE_REPS[resolved]) / 1e12
    roofline["probe"] = {"value": probe, "unit": roofline["unit"], "frac": roofline["achieved"] / probe,
                         "what": PROBE_WHAT[resolved]}
    roofline["frac_probe"] = roofline["achieved"] / probe
    # the clock the count ran at: the time in SM cycles makes runs at
    # different clocks comparable
    roofline["sm_mhz_median"] = clocks.get("sm_mhz")
    if clocks.get("sm_mhz"):
        roofline["count_mcycles"] = roofline["count_ms"] * clocks["sm_mhz"] / 1e3
    line = {
        "metric": f"interval-count Gpairs/s ({desc})", "value": value, "unit": "Gpairs/s", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": elapsed_ms / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        # the count's arithmetic: 0/1 E4M3 (FP8 path) or E2M1 (FP4 path) products summed
        # in FP32 on the tensor paths, AND + popcount on 64-bit words on the POPC path
        "dtype": {1: "u64", 2: "fp8e4m3", 3: "fp4e2m1"}[cs.resolved_path(n, path)], "data": "synthetic",
        "config": {"workload": args.workload, "kind": cs.KIND_NAMES[kind], "n": n, "seed": seed0,
                   "path": args.path, "resolved_path": PATH_NAMES[cs.resolved_path(n, path)],
                   "eps": list(EPS),
                   "l2": "inputs larger than L2" if cs.bitset_bytes(n) > 129e6 else "inputs smaller than L2",
                   "parallelism": f"replicas{args.gpus}"},
        "actions_per_s": args.steps * ws / (elapsed_ms / 1e3),
        "pairs_per_step": pairs, "actions": actions,
        "e2e": {"value": e2e_value, "unit": "Gpairs/s", "h2d_bytes_per_step": int(cp.nbytes),
                "d2h_bytes_per_step": int(hist_pinned.nbytes + 8 * len(EPS) + 8), "steps": e2e_steps},
        "gpu_launches": launches_per_step(kind, cs.resolved_path(n, path)) * args.steps,
        "roofline": roofline,
        "clocks": clocks,
        "stages_ms": stages_ms,
        "tuning": tuning if tuning is not None else {"paths": cs.get_auto_paths(), "tiles": cs.get_auto_tiles(),
                                                    "batch_path_run": list(cs.get_batch_tuning()),
                                                    "source": "built-in (--no-tune)"},
    }
    if not args.no_extras:
        line.update(extras_bench(cs, torch, buf, kind, n, path, stream, peaks))
    if not args.no_ensemble:
        n2d, n4d = (int(x) for x in args.ensemble_sets.split(","))
        line["ensemble"] = ensemble_bench(cs, torch, batch_path(args.path), n2d=n2d, n4d=n4d)
    if not args.no_serve:
        line["serving"] = serving_bench(batch_path(args.path))
    if not args.no_cpu_baseline:
        cb = cpu_baseline(kind, n, seed0)
        line["cpu_baseline"] = {k: cb[k] for k in ("value", "unit", "cores", "kind", "sample", "single_thread")}
    print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
