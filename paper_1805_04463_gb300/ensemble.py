"""Ensemble driver with checkpoint / resume.

Evaluates many causal sets (kind, n, seed) -- the averages over sprinklings
that the thesis's experiments report (Section "Convergence and Running
Times") -- and appends one JSON line per finished set to a results file.  A
restarted run reads the file first and evaluates only the sets not yet
recorded, so an interrupted job loses at most the batch in flight; results
are deterministic from (kind, n, seed), so a re-run set gives the same
record.  A last line torn by a crash is ignored.

Small sets (n <= CS_BATCH_MAX_N) go through one batched launch per chunk
(`cs.Batch`), larger ones through the single-set entry points.

    python -m paper_1805_04463_gb300.ensemble --kind 2d_ds_slab --n 65536 \\
        --graphs 40 --eps 0.015625 --out ds_65536.jsonl
"""
from __future__ import annotations

import argparse
import json
import os

HIST_HEAD = 64  # abundances kept per record (k < 64); the pair count keeps the total


def key(kind, n, seed):
    return (int(kind), int(n), int(seed))


def load_done(path):
    """Records already in the results file, by (kind, n, seed); unreadable lines are skipped."""
    done = {}
    if not os.path.exists(path):
        return done
    with open(path) as f:
        for line in f:
            try:
                r = json.loads(line)
                done[key(r["kind"], r["n"], r["seed"])] = r
            except (ValueError, KeyError, TypeError):
                continue  # a line torn by an interrupted write
    return done


def _end_line(path):
    """Terminate a line torn by an interrupted write, so new records start clean."""
    if os.path.exists(path) and os.path.getsize(path) > 0:
        with open(path, "rb") as f:
            f.seek(-1, os.SEEK_END)
            last = f.read(1)
        if last != b"\n":
            with open(path, "a") as f:
                f.write("\n")


def record(kind, n, seed, hist, actions, bracket, eps):
    hist = [int(x) for x in hist]
    return {"kind": int(kind), "n": int(n), "seed": int(seed), "pairs": int(sum(hist)),
            "hist_head": hist[:HIST_HEAD], "bracket": int(bracket),
            "actions": {repr(float(e)): float(a) for e, a in zip(eps, actions)}}


def gpu_runner(path=0):
    """Runner evaluating a chunk of sets on the GPU: batched when every set fits a batch."""
    import paper_1805_04463_gb300 as cs

    def run(chunk, eps):
        import torch
        if all(n <= cs.BATCH_MAX_N for _, n, _ in chunk):
            b = cs.Batch(list(chunk), path=path, n_eps=len(eps))
            b.launch(tuple(eps))
            torch.cuda.synchronize()
            st = b.status()
            if st != 0:
                raise cs.CsError(st, "ensemble batch")
            acts = b.actions.cpu().numpy()
            brs = b.brackets.cpu().numpy()
            out = []
            for s, (kind, n, seed) in enumerate(chunk):
                h = b.set_hist(s).cpu().numpy()
                out.append((h, acts[s, :len(eps)].tolist(), int(brs[s])))
            return out
        out = []
        for kind, n, seed in chunk:
            buf = cs.allocate(kind, n, path=path)
            cs.run(buf, seed, eps=tuple(eps))
            torch.cuda.synchronize()
            st = cs.workspace_status(buf.workspace)
            if st != 0:
                raise cs.CsError(st, "ensemble set")
            out.append((buf.hist.cpu().numpy(), buf.actions.cpu().numpy()[:len(eps)].tolist(),
                        int(buf.bracket.item())))
        return out
    return run


def run(sets, out_path, eps=(0.0,), chunk=256, runner=None):
    """Evaluate `sets` (an iterable of (kind, n, seed)), resuming from out_path.
    Returns the records of all sets, in the order given."""
    sets = [key(*s) for s in sets]
    done = load_done(out_path)
    _end_line(out_path)
    todo = [s for s in sets if s not in done]
    runner = runner or gpu_runner()
    for lo in range(0, len(todo), chunk):
        part = todo[lo:lo + chunk]
        results = runner(part, list(eps))
        with open(out_path, "a") as f:
            for s, (hist, acts, br) in zip(part, results):
                r = record(*s, hist, acts, br, eps)
                done[s] = r
                f.write(json.dumps(r) + "\n")
            f.flush()
            os.fsync(f.fileno())
    return [done[s] for s in sets]


def main(argv=None):
    import paper_1805_04463_gb300 as cs
    ap = argparse.ArgumentParser(description=__doc__.splitlines()[0])
    ap.add_argument("--kind", default="2d_order", choices=sorted(cs.KIND_NAMES.values()))
    ap.add_argument("--n", type=int, required=True)
    ap.add_argument("--graphs", type=int, default=10)
    ap.add_argument("--seed", type=int, default=0xD5000000)
    ap.add_argument("--eps", type=float, nargs="+", default=[0.0])
    ap.add_argument("--chunk", type=int, default=256)
    ap.add_argument("--out", required=True)
    a = ap.parse_args(argv)
    kind = {v: k for k, v in cs.KIND_NAMES.items()}[a.kind]
    recs = run([(kind, a.n, a.seed + g) for g in range(a.graphs)], a.out, a.eps, a.chunk)
    for e in a.eps:
        vals = [r["actions"][repr(float(e))] for r in recs]
        mean = sum(vals) / len(vals)
        sd = (sum((v - mean) ** 2 for v in vals) / max(len(vals) - 1, 1)) ** 0.5
        print(json.dumps({"eps": e, "graphs": len(vals), "mean_action": mean, "sd": sd,
                          "se": sd / max(len(vals), 1) ** 0.5}))


if __name__ == "__main__":
    main()
