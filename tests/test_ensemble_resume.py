"""Checkpoint / resume of the ensemble driver (host logic, a fake runner):
finished sets are recorded one JSON line each, a restart evaluates only the
rest, a torn last line is ignored, and the records come back in input order."""
import json

import numpy as np
import pytest

from paper_1805_04463_gb300 import ensemble


def _fake_runner(calls, fail_after=None):
    def run(chunk, eps):
        calls.append(list(chunk))
        if fail_after is not None and len(calls) > fail_after:
            raise RuntimeError("interrupted")
        out = []
        for kind, n, seed in chunk:
            h = np.arange(max(n - 1, 1), dtype=np.int64) + seed % 7
            out.append((h, [float(seed) + e for e in eps], kind + n))
        return out
    return run


def test_resume_runs_only_missing_sets(tmp_path):
    out = tmp_path / "res.jsonl"
    sets = [(0, 100 + i, 1000 + i) for i in range(10)]
    calls = []
    with pytest.raises(RuntimeError):
        ensemble.run(sets, str(out), eps=(0.0, 0.1), chunk=3, runner=_fake_runner(calls, fail_after=2))
    assert len(ensemble.load_done(str(out))) == 6          # two chunks landed before the failure
    calls2 = []
    recs = ensemble.run(sets, str(out), eps=(0.0, 0.1), chunk=3, runner=_fake_runner(calls2))
    assert [c for ch in calls2 for c in ch] == [ensemble.key(*s) for s in sets[6:]]
    assert [(r["kind"], r["n"], r["seed"]) for r in recs] == sets
    assert recs[4]["actions"] == {"0.0": 1004.0, "0.1": 1004.1}
    assert recs[4]["pairs"] == int((np.arange(103) + 1004 % 7).sum())
    calls3 = []
    again = ensemble.run(sets, str(out), eps=(0.0, 0.1), chunk=3, runner=_fake_runner(calls3))
    assert not calls3 and again == recs


def test_torn_last_line_is_ignored(tmp_path):
    out = tmp_path / "res.jsonl"
    sets = [(2, 50, 7), (2, 60, 8)]
    ensemble.run(sets[:1], str(out), runner=_fake_runner([]))
    with open(out, "a") as f:
        f.write('{"kind": 2, "n": 60, "se')          # interrupted mid-write
    calls = []
    recs = ensemble.run(sets, str(out), runner=_fake_runner(calls))
    assert calls == [[(2, 60, 8)]]
    assert [r["seed"] for r in recs] == [7, 8]
    lines = [json.loads(x) for x in open(out) if x.strip().endswith("}")]
    assert {r["seed"] for r in lines} == {7, 8}
