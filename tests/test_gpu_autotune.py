"""The project's autotuner of the eigen-solver schedule: it times each
candidate (subspace width, largest filter degree) through the library and
keeps the fastest whose held-out RMSE stays within its slack of the default
schedule's, caching the choice per block-shape signature."""
import json

import numpy as np
import pytest

import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_1907_07410_gb300 as bs  # noqa: E402
from paper_1907_07410_gb300 import autotune  # noqa: E402


def test_autotune_picks_a_valid_schedule_and_caches_it(tmp_path, monkeypatch):
    monkeypatch.setenv("BSVD_TUNE_CACHE", str(tmp_path / "tune.json"))
    w = synth.MEDIUM
    r = synth.generate(w)
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()  # noqa: E731
    br, bc = -(-w.m // w.p), -(-w.n // w.q)
    shapes = []
    for bi in range(w.p):
        for bj in range(w.q):
            mb = min(br, w.m - bi * br)
            nb = min(bc, w.n - bj * bc)
            shapes.append((min(mb, nb), max(mb, nb)))
    args = (w.m, w.n, w.p, w.q, w.k, dev(r.u_train), dev(r.i_train),
            dev(r.x_train), dev(r.u_test), dev(r.i_test), dev(r.x_test),
            shapes)
    first = autotune.tune(*args, trials=1)
    assert not first["cached"]
    cands = [{}] + autotune.candidates(w.k)
    assert first["params"] in cands
    assert len(first["trials"]) == len(cands)
    base = first["trials"][0]["rmse"]
    chosen = next(t for t in first["trials"] if t["params"] == first["params"])
    assert chosen["status"] == bs.OK
    assert abs(chosen["rmse"] - base) <= autotune.RMSE_SLACK
    assert chosen["seconds"] == min(
        t["seconds"] for t in first["trials"]
        if t["status"] == bs.OK and abs(t["rmse"] - base) <= autotune.RMSE_SLACK)
    again = autotune.tune(*args, trials=1)
    assert again["cached"] and again["params"] == first["params"]
    db = json.load(open(tmp_path / "tune.json"))
    assert first["key"] in db
    # a different k is a different workload
    assert autotune.signature(shapes, 10, 0) != first["key"]
