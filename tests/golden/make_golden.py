"""Write the oracle's results for the medium workloads to JSON fixtures.

Calls only ``oracle`` and the seeded generator ``synth``: no stored value
here comes from the CUDA library. Run from the repository root:

    python tests/golden/make_golden.py
"""
from __future__ import annotations

import json
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import numpy as np  # noqa: E402

import oracle  # noqa: E402
import synth  # noqa: E402


def golden(w: synth.Workload) -> dict:
    r = synth.generate(w)
    t0 = time.time()
    part = oracle.partition(w.m, w.n, r.u_train, r.i_train, r.x_train, w.p,
                            w.q)
    model = oracle.factor(part, w.k)
    rmse = oracle.rmse(model, r.u_test, r.i_test, r.x_test)
    yhat = oracle.predict(model, r.u_test, r.i_test)
    out = dict(
        workload=w.name, digest=r.digest(), k=w.k, p=w.p, q=w.q,
        counts=part.counts.tolist(),
        mu64=part.mu64.tolist(),
        sigma=[model.blocks[b].sigma[:w.k + 1].tolist()
               for b in range(w.p * w.q)],
        gap=[model.blocks[b].gap for b in range(w.p * w.q)],
        rmse=rmse,
        yhat_first_1000=yhat[:1000].tolist(),
        oracle_seconds=time.time() - t0,
    )
    return out


def main():
    names = sys.argv[1:] or [synth.MEDIUM.name]
    for name in names:
        w = synth.WORKLOADS[name]
        g = golden(w)
        path = os.path.join(HERE, w.name + ".json")
        with open(path, "w") as f:
            json.dump(g, f, indent=1)
        print(path, "rmse", g["rmse"], "%.1fs" % g["oracle_seconds"])


if __name__ == "__main__":
    main()
