"""Autotuner of the eigen-solver's schedule for a workload's block shapes.

The truncated SVD of every block (Section 2, Eq. 1) is found by Chebyshev-
filtered subspace iteration. Three knobs trade work for speed and are not
fixed by the method: the subspace width b (k plus an oversample, rounded to
the 16, 32 or 64 columns the kernels are built for), the largest filter
degree (panel products between Rayleigh-Ritz steps), and how the loop is
driven (from the host, one step at a time, or as one CUDA graph whose loop
the device ends; the graph's conditional nodes cost a few microseconds a
step, which small workloads notice). Which setting is fastest depends on
the blocks' spectra and sizes, that is, on the data, so it is measured:
each candidate factorises the workload through the library (after one
untimed call, which also lets the graph form capture its graph), and the
fastest one whose held-out RMSE stays within RMSE_SLACK of the default's
and whose blocks all converge wins.

Results are cached per workload signature: the blocks' (shorter side,
longer side) pairs binned by powers of two, k and the precision, so a
workload of the same block-shape mix reuses the choice. The cache is a JSON
file (``BSVD_TUNE_CACHE``, else ``bsvd_autotune.json`` in the system's
temporary directory).
"""
from __future__ import annotations

import hashlib
import itertools
import json
import math
import os
import tempfile
import time

import numpy as np

# allowed difference in held-out RMSE from the default schedule's
RMSE_SLACK = 1e-5
DEGREES = (4, 6, 8, 10, 12)
OVERSAMPLES = (0, 8, 24, 48)


def _width(k: int, oversample: int) -> int:
    extra = oversample if oversample > 0 else max(8, k // 2)
    want = k + extra
    return 16 if want <= 16 else (32 if want <= 32 else 64)


LOOPS = (0, 1)       # bsvd_config.loop: graph from the second call, host


def candidates(k: int):
    """(oversample, cheb_degree, loop) settings, one per distinct subspace
    width and degree, with each loop form."""
    seen, out = set(), []
    for ov, deg, loop in itertools.product(OVERSAMPLES, DEGREES, LOOPS):
        b = _width(k, ov)
        if k + (ov if ov > 0 else 0) > 64 or (b, deg, loop) in seen:
            continue
        seen.add((b, deg, loop))
        out.append({"oversample": ov, "cheb_degree": deg, "loop": loop})
    return out


def signature(shapes, k: int, precision: int) -> str:
    """Key of a workload: its block shapes binned by powers of two."""
    bins = sorted((int(math.log2(max(s, 1))), int(math.log2(max(L, 1))))
                  for (s, L) in shapes)
    h = hashlib.sha256(json.dumps([bins, k, precision]).encode())
    return h.hexdigest()[:24]


def cache_path() -> str:
    return os.environ.get("BSVD_TUNE_CACHE") or os.path.join(
        tempfile.gettempdir(), "bsvd_autotune.json")


def _load(path):
    try:
        with open(path) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def tune(m, n, p, q, k, u, i, x, ut, it, yt, shapes, precision=0,
         grid=None, trials=2, stream=None, use_cache=True, **cfg):
    """Pick (oversample, cheb_degree, loop) for this workload.

    u, i, x: training ratings; ut, it, yt: held-out ratings (host or
    device); shapes: (s, L) per block; grid: partition keyword arguments
    (bounds and permutations) or None. Returns a dict with the chosen
    parameters, the time per factorisation of each candidate, and whether
    the result came from the cache."""
    import paper_1907_07410_gb300 as bs
    key = signature(shapes, k, precision)
    path = cache_path()
    if use_cache:
        hit = _load(path).get(key)
        if hit is not None:
            return dict(hit, cached=True)
    grid = grid or {}
    results = []
    for cand in [{}] + candidates(k):
        ctx = bs.Context(stream=stream, precision=precision, **cfg, **cand)
        try:
            times, st, rmse = [], bs.OK, None
            for rep in range(trials + 1):
                ctx.partition(m, n, u, i, x, p, q, **grid)
                t0 = time.perf_counter()
                st = ctx.factor(k, warn=False)
                rmse = ctx.rmse(ut, it, yt)       # synchronises the stream
                if rep > 0:                       # the first call is untimed
                    times.append(time.perf_counter() - t0)
            results.append(dict(params=cand, seconds=float(np.median(times)),
                                status=int(st), rmse=float(rmse)))
        finally:
            ctx.close()
    base = results[0]
    ok = [r for r in results
          if r["status"] == bs.OK and abs(r["rmse"] - base["rmse"]) <= RMSE_SLACK]
    best = min(ok, key=lambda r: r["seconds"]) if ok else base
    out = {"key": key, "params": best["params"], "seconds": best["seconds"],
           "default_seconds": base["seconds"],
           "trials": [{"params": r["params"], "seconds": r["seconds"],
                       "status": r["status"], "rmse": r["rmse"]}
                      for r in results]}
    if use_cache:
        db = _load(path)
        db[key] = out
        try:
            tmp = path + ".tmp%d" % os.getpid()
            with open(tmp, "w") as f:
                json.dump(db, f, indent=1)
            os.replace(tmp, path)
        except OSError:
            pass
    return dict(out, cached=False)
