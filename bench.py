"""Benchmark of the block-SVD recommender hot path on GB300.

One step = the whole hot path on one synthetic rating matrix already in
HBM: partition (block ids, exact block means, the dense centred blocks),
Gram products, truncated eigen-solve, projection, held-out prediction and
RMSE. The default workload is the Netflix-prize-shaped matrix (480,189
users x 17,770 items, 100,480,507 ratings, 90/10 split) cut at rating-
activity quantiles into a 32 x 8 grid of uneven blocks, k = 40, with the
BF16 Gram and float32 eigen-solver of the batched form.

The line's value is that fast form. Beside it ("forms") the same workload
runs with the exact tensor-core Gram (float32 result) and on the plain FP32
path (FP32 SIMT Gram, panel products and projection), and the
MovieLens-1M-shaped medium matrix (4 x 4 grid, k = 20) runs as a second
workload ("medium"). Every RMSE is compared with the FP64 oracle's value in
the workload's fixture under tests/golden/.

At N=1 the line also carries the served form ("served"): Poisson streams of
factorise-then-predict requests through the continuous-batching server at
each --serve-rates rate, beside the same requests run one at a time; and
the paper's own blocked SGD ("sgd", Algorithms 1-2): seconds per epoch on
the medium matrix, beside one epoch of the FP64 oracle.

Prints one JSON line (rank 0). Usage:
    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
Under torchrun the ranks share one workload (strong scaling): each holds and
factorises its longest-processing-time share of the blocks, and the step's
held-out RMSE is combined by one all-reduce of (sum of squared errors,
count); the blocks need no other exchange.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import synth  # noqa: E402

FP32_LANES_PER_SM = 128
SMS = 152
PROFILES = os.path.join(ROOT, "profiles")
CSRC = os.path.join(ROOT, "paper_1907_07410_gb300", "csrc")
# kernel -> source file whose contents the ncu traffic figures belong to
KERNEL_SOURCES = {"k_gpanel_tc": "kernels_panel_tc.cu",
                  "k_gram_tc": "kernels_gram_tc.cu",
                  "k_gram_bf16": "kernels_gram_tc.cu",
                  "k_gram_tf32": "kernels_gram_tc.cu",
                  "k_gram_f32": "kernels_gram.cu"}


def profiled_traffic_ratio(kernel):
    """DRAM bytes (read + write) over algorithmic bytes of one launch of
    `kernel`, from the ncu summaries under profiles/, if one was captured
    from the kernel's current source. A summary records it in a line
    ``traffic_ratio: <kernel> <ratio> <sha256 of the source file>``; a
    figure taken from other source is stale and gives None. The captures
    run on a workload small enough for a multi-pass ncu capture; the bench
    scales the ratio by its own launches' algorithmic bytes."""
    src = KERNEL_SOURCES.get(kernel)
    if not src or not os.path.isdir(PROFILES):
        return None
    import hashlib
    with open(os.path.join(CSRC, src), "rb") as f:
        sha = hashlib.sha256(f.read()).hexdigest()
    for name in sorted(os.listdir(PROFILES)):
        with open(os.path.join(PROFILES, name)) as f:
            for line in f:
                parts = line.strip().strip("`").split()
                if (len(parts) == 4 and parts[0] == "traffic_ratio:"
                        and parts[1] == kernel and parts[3] == sha):
                    return float(parts[2])
    return None


def load_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            return json.load(f), "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "sm_max_mhz": 2070.0}, \
        "fallback"


def fp32_alu_peak_tflops(peaks):
    # 152 SMs x 128 FP32 lanes x 2 flops (FMA) x max SM clock
    return SMS * FP32_LANES_PER_SM * 2 * peaks.get("sm_max_mhz", 2070.0) * 1e6 / 1e12


def gram_flops(blocks):
    """Gram work as a general product counts it: 2 m_b n_b s_b flop per
    block (s = min side), both triangles of the symmetric product."""
    return float(sum(2.0 * L * s * s for (s, L) in blocks))


def gram_flops_min(blocks):
    """The Gram's least dense work: its s (s + 1) / 2 distinct entries, 2 L
    flop each (G is symmetric, and the kernels compute one triangle). The
    rooflines use this count, so that no kernel can beat its bound by
    exploiting the symmetry."""
    return float(sum(float(L) * s * (s + 1) for (s, L) in blocks))


def grid_bounds(w, gridkw):
    """Row and column bounds of the workload's grid."""
    if gridkw:
        return gridkw["row_bounds"], gridkw["col_bounds"]
    br, bc = -(-w.m // w.p), -(-w.n // w.q)
    rb = np.minimum(np.arange(w.p + 1) * br, w.m)
    cb = np.minimum(np.arange(w.q + 1) * bc, w.n)
    return rb, cb


def block_shapes(w, gridkw=None):
    rb, cb = grid_bounds(w, gridkw)
    shapes = []
    for bi in range(w.p):
        mb = int(rb[bi + 1] - rb[bi])
        for bj in range(w.q):
            nb = int(cb[bj + 1] - cb[bj])
            shapes.append((min(mb, nb), max(mb, nb)))
    return shapes


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed loop."""
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,"
              "clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.path = os.path.join("/tmp", "bsvd_clocks_%d.csv" % os.getpid())

    def start(self):
        try:
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + self.FIELDS,
                 "--format=csv,noheader,nounits", "-lms", "50"],
                stdout=self.f, stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.f.close()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown",
                 "sw_power_cap"]
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx),
                "samples": len(sm), "reasons": sorted(reasons)}


def golden(w):
    path = os.path.join(ROOT, "tests", "golden", w.name + ".json")
    if os.path.exists(path):
        with open(path) as f:
            return json.load(f)
    return None


def bench_config(w, r):
    """The workload as both arms name it (identical dicts)."""
    return {"workload": w.name, "m": w.m, "n": w.n,
            "nnz_train": int(r.u_train.size), "nnz_test": int(r.u_test.size),
            "p": w.p, "q": w.q, "k": w.k, "grid": w.grid,
            "l2": "flushed (256 MB write) before each step, untimed"}


def jacobi_work(shape):
    """One-sided Jacobi work of a block, m_b n_b s_b (flops per sweep / 6)."""
    mb, nb = shape
    return float(mb) * nb * min(mb, nb)


def oracle_block_sample(w, r, count, max_work=2.0e9):
    """A bounded, spread-out sample of the workload's blocks for timing the
    oracle: of the blocks whose Jacobi work m_b n_b s_b is at most
    `max_work` (the largest blocks take the oracle hours), `count` evenly
    spaced in work order. Returns (oracle partition restricted to the
    sample's ratings, sample ids, work per block of the whole grid)."""
    import oracle
    gridkw = oracle_grid(w, r)
    g = oracle.make_grid(w.m, w.n, w.p, w.q, **gridkw)
    nb = w.p * w.q
    work = [jacobi_work(g.block_shape(b)) for b in range(nb)]
    ok = sorted((b for b in range(nb) if 0 < work[b] <= max_work),
                key=lambda b: (work[b], b))
    count = min(count, len(ok))
    pick = sorted({ok[int(round(j * (len(ok) - 1) / max(count - 1, 1)))]
                   for j in range(count)})
    b_tr, _, _ = g.locate(r.u_train, r.i_train)
    sel = np.isin(b_tr, pick)
    part = oracle.partition(w.m, w.n, r.u_train[sel], r.i_train[sel],
                            r.x_train[sel], w.p, w.q, **gridkw)
    return part, pick, work


def oracle_grid(w, r):
    """Bounds and permutations of the workload's grid, from the oracle."""
    if w.grid != "quantile":
        return {}
    import oracle
    rp, rb = oracle.activity_quantile_cut(r.u_train, w.m, w.p)
    cp, cb = oracle.activity_quantile_cut(r.i_train, w.n, w.q)
    return dict(row_bounds=rb, col_bounds=cb, row_perm=rp, col_perm=cp)


def oracle_sample(w, r, threads):
    """The oracle (as it stands) on a bounded sample: FP64 Jacobi SVDs of
    `threads` sampled blocks at once, one thread each, and the RMSE of their
    held-out ratings. The measured rate (Jacobi work per second) is scaled
    to the whole grid: value = blocks / (total work / rate)."""
    import oracle
    part, pick, work = oracle_block_sample(w, r, threads)
    t0 = time.perf_counter()
    model = oracle.factor(part, w.k, blocks=pick, threads=threads)
    b, _, _ = part.grid.locate(r.u_test, r.i_test)
    sel = np.isin(b, pick)
    if sel.any():
        oracle.rmse(model, r.u_test[sel], r.i_test[sel], r.x_test[sel])
    dt = time.perf_counter() - t0
    done = sum(work[b] for b in pick)
    nb = w.p * w.q
    value = nb / (sum(work) / (done / dt))
    return value, dt, pick, done / sum(work)


def run_reference(args, w, r, rank):
    """Reference arm: the FP64 oracle on the host cores. A step is one block
    of a bounded sample of the workload's blocks (cycling through it): its
    FP64 Jacobi SVD and the held-out RMSE of its ratings. Steps run on a
    pool of one thread per core (the C routine releases the GIL). The
    sample's rate (Jacobi work per second of wall time) is scaled to the
    whole grid, so the value is block-SVDs/s of the workload's own mix."""
    if rank != 0:
        return
    import concurrent.futures as cf
    import oracle
    oracle.build()           # once, before the worker threads use it
    cores = os.cpu_count() or 1
    t0 = time.perf_counter()
    part, pick, work = oracle_block_sample(w, r, 4 * cores, max_work=1.0e9)
    t_part = time.perf_counter() - t0
    b_te, _, _ = part.grid.locate(r.u_test, r.i_test)

    def one(step):
        b = pick[step % len(pick)]
        model = oracle.Model(part, w.k,
                             {b: oracle.factor_block(oracle.dense_block(part, b),
                                                     w.k)})
        sel = b_te == b
        if sel.any():
            oracle.rmse(model, r.u_test[sel], r.i_test[sel], r.x_test[sel])
        return work[b]
    with cf.ThreadPoolExecutor(max_workers=cores) as ex:
        list(ex.map(one, range(args.warmup)))
        t0 = time.perf_counter()
        done = sum(ex.map(one, range(args.warmup, args.warmup + args.steps)))
        wall = time.perf_counter() - t0
    nb = w.p * w.q
    raw = args.steps / wall
    value = nb / (sum(work) / (done / wall))
    sample = ("per step: one of %d sampled blocks (Jacobi work m_b n_b s_b <= "
              "1e9, evenly spread in work order; cycling), its FP64 Jacobi "
              "SVD and the RMSE of its held-out ratings; %d threads at once; "
              "%.1f sampled blocks/s, scaled by Jacobi work to the whole "
              "%d-block grid; oracle grid + partition of the sample's "
              "ratings ran first (%.1f s, not in the timing)"
              % (len(pick), cores, raw, nb, t_part))
    line = {
        "impl": "reference", "metric": "block SVDs/s", "value": value,
        "unit": "block-SVDs/s", "n_gpus": args.gpus, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": 1e3 * wall / args.steps,
        "higher_is_better": True, "scaling": "strong", "vs_baseline": None,
        "dtype": "f64", "data": "synthetic",
        "config": bench_config(w, r),
        "cpu_baseline": {"value": value, "unit": "block-SVDs/s",
                         "cores": cores, "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": "block-SVDs/s",
                "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def served_pool():
    """The served form's request pool and the held-out ratings per request."""
    from paper_1907_07410_gb300 import serve
    pool, qy = [], []
    for d in synth.served_requests(synth.SERVED_POOL_SEED,
                                   synth.SERVED_POOL_SIZE, dense=False):
        pool.append(serve.Request(d["m"], d["n"], d["k"], d["r"], d["c"],
                                  d["x"], d["qr"], d["qc"]))
        qy.append(d["qy"])
    return pool, qy


def poisson_run(srv, pool, rate, count, seed):
    """Submit `count` copies of pool requests (cycling) at Poisson arrivals
    of `rate` per second; return (results in submission order, seconds from
    the first arrival to the last completion)."""
    import dataclasses
    gaps = np.random.default_rng(seed).exponential(1.0 / rate, size=count)
    due = np.cumsum(gaps)
    futs, reqs = [], []
    t0 = time.perf_counter()
    for j in range(count):
        wait = t0 + due[j] - time.perf_counter()
        if wait > 0:
            time.sleep(wait)
        q = dataclasses.replace(pool[j % len(pool)])
        reqs.append(q)
        futs.append(srv.submit(q))
    res = [f.result(timeout=600) for f in futs]
    span = max(q.arrival + r.latency for q, r in zip(reqs, res)) - min(
        q.arrival for q in reqs)
    return res, span


def serve_leg(rates, per_rate=None, workers=4, max_batch=64, budget=120e9):
    """The served form: Poisson streams of factorise-then-predict requests
    through the continuous-batching server at each rate, beside the same
    requests run one at a time through one context. `per_rate` requests per
    rate (None: 2 s of traffic, 64 to 10,000). The predictions of a seeded
    1% sample of each stream's requests are compared with the oracle's
    fixture for the pool."""
    import paper_1907_07410_gb300 as bs
    from paper_1907_07410_gb300 import serve
    pool, qy = served_pool()
    P = len(pool)
    out = {"pool": P, "requests": "rows ~U[128,8192] x cols ~U[64,2048], "
           "3-10% observed, k in {10,20,40}, 64 held-out queries each",
           "workers": workers, "max_batch": max_batch,
           "hbm_budget_gb": budget / 1e9, "sweep": []}
    gpath = os.path.join(ROOT, "tests", "golden", "served-pool-%d.json" % P)
    gold = None
    if os.path.exists(gpath):
        with open(gpath) as f:
            gold = {q["index"]: np.array(q["yhat"])
                    for q in json.load(f)["requests"]}
    served_y = [None] * P
    sample_err, sample_diff, sample_n = [], 0.0, 0
    with serve.Server(workers=workers, max_batch=max_batch,
                      hbm_budget=budget) as srv:
        for f in [srv.submit(__import__("dataclasses").replace(q))
                  for q in pool * 2]:
            f.result(timeout=600)                  # warm-up: buffers, code
        for n, rate in enumerate(rates):
            count = int(per_rate or min(max(rate * 2.0, 64), 10000))
            nb0 = len(srv.batches)
            res, span = poisson_run(srv, pool, rate, count, 1000 + n)
            for j, r in enumerate(res[:P]):
                served_y[j] = r.yhat
            if gold is not None:
                rng = np.random.default_rng(2000 + n)
                pick = rng.choice(count, max(1, count // 100), replace=False)
                for j in sorted(pick.tolist()):
                    pj = j % P
                    if pj in gold:
                        d = res[j].yhat.astype(np.float64) - gold[pj]
                        sample_diff = max(sample_diff, float(np.max(np.abs(d))))
                        sample_err.append(res[j].yhat.astype(np.float64)
                                          - qy[pj])
                        sample_n += 1
            sizes = [len(ids) for ids, _ in srv.batches[nb0:]]
            lat = serve.latency_percentiles(res)
            out["sweep"].append({
                "rate": rate, "requests": count,
                "throughput_rps": count / span, "p50_ms": lat["p50_ms"],
                "p99_ms": lat["p99_ms"],
                "mean_batch": float(np.mean(sizes)),
                "batches": len(sizes)})
        out["max_in_flight"] = srv.max_in_flight
        out["max_held_gb"] = srv.max_held / 1e9
    # one at a time: one context, one request per call, no overlap
    ctx = bs.Context()
    for q in pool:
        serve.run_batch(ctx, [q])
    one_y, lat1 = [None] * P, []
    t0 = time.perf_counter()
    count1 = 2 * P
    for j in range(count1):
        t = time.perf_counter()
        y = serve.run_batch(ctx, [pool[j % P]])[0]
        lat1.append(time.perf_counter() - t)
        one_y[j % P] = y
    span1 = time.perf_counter() - t0
    out["one_at_a_time"] = {
        "requests": count1, "throughput_rps": count1 / span1,
        "p50_ms": float(np.percentile(lat1, 50) * 1e3),
        "p99_ms": float(np.percentile(lat1, 99) * 1e3)}
    ctx.close()
    err_s = np.concatenate([served_y[j] - qy[j] for j in range(P)])
    err_1 = np.concatenate([one_y[j] - qy[j] for j in range(P)])
    out["rmse"] = float(np.sqrt(np.mean(err_s.astype(np.float64) ** 2)))
    out["rmse_one_at_a_time"] = float(np.sqrt(np.mean(
        err_1.astype(np.float64) ** 2)))
    out["max_abs_diff_served_vs_one"] = float(max(
        np.max(np.abs(served_y[j] - one_y[j])) for j in range(P)))
    if gold is not None:
        ids = sorted(gold)
        e = np.concatenate([served_y[j] - qy[j] for j in ids])
        eo = np.concatenate([gold[j] - qy[j] for j in ids])
        got = float(np.sqrt(np.mean(e.astype(np.float64) ** 2)))
        want = float(np.sqrt(np.mean(eo ** 2)))
        out["rmse_oracle_pool"] = {
            "requests": len(ids), "served": got, "oracle": want,
            "parity": abs(got - want) <= 1e-4}
        if sample_n:
            es = np.concatenate(sample_err)
            out["oracle_sample"] = {
                "requests": sample_n, "of": "a seeded 1% of each stream",
                "max_abs_yhat_diff": sample_diff,
                "rmse_served": float(np.sqrt(np.mean(es ** 2)))}
    return out


def sgd_leg(r, w, epochs=10, grids=(8, 64, 256), gpu=0):
    """The paper's own method (blocked SGD, Algorithms 1-2) on the same
    matrix: `epochs` epochs from seeded starting factors with the Section 5
    hyper-parameters (k = 13), on the 8 x 8 grid the paper's CPU run used
    and on a finer grid (more blocks per step). The time of an epoch covers
    its schedule steps and the training-RMSE of Algorithm 1's stopping rule.
    Both arithmetic forms run: float64 (bit-identical to the float64
    oracle) and float32 (bit-identical to the float32 oracle). Beside them,
    one epoch of each sequential oracle on the host. The SM clock is
    sampled during each timed run: a walk of one warp per block keeps only
    a few SMs busy."""
    import torch
    import paper_1907_07410_gb300 as bs
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()  # noqa: E731
    k = 13
    P0, Q0 = synth.sgd_start(w.m, w.n, k)
    dP, dQ = dev(P0), dev(Q0)
    u, i, x = dev(r.u_train), dev(r.i_train), dev(r.x_train)
    out = {"k": k, "epochs": epochs, "rates": "Section 5 (SVD model)",
           "start": "P0, Q0 ~ N(0, 0.1^2) (seeded), biases 0", "grids": []}
    for g in grids:
        ctx = bs.Context()
        ctx.partition(w.m, w.n, u, i, x, g, g)
        ctx.sgd_prepare(u, i, x)
        for prec, name in ((bs.SGD_FP64, "fp64"), (bs.SGD_FP32, "fp32")):
            ctx.sgd_train(dP, dQ, max_steps=1, delta=-1e300,
                          precision=prec)                       # warm-up
            torch.cuda.synchronize()
            clocks = ClockSampler(gpu)
            clocks.start()
            t0 = time.perf_counter()
            hist, ran = ctx.sgd_train(dP, dQ, max_steps=epochs, delta=-1e300,
                                      precision=prec)
            torch.cuda.synchronize()
            dt = time.perf_counter() - t0
            clk = clocks.stop()
            yh = ctx.sgd_predict(r.u_test, r.i_test)
            test = float(np.sqrt(np.mean((yh - r.x_test) ** 2)))
            out["grids"].append({
                "grid": "%dx%d" % (g, g), "precision": name,
                "s_per_epoch": dt / ran,
                "ratings_per_s": r.u_train.size * ran / dt,
                "train_rmse_start": float(hist[0]),
                "train_rmse_end": float(hist[-1]), "test_rmse_end": test,
                "clocks": clk})
    # the oracle: one epoch, sequential, on the host
    import oracle
    from oracle import sgd as osgd
    grid = oracle.make_grid(w.m, w.n, grids[0], grids[0])
    order = osgd.processing_order(grid, r.u_train, r.i_train)
    uo, io, xo = r.u_train[order], r.i_train[order], r.x_train[order]
    for dt, key, name in ((np.float64, "cpu_baseline", "FP64"),
                          (np.float32, "cpu_baseline_fp32", "FP32")):
        P, Q = P0.astype(dt), Q0.astype(dt)
        bu, bi = np.zeros(w.m, dt), np.zeros(w.n, dt)
        t0 = time.perf_counter()
        osgd.sgd_pass(uo, io, xo, P, Q, bu, bi, osgd.Rates())
        out[key] = {"kind": "oracle", "cores": 1,
                    "s_per_epoch": time.perf_counter() - t0,
                    "sample": "one epoch of the sequential %s oracle (C), "
                              "%dx%d grid order" % (name, grids[0], grids[0])}
    out["paper_context"] = ("BGSVD 13.45 s/iteration and BCSVD 34.53 "
                            "s/iteration on MovieLens 1M (Tesla M40, Xeon "
                            "E5-2640 v3); real data, not comparable")
    return out


def grid_bounds_of(w, r):
    """Row and column bounds of the workload's grid, for counting the
    method's work: the activity-quantile cut (from the library) or the
    paper's equal blocks."""
    if w.grid != "quantile":
        return None
    import paper_1907_07410_gb300 as bs
    with bs.Context() as ctx:
        kw = ctx.quantile_grid(w.m, w.n, r.u_train, r.i_train, w.p, w.q)
    return kw


def step_rmse(ctx, u, i, y, sharded):
    """The step's held-out RMSE: on one GPU the library's; across ranks each
    rank's squared-error sum over its own blocks, combined by one
    all-reduce of the sum and the count."""
    if not sharded:
        return ctx.rmse(u, i, y)
    from paper_1907_07410_gb300 import dist as bdist
    return bdist.sharded_rmse(ctx, u, i, y)


def time_form(w, data, steps, warmup, flush, stream, owned=None, **cfg):
    """Warm up, then time `steps` steps of one form of the path (this rank's
    blocks only when `owned` is given). Returns the per-step times, phases,
    RMSE, launches and the solver report."""
    import torch
    import paper_1907_07410_gb300 as bs
    u_tr, i_tr, x_tr, u_te, i_te, x_te = data
    ctx = bs.Context(stream=stream, profile=1, **cfg)
    sharded = owned is not None
    if sharded:
        ctx.set_owned(owned)
    for _ in range(warmup):
        step_partition(ctx, w, u_tr, i_tr, x_tr)
        ctx.factor(w.k, warn=False)
        step_rmse(ctx, u_te, i_te, x_te, sharded)
    phases = {k: [] for k in bs.PHASES}
    step_ms = []
    launches0 = ctx.kernel_launches()
    for _ in range(steps):
        flush.fill_(1)                       # evict L2 between steps (untimed)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        step_partition(ctx, w, u_tr, i_tr, x_tr)
        part_ph = ctx.phase_times()["partition"]
        status = ctx.factor(w.k, warn=False)
        fac_ph = ctx.phase_times()
        rm = step_rmse(ctx, u_te, i_te, x_te, sharded)
        e1.record(stream)
        e1.synchronize()
        step_ms.append(e0.elapsed_time(e1))
        ph = ctx.phase_times()
        phases["partition"].append(part_ph)
        for key in ("gram", "eigen", "project", "eigen_filter", "eigen_rr",
                    "eigen_other"):
            phases[key].append(fac_ph[key])
        phases["predict"].append(ph["predict"])
    return dict(ctx=ctx, step_ms=step_ms, rmse=rm, status=status,
                loop={1: "host-driven", 2: "CUDA graph, device-driven"}.get(
                    ctx.loop_form(), "none"),
                launches=ctx.kernel_launches() - launches0,
                phases={k: statistics.mean(v) for k, v in phases.items()},
                report=dict(ctx.factor_report(full=True),
                            launches=ctx.panel_launches()),
                gram_path=ctx.gram_path())


def step_partition(ctx, w, u, i, x):
    """The step's partition: for the uneven workloads the activity-quantile
    cut and the partition on it in one library call (the ratings go up
    once when they are on the host), else the paper's equal blocks."""
    if w.grid == "quantile":
        ctx.partition_quantile(w.m, w.n, u, i, x, w.p, w.q)
    else:
        ctx.partition(w.m, w.n, u, i, x, w.p, w.q)


def step_grid(ctx, w, u, i):
    """The grid's bounds and permutations for partition(): the activity-
    quantile cut (computed by the library, part of the step) for the
    uneven workloads, the paper's equal blocks otherwise."""
    if w.grid != "quantile":
        return {}
    return ctx.quantile_grid(w.m, w.n, u, i, w.p, w.q)


GRAM_NAMES = {1: "fp32 simt", 2: "tensor cores, exact (bf16 planes)",
              3: "tensor cores, tf32", 4: "tensor cores, bf16"}
GRAM_KERNELS = {1: "k_gram_f32", 2: "k_gram_tc", 3: "k_gram_tf32",
                4: "k_gram_bf16"}


def gram_peak(gram_path, peaks, peak_kind):
    """(bound, peak TFLOP/s, what the peak is) of a Gram kernel."""
    bf16 = peaks.get("bf16_tflops", 1900.0)
    if gram_path in (2, 4):
        return "tensor", bf16, "bf16 dense, burst, of %s" % peak_kind
    if gram_path == 3:
        return "tensor", 0.5 * bf16, "0.5 x bf16 dense burst, of %s" % peak_kind
    return "alu", fp32_alu_peak_tflops(peaks), (
        "152 SMs x 128 FP32 lanes x 2 x %.0f MHz" % peaks.get("sm_max_mhz",
                                                           2070.0))


def step_roofline(w, r, shapes, keff, gram_path, step_s, peaks, peak_kind):
    """The whole step against its roofline: the method's algorithmic flops
    (Gram 2 m_b n_b s_b, projection 2 m_b n_b k, prediction 2 k per query)
    and bytes (COO read 12 B per training rating, dense blocks written once
    in float32, read once by the Gram in its operand type and once by the
    projection in float32, 12 B plus two k-float factor rows per query).
    The eigen-solver's iterations are not counted."""
    cells = float(sum(s * L for (s, L) in shapes))
    f_gram = gram_flops_min(shapes)
    f_proj = 2.0 * sum(s * L * min(keff, s) for (s, L) in shapes)
    f_pred = 2.0 * keff * r.u_test.size
    gram_operand = {1: 4, 2: 4, 3: 4, 4: 2}.get(gram_path, 4)
    by = (12.0 * r.u_train.size + cells * (4 + gram_operand + 4)
          + r.u_test.size * (12.0 + 8.0 * keff))
    bound, tc_peak, _ = gram_peak(gram_path, peaks, peak_kind)
    flops = f_gram + f_proj + f_pred
    t_tc = flops / (tc_peak * 1e12)
    t_hbm = by / (peaks.get("hbm_gbs", 6800.0) * 1e9)
    t_roof = max(t_tc, t_hbm)
    return {"bound": (bound if t_tc >= t_hbm else "hbm"),
            "roofline_ms": t_roof * 1e3, "measured_ms": step_s * 1e3,
            "frac": t_roof / step_s, "algorithmic_flops": flops,
            "algorithmic_bytes": by, "tensor_ms": t_tc * 1e3,
            "hbm_ms": t_hbm * 1e3,
            "note": "the Gram counted as its s(s+1)/2 distinct entries "
                    "(2 L flop each); eigen-solver iterations excluded from "
                    "the work; the exact Gram counts its float32 operand "
                    "bytes"}


def panel_roofline(w, shapes, rep, filter_ms, peaks, peak_kind,
                   oversample=0):
    """The eigen-solver's panel products G X (k_gpanel_tc): algorithmic
    bytes per product = G once (4 s^2) + the panel in and out (4 s b each),
    summed over every product of every block and divided by the products'
    own device time (the library sums each launch's span, first CTA start
    to last CTA end, with the GPU's timer). b/2 flop per byte of G: far
    below the tensor ridge, so the bound is bandwidth. b is the subspace
    width the schedule's oversample gives (the library's rule)."""
    want = w.k + (oversample if oversample > 0 else max(8, w.k // 2))
    bsub = 16 if want <= 16 else (32 if want <= 32 else 64)
    pflops = pbytes = 0.0
    nprod = 0
    for (s_b, L_b), prods in zip(shapes, rep["products"]):
        n_f = int(prods)
        b_b = min(bsub, s_b)
        pflops += n_f * 2.0 * s_b * s_b * b_b
        pbytes += n_f * (4.0 * s_b * s_b + 8.0 * s_b * b_b)
        nprod += int(prods)
    t = filter_ms * 1e-3
    hbm = peaks.get("hbm_gbs", 6800.0)
    gbs = pbytes / t / 1e9 if t > 0 else 0.0
    tf = pflops / t / 1e12 if t > 0 else 0.0
    tf32 = 0.5 * peaks.get("bf16_tflops", 1900.0)
    ratio = profiled_traffic_ratio("k_gpanel_tc")
    nlaunch = max(int(rep.get("launches", 0)), 1)
    return {"kernel": "k_gpanel_tc", "bound": "hbm", "achieved": gbs,
            "peak": hbm, "unit": "GB/s", "frac": gbs / hbm,
            "traffic": (ratio * pbytes / nlaunch if ratio else None),
            "traffic_ratio": ratio, "launches": nlaunch,
            "peak_source": "STREAM-style copy, of %s" % peak_kind,
            "products": nprod, "algorithmic_bytes": pbytes,
            "tensor_tflops": tf,
            "tensor_frac_of_fp32_equivalent": tf / (tf32 / 3.0),
            "note": "algorithmic bytes (G once, panel in and out) of all "
                    "block products over the products' summed device time; "
                    "tensor_tflops counts 2 s^2 b flops per product "
                    "against one third of the tf32 peak (0.5 x measured "
                    "bf16), as the kernel issues three tf32 products for "
                    "float32 accuracy"}


def form_summary(w, r, res, gold, steps):
    total = sum(res["step_ms"])
    g_rmse = gold["rmse"] if gold else None
    rep = res["report"]
    return {"value": w.p * w.q * steps / (total * 1e-3),
            "ms_per_step": total / steps, "steps": steps,
            "gram": GRAM_NAMES.get(res["gram_path"], "none"),
            "eigen_loop": res["loop"],
            "rmse": res["rmse"], "rmse_oracle": g_rmse,
            "rmse_parity": (g_rmse is not None
                            and abs(res["rmse"] - g_rmse) <= 1e-4),
            "converged_blocks": int(np.sum(rep["converged"])),
            "phases_ms": res["phases"]}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=100)
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--impl", default="ours", choices=("ours", "reference"))
    ap.add_argument("--workload", default=synth.LARGE.name,
                    choices=sorted(synth.WORKLOADS))
    ap.add_argument("--precision", default="bf16",
                    choices=("fp32", "tf32", "bf16"))
    ap.add_argument("--forms", default="exact,plain",
                    help="other forms timed beside the main one: exact "
                         "(tensor-core exact Gram, float32 result), plain "
                         "(FP32 SIMT Gram, panel products and projection); "
                         "empty to skip")
    ap.add_argument("--form-steps", type=int, default=3,
                    help="timed steps of each other form (after 3 warm-up steps)")
    ap.add_argument("--no-medium", action="store_true",
                    help="skip the medium-matrix leg")
    ap.add_argument("--loop", default="tuned",
                    choices=("tuned", "host", "graph"),
                    help="eigen loop form: the autotuner's choice, or forced "
                         "host-driven (ncu cannot profile kernels inside a "
                         "graph with conditional nodes) or graph")
    ap.add_argument("--no-autotune", action="store_true",
                    help="keep the default eigen-solver schedule instead of "
                         "the autotuner's choice for this workload")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-sgd", action="store_true",
                    help="skip the blocked-SGD leg (the paper's Algorithms 1-2)")
    ap.add_argument("--serve-rates", default="50,100,200,500,1000,2000,5000",
                    help="Poisson rates (req/s) of the served-form leg; "
                         "empty to skip it")
    ap.add_argument("--serve-requests", type=int, default=0,
                    help="requests per rate (0: 2 s of traffic, 64 to 10000)")
    args = ap.parse_args()
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    w = synth.WORKLOADS[args.workload]
    r = synth.generate(w)

    if args.impl == "reference":
        run_reference(args, w, r, rank)
        return

    import torch
    import paper_1907_07410_gb300 as bs
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    def barrier():
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()

    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()  # noqa: E731
    stream = torch.cuda.current_stream()
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    def device_data(rr):
        return (dev(rr.u_train), dev(rr.i_train), dev(rr.x_train),
                dev(rr.u_test), dev(rr.i_test), dev(rr.x_test))

    data = device_data(r)
    prec = {"fp32": bs.FP32, "tf32": bs.TF32, "bf16": bs.BF16}
    nblocks = w.p * w.q
    shapes = block_shapes(w, grid_bounds_of(w, r))
    owned = None
    if world > 1:
        # this rank's share of the blocks (longest processing time first)
        from paper_1907_07410_gb300 import dist as bdist
        owned = bdist.owned_mask(bdist.block_costs(shapes), world, rank)

    # ---- the solver schedule for this workload (autotuner, cached) -------
    tuned = {"params": {}, "note": "default schedule (--no-autotune)"}
    if not args.no_autotune and world == 1:
        from paper_1907_07410_gb300 import autotune
        with bs.Context() as gctx:
            gkw = step_grid(gctx, w, data[0], data[1])
        tuned = autotune.tune(w.m, w.n, w.p, w.q, w.k, *data, shapes,
                              precision=prec[args.precision], grid=gkw,
                              stream=stream)

    # ---- device-resident timed region (the main form) --------------------
    clocks = ClockSampler(local)
    barrier()
    clocks.start()
    params = dict(tuned["params"])
    if args.loop != "tuned":
        params["loop"] = {"host": 1, "graph": 2}[args.loop]
    main_res = time_form(w, data, args.steps, args.warmup, flush, stream,
                         owned, precision=prec[args.precision], **params)
    barrier()
    clk = clocks.stop()
    ctx = main_res["ctx"]
    total_ms = sum(main_res["step_ms"])
    if dist is not None:
        from paper_1907_07410_gb300 import dist as bdist
        total_ms = bdist.max_over_ranks(total_ms)

    # ---- end to end through the public API with host buffers -------------
    pin = lambda a: torch.from_numpy(np.ascontiguousarray(a)).pin_memory()  # noqa: E731
    h_u, h_i, h_x = pin(r.u_train), pin(r.i_train), pin(r.x_train)
    h_ut, h_it, h_xt = pin(r.u_test), pin(r.i_test), pin(r.x_test)
    e2e_ms = []
    barrier()
    for _ in range(args.steps):
        flush.fill_(1)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        step_partition(ctx, w, h_u, h_i, h_x)
        ctx.factor(w.k, warn=False)
        rm_e2e = step_rmse(ctx, h_ut, h_it, h_xt, owned is not None)
        e2e_ms.append(1e3 * (time.perf_counter() - t0))
    barrier()
    e2e_total = sum(e2e_ms)
    if dist is not None:
        e2e_total = bdist.max_over_ranks(e2e_total)
    ctx.close()

    # ---- the other forms, the same workload ------------------------------
    forms = {}
    form_cfg = {"exact": dict(precision=bs.FP32),
                "plain": dict(precision=bs.FP32, gram_path=1, panel_path=1),
                "bf16": dict(precision=bs.BF16), "tf32": dict(precision=bs.TF32)}
    for name in [f for f in args.forms.split(",") if f.strip()]:
        fcfg = dict(form_cfg[name])
        if args.loop != "tuned":
            fcfg["loop"] = {"host": 1, "graph": 2}[args.loop]
        res = time_form(w, data, args.form_steps, 3, flush, stream,
                        owned, **fcfg)
        res["ctx"].close()
        forms[name] = res

    if rank != 0:
        if dist is not None:
            dist.destroy_process_group()
        return

    quant = w.grid == "quantile"
    # the ratings once, and the held-out ones; the grid's bounds come back
    e2e_h2d = int(12 * (r.u_train.size + r.u_test.size))
    e2e_d2h = int(8 + (8 * (w.p + w.q + 2) if quant else 0))
    peaks, peak_kind = load_peaks()
    gold = golden(w)
    gflops = gram_flops(shapes)
    gflops_min = gram_flops_min(shapes)
    gram_path = main_res["gram_path"]
    bound, gpeak, gsrc = gram_peak(gram_path, peaks, peak_kind)
    gram_ms = main_res["phases"]["gram"]
    g_tf = gflops_min / (gram_ms * 1e-3) / 1e12 if gram_ms > 0 else 0.0
    # the Gram's algorithmic bytes: its operand read once, G written once
    opnd = {1: 4, 2: 4, 3: 4, 4: 2}.get(gram_path, 4) * (2 if gram_path == 2 else 1)
    gram_bytes = float(sum(opnd * s * L + 4.0 * s * s for (s, L) in shapes))
    gram_ratio = profiled_traffic_ratio(GRAM_KERNELS.get(gram_path))
    # the ranks share the workload's blocks: all of them per step
    value = nblocks * args.steps / (total_ms * 1e-3)
    step_s = total_ms * 1e-3 / args.steps
    proj_flops = 2.0 * sum(L * s * min(w.k, s) for (s, L) in shapes)
    pred_flops = 2.0 * w.k * r.u_test.size
    tflops = (gflops_min + proj_flops + pred_flops) / step_s / 1e12
    main_sum = form_summary(w, r, main_res, gold, args.steps)
    line = {
        "metric": "block SVDs/s", "value": value, "unit": "block-SVDs/s",
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": total_ms / args.steps, "higher_is_better": True,
        "scaling": "strong", "vs_baseline": None,
        "dtype": {"fp32": "f32", "tf32": "tf32 gram, f32",
                  "bf16": "bf16 gram, f32"}[args.precision],
        "data": "synthetic (seeded, shaped like the paper's rating data; "
                "inputs in HBM)",
        "config": bench_config(w, r),
        "path": {"precision": args.precision,
                 "gram": GRAM_NAMES.get(gram_path, "none"),
                 "eigen_loop": main_res["loop"],
                 "schedule": params or "default"},
        "autotune": {k: v for k, v in tuned.items() if k != "trials"},
        "latency_ms": {"p50": float(np.percentile(main_res["step_ms"], 50)),
                       "p99": float(np.percentile(main_res["step_ms"], 99))},
        "tflops": tflops,
        "phases_ms": main_res["phases"],
        "rmse": main_res["rmse"], "rmse_oracle": main_sum["rmse_oracle"],
        "rmse_parity": main_sum["rmse_parity"],
        "converged_blocks": main_sum["converged_blocks"],
        "roofline": panel_roofline(w, shapes, main_res["report"],
                                   main_res["phases"]["eigen_filter"], peaks,
                                   peak_kind, params.get("oversample", 0)),
        "roofline_step": step_roofline(w, r, shapes, w.k, gram_path, step_s,
                                       peaks, peak_kind),
        "roofline_gram": {"kernel": GRAM_KERNELS.get(gram_path), "bound": bound,
                          "achieved": g_tf, "peak": gpeak, "unit": "TFLOP/s",
                          "frac": g_tf / gpeak,
                          "traffic": (gram_ratio * gram_bytes
                                      if gram_ratio else None),
                          "traffic_ratio": gram_ratio,
                          "algorithmic_flops_per_launch": gflops_min,
                          "full_product_flops": gflops,
                          "peak_source": gsrc,
                          "note": "algorithmic flops: the symmetric Gram's "
                                  "distinct entries, L s (s+1) per block "
                                  "(half of 2 L s^2 plus the diagonal)"},
        "forms": {name: form_summary(w, r, res, gold, args.form_steps)
                  for name, res in forms.items()},
        "gpu_launches": int(main_res["launches"]),
        "e2e": {"value": nblocks * args.steps / (e2e_total * 1e-3),
                "unit": "block-SVDs/s",
                "h2d_bytes_per_step": e2e_h2d, "d2h_bytes_per_step": e2e_d2h,
                "rmse": rm_e2e,
                "note": "host (pinned) inputs every step: the training "
                        "ratings go up once (partition_quantile: x while "
                        "the grid is cut), the held-out ones for the RMSE"},
        "clocks": clk,
    }
    if world == 1 and not args.no_medium and w.name != synth.MEDIUM.name:
        wm = synth.MEDIUM
        rm_ = synth.generate(wm)
        dm = device_data(rm_)
        mparams = {}
        if not args.no_autotune:
            from paper_1907_07410_gb300 import autotune
            mparams = autotune.tune(wm.m, wm.n, wm.p, wm.q, wm.k, *dm,
                                    block_shapes(wm), stream=stream,
                                    precision=prec[args.precision])["params"]
        res = time_form(wm, dm, args.steps, args.warmup, flush, stream,
                        precision=prec[args.precision], **mparams)
        res["ctx"].close()
        line["medium"] = dict(form_summary(wm, rm_, res, golden(wm),
                                           args.steps), workload=wm.name,
                              schedule=mparams or "default")
    if world == 1 and not args.no_cpu_baseline:
        cores = min(os.cpu_count() or 1, nblocks)
        value_cpu, dt, pick, frac = oracle_sample(w, r, cores)
        line["cpu_baseline"] = {
            "value": value_cpu, "unit": "block-SVDs/s", "cores": cores,
            "kind": "oracle",
            "sample": "FP64 Jacobi SVDs of %d of the %d blocks (Jacobi work "
                      "m_b n_b s_b <= 2e9, evenly spread in work order; one "
                      "thread each) and their held-out RMSE, %.1f s for "
                      "%.2f%% of the grid's Jacobi work; scaled by work to "
                      "the whole grid" % (len(pick), nblocks, dt, 100 * frac)}
    rates = [float(v) for v in args.serve_rates.split(",") if v.strip()]
    if world == 1 and rates:
        line["served"] = serve_leg(rates, args.serve_requests or None)
    if world == 1 and not args.no_sgd:
        wm = synth.MEDIUM
        line["sgd"] = sgd_leg(synth.generate(wm), wm, gpu=local)
    print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
