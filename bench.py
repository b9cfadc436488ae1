"""Benchmark of the block-SVD recommender hot path on GB300.

One step = the whole hot path on one synthetic rating matrix already in
HBM: partition + block means + dense scatter, Gram products, truncated
eigen-solve, projection, held-out prediction and RMSE. The default workload
is the MovieLens-1M-shaped matrix (6040 users x 3952 items, 1,000,209
ratings, 90/10 split) on a 4 x 4 grid with k = 20.

At N=1 the line also carries the served form ("served"): Poisson streams of
factorise-then-predict requests through the continuous-batching server, at
each --serve-rates rate, beside the same requests run one at a time; and the
paper's own blocked SGD ("sgd", Algorithms 1-2): seconds per epoch on the
same matrix, beside one epoch of the FP64 oracle.

Prints one JSON line (rank 0). Usage:
    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
Under torchrun each rank solves its own copy of the workload (weak scaling;
no collective on the data path).
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
# DRAM bytes (read + write) of one k_gram_tc launch, from the ncu capture
# summarised in profiles/k_gram_tc_medium-4x4-k20.md; None until captured.
GRAM_TC_TRAFFIC = {"medium-6040x3952-4x4-k20": 133.9e6}
GRAM_BF16_TRAFFIC = {}
# DRAM bytes of one k_gpanel_tc launch with every block running, from the
# ncu capture summarised in profiles/k_gpanel_tc_medium-4x4-k20.md.
PANEL_TRAFFIC = {"medium-6040x3952-4x4-k20": 67.94e6}


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
    """Algorithmic Gram work: 2 m_b n_b s_b flop per block (s = min side)."""
    return float(sum(2.0 * L * s * s for (s, L) in blocks))


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


def golden_rmse(w):
    path = os.path.join(ROOT, "tests", "golden", w.name + ".json")
    if os.path.exists(path):
        with open(path) as f:
            return json.load(f)["rmse"]
    return None


def oracle_sample(w, r, nblocks, threads, gridkw=None):
    """The oracle (as it stands) on a bounded sample: partition of all the
    ratings, factorisation of the `nblocks` blocks with the fewest cells
    (lowest ids on ties), RMSE over their held-out ratings.
    Returns (seconds, blocks)."""
    import oracle
    t0 = time.perf_counter()
    part = oracle.partition(w.m, w.n, r.u_train, r.i_train, r.x_train, w.p,
                            w.q, **(gridkw or {}))
    cells = [np.prod(part.grid.block_shape(b)) for b in range(w.p * w.q)]
    ids = sorted(int(b) for b in
                 np.argsort(cells, kind="stable")[:min(nblocks, w.p * w.q)])
    model = oracle.factor(part, w.k, blocks=ids, threads=threads)
    b, _, _ = part.grid.locate(r.u_test, r.i_test)
    sel = np.isin(b, ids)
    if sel.any():
        oracle.rmse(model, r.u_test[sel], r.i_test[sel], r.x_test[sel])
    return time.perf_counter() - t0, len(ids)


def run_reference(args, w, r, rank):
    """Reference arm: the FP64 oracle on the host cores. A step is one block
    of the workload (cycling through the grid): its FP64 Jacobi SVD and the
    held-out RMSE of its ratings. Steps run on a pool of one thread per
    core (the C routine releases the GIL), so the value is the oracle's
    throughput on the whole host: timed blocks / wall time."""
    if rank != 0:
        return
    import concurrent.futures as cf
    import oracle
    oracle.build()           # once, before the worker threads use it
    cores = os.cpu_count() or 1
    gridkw = host_grid(w, r)
    t0 = time.perf_counter()
    part = oracle.partition(w.m, w.n, r.u_train, r.i_train, r.x_train, w.p,
                            w.q, **(gridkw or {}))
    t_part = time.perf_counter() - t0
    b_te, _, _ = part.grid.locate(r.u_test, r.i_test)
    nb = w.p * w.q

    def one(step):
        b = step % nb
        t = time.perf_counter()
        model = oracle.Model(part, w.k,
                             {b: oracle.factor_block(oracle.dense_block(part, b),
                                                     w.k)})
        sel = b_te == b
        if sel.any():
            oracle.rmse(model, r.u_test[sel], r.i_test[sel], r.x_test[sel])
        return time.perf_counter() - t
    with cf.ThreadPoolExecutor(max_workers=cores) as ex:
        list(ex.map(one, range(args.warmup)))
        t0 = time.perf_counter()
        per = list(ex.map(one, range(args.warmup, args.warmup + args.steps)))
        wall = time.perf_counter() - t0
    value = args.steps / wall
    sample = ("per step: one block of the %d (cycling), FP64 Jacobi SVD of "
              "its centred dense block and the RMSE of its held-out ratings; "
              "steps on %d threads at once; the oracle partition of all %d "
              "training ratings ran once first (%.2f s, not in the timing)"
              % (nb, cores, r.u_train.size, t_part))
    line = {
        "impl": "reference", "metric": "block SVDs/s", "value": value,
        "unit": "block-SVDs/s", "n_gpus": args.gpus, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": 1e3 * statistics.mean(per),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f64", "data": "synthetic",
        "config": {"workload": w.name, "m": w.m, "n": w.n, "p": w.p,
                   "q": w.q, "k": w.k},
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


def serve_leg(rates, workers=4, max_batch=64, budget=120e9):
    """The served form: Poisson streams of factorise-then-predict requests
    through the continuous-batching server at each rate, beside the same
    requests run one at a time through one context."""
    import paper_1907_07410_gb300 as bs
    from paper_1907_07410_gb300 import serve
    pool, qy = served_pool()
    P = len(pool)
    out = {"pool": P, "requests": "rows ~U[128,8192] x cols ~U[64,2048], "
           "3-10% observed, k in {10,20,40}, 64 held-out queries each",
           "workers": workers, "max_batch": max_batch,
           "hbm_budget_gb": budget / 1e9, "sweep": []}
    served_y = [None] * P
    with serve.Server(workers=workers, max_batch=max_batch,
                      hbm_budget=budget) as srv:
        for f in [srv.submit(__import__("dataclasses").replace(q))
                  for q in pool * 2]:
            f.result(timeout=600)                  # warm-up: buffers, code
        for n, rate in enumerate(rates):
            count = int(min(max(rate * 2.0, 64), 1500))
            nb0 = len(srv.batches)
            res, span = poisson_run(srv, pool, rate, count, 1000 + n)
            for j, r in enumerate(res[:P]):
                served_y[j] = r.yhat
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
    gpath = os.path.join(ROOT, "tests", "golden",
                         "served-pool-%d.json" % P)
    if os.path.exists(gpath):
        with open(gpath) as f:
            g = json.load(f)
        ids = [q["index"] for q in g["requests"]]
        e = np.concatenate([served_y[j] - qy[j] for j in ids])
        got = float(np.sqrt(np.mean(e.astype(np.float64) ** 2)))
        out["rmse_oracle_subset"] = {
            "requests": len(ids), "served": got, "oracle": g["rmse"],
            "parity": abs(got - g["rmse"]) <= 1e-4}
    return out


def sgd_leg(r, w, epochs=10, grids=(8, 64, 256)):
    """The paper's own method (blocked SGD, Algorithms 1-2) on the same
    matrix: `epochs` epochs from seeded starting factors with the Section 5
    hyper-parameters (k = 13), on the 8 x 8 grid the paper's CPU run used
    and on a finer grid (more blocks per step). The time of an epoch covers
    its schedule steps and the training-RMSE of Algorithm 1's stopping rule.
    Beside it, one epoch of the sequential FP64 oracle on the host."""
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
        ctx.sgd_train(dP, dQ, max_steps=1, delta=-1e300)       # warm-up
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        hist, ran = ctx.sgd_train(dP, dQ, max_steps=epochs, delta=-1e300)
        torch.cuda.synchronize()
        dt = time.perf_counter() - t0
        yh = ctx.sgd_predict(r.u_test, r.i_test)
        test = float(np.sqrt(np.mean((yh - r.x_test) ** 2)))
        out["grids"].append({
            "grid": "%dx%d" % (g, g), "s_per_epoch": dt / ran,
            "ratings_per_s": r.u_train.size * ran / dt,
            "train_rmse_start": float(hist[0]),
            "train_rmse_end": float(hist[-1]), "test_rmse_end": test})
    # the oracle: one epoch, sequential, on the host
    import oracle
    from oracle import sgd as osgd
    grid = oracle.make_grid(w.m, w.n, grids[0], grids[0])
    order = osgd.processing_order(grid, r.u_train, r.i_train)
    uo, io, xo = r.u_train[order], r.i_train[order], r.x_train[order]
    P, Q = P0.copy(), Q0.copy()
    bu, bi = np.zeros(w.m), np.zeros(w.n)
    t0 = time.perf_counter()
    osgd.sgd_pass(uo, io, xo, P, Q, bu, bi, osgd.Rates())
    out["cpu_baseline"] = {"kind": "oracle", "cores": 1,
                           "s_per_epoch": time.perf_counter() - t0,
                           "sample": "one epoch of the sequential FP64 oracle "
                                     "(C), %dx%d grid order" % (grids[0],
                                                                grids[0])}
    out["paper_context"] = ("BGSVD 13.45 s/iteration and BCSVD 34.53 "
                            "s/iteration on MovieLens 1M (Tesla M40, Xeon "
                            "E5-2640 v3); real data, not comparable")
    return out


def host_grid(w, r):
    """Bounds and permutations of an activity-quantile grid (host side)."""
    if w.grid != "quantile":
        return None
    from paper_1907_07410_gb300 import grid
    return grid.quantile_grid(r.u_train, r.i_train, w.m, w.n, w.p, w.q)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=100)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=("ours", "reference"))
    ap.add_argument("--workload", default=synth.MEDIUM.name,
                    choices=sorted(synth.WORKLOADS))
    ap.add_argument("--precision", default="fp32",
                    choices=("fp32", "tf32", "bf16"))
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-sgd", action="store_true",
                    help="skip the blocked-SGD leg (the paper's Algorithms 1-2)")
    ap.add_argument("--serve-rates", default="50,500,5000",
                    help="Poisson rates (req/s) of the served-form leg; "
                         "empty to skip it")
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
    gridkw = host_grid(w, r)
    pkw = {}
    if gridkw:
        pkw = dict(row_bounds=gridkw["row_bounds"],
                   col_bounds=gridkw["col_bounds"],
                   row_perm=dev(gridkw["row_perm"]),
                   col_perm=dev(gridkw["col_perm"]))
    u_tr, i_tr, x_tr = dev(r.u_train), dev(r.i_train), dev(r.x_train)
    u_te, i_te, x_te = dev(r.u_test), dev(r.i_test), dev(r.x_test)
    stream = torch.cuda.current_stream()
    ctx = bs.Context(stream=stream, profile=1,
                     precision={"fp32": bs.FP32, "tf32": bs.TF32,
                                "bf16": bs.BF16}[args.precision])
    nblocks = w.p * w.q
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")

    def step():
        ctx.partition(w.m, w.n, u_tr, i_tr, x_tr, w.p, w.q, **pkw)
        ctx.factor(w.k)
        return ctx.rmse(u_te, i_te, x_te)

    for _ in range(args.warmup):
        rm = step()

    # ---- device-resident timed region -----------------------------------
    phases = {k: [] for k in bs.PHASES}
    step_ms = []
    launches0 = ctx.kernel_launches()
    clocks = ClockSampler(local)
    barrier()
    clocks.start()
    for _ in range(args.steps):
        flush.fill_(1)                       # evict L2 between steps (untimed)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        ctx.partition(w.m, w.n, u_tr, i_tr, x_tr, w.p, w.q, **pkw)
        part_ph = ctx.phase_times()["partition"]
        ctx.factor(w.k)
        fac_ph = ctx.phase_times()
        rm = ctx.rmse(u_te, i_te, x_te)
        e1.record(stream)
        e1.synchronize()
        step_ms.append(e0.elapsed_time(e1))
        ph = ctx.phase_times()
        phases["partition"].append(part_ph)
        for key in ("gram", "eigen", "project", "eigen_filter", "eigen_rr",
                    "eigen_other"):
            phases[key].append(fac_ph[key])
        phases["predict"].append(ph["predict"])
    barrier()
    clk = clocks.stop()
    launches = ctx.kernel_launches() - launches0
    total_ms = sum(step_ms)
    if dist is not None:
        from paper_1907_07410_gb300 import dist as bdist
        total_ms = bdist.max_over_ranks(total_ms)

    # ---- end to end through the public API with host buffers -------------
    pin = lambda a: torch.from_numpy(np.ascontiguousarray(a)).pin_memory()  # noqa: E731
    h_u, h_i, h_x = pin(r.u_train), pin(r.i_train), pin(r.x_train)
    h_ut, h_it, h_xt = pin(r.u_test), pin(r.i_test), pin(r.x_test)
    pkw_host = {}
    if gridkw:
        pkw_host = dict(row_bounds=gridkw["row_bounds"],
                        col_bounds=gridkw["col_bounds"],
                        row_perm=pin(gridkw["row_perm"]),
                        col_perm=pin(gridkw["col_perm"]))
    e2e_ms = []
    barrier()
    for _ in range(args.steps):
        flush.fill_(1)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        ctx.partition(w.m, w.n, h_u, h_i, h_x, w.p, w.q, **pkw_host)
        ctx.factor(w.k)
        rm_e2e = ctx.rmse(h_ut, h_it, h_xt)
        e2e_ms.append(1e3 * (time.perf_counter() - t0))
    barrier()
    e2e_total = sum(e2e_ms)
    if dist is not None:
        e2e_total = bdist.max_over_ranks(e2e_total)

    if rank != 0:
        if dist is not None:
            dist.destroy_process_group()
        return

    peaks, peak_kind = load_peaks()
    shapes = block_shapes(w, gridkw)
    gflops = gram_flops(shapes)
    gram_ms = statistics.mean(phases["gram"])
    achieved = gflops / (gram_ms * 1e-3) / 1e12
    gram_path = ctx.gram_path()
    if gram_path == 4:
        roof = {"kernel": "k_gram_bf16", "bound": "tensor",
                "peak": peaks.get("bf16_tflops", 1900.0),
                "peak_source": "bf16 dense, burst, of %s" % peak_kind,
                "traffic": GRAM_BF16_TRAFFIC.get(w.name)}
    elif gram_path == 3:
        # tf32 peak: the bf16 measurement scaled by the nominal ratio 1/2
        roof = {"kernel": "k_gram_tf32", "bound": "tensor",
                "peak": 0.5 * peaks.get("bf16_tflops", 1900.0),
                "peak_source": "0.5 x bf16 dense burst, of %s" % peak_kind,
                "traffic": None}
    elif gram_path == 2:
        roof = {"kernel": "k_gram_tc", "bound": "tensor",
                "peak": peaks.get("bf16_tflops", 1900.0),
                "peak_source": "bf16 dense, burst, of %s" % peak_kind,
                "traffic": GRAM_TC_TRAFFIC.get(w.name)}
    else:
        roof = {"kernel": "k_gram_f32", "bound": "alu",
                "peak": fp32_alu_peak_tflops(peaks),
                "peak_source": "152 SMs x 128 FP32 lanes x 2 x %.0f MHz"
                               % peaks.get("sm_max_mhz", 2070.0),
                "traffic": None}
    # the dominant kernel: panel products G X of the eigen-solver, counted
    # per block by the library (the last timed step's factorisation). The
    # first product of each block runs before the filter phase's events, so
    # it is left out of both the work and the time. Its arithmetic intensity
    # (2 s^2 b flops per 4 s^2 bytes of G, b/2 flop/B) is far below the
    # tensor ridge, so its roofline is bandwidth: algorithmic bytes per
    # product = G once (4 s^2) + the panel in and the panel out (4 s b each).
    rep = ctx.factor_report(full=True)
    bsub = 16 if w.k + max(8, w.k // 2) <= 16 else (
        32 if w.k + max(8, w.k // 2) <= 32 else 64)
    pflops = pbytes = 0.0
    nprod = 0
    for (s_b, L_b), prods in zip(shapes, rep["products"]):
        n_f = max(int(prods) - 1, 0)
        b_b = min(bsub, s_b)
        pflops += n_f * 2.0 * s_b * s_b * b_b
        pbytes += n_f * (4.0 * s_b * s_b + 8.0 * s_b * b_b)
        nprod += int(prods)
    t_filter = statistics.mean(phases["eigen_filter"]) * 1e-3
    tf32_peak = 0.5 * peaks.get("bf16_tflops", 1900.0)
    hbm_peak = peaks.get("hbm_gbs", 6800.0)
    p_gbs = pbytes / t_filter / 1e9 if t_filter > 0 else 0.0
    p_tf = pflops / t_filter / 1e12 if t_filter > 0 else 0.0
    roof_panel = {
        "kernel": "k_gpanel_tc", "bound": "hbm",
        "achieved": p_gbs, "peak": hbm_peak, "unit": "GB/s",
        "frac": p_gbs / hbm_peak,
        "traffic": PANEL_TRAFFIC.get(w.name),
        "peak_source": "STREAM-style copy, of %s" % peak_kind,
        "products": nprod,
        "algorithmic_bytes": pbytes,
        "tensor_tflops": p_tf,
        "tensor_frac_of_fp32_equivalent": p_tf / (tf32_peak / 3.0),
        "note": "algorithmic bytes (G once, panel in and out) of the filter "
                "phase's block products over that phase's event time; "
                "tensor_tflops counts 2 s^2 b flops per product against "
                "one third of the tf32 peak (0.5 x measured bf16), as the "
                "kernel issues three tf32 products for float32 accuracy"}
    value = world * nblocks * args.steps / (total_ms * 1e-3)
    proj_flops = 2.0 * sum(L * s * w.k for (s, L) in shapes)
    pred_flops = 2.0 * w.k * r.u_test.size
    tflops = (gflops + proj_flops + pred_flops) * args.steps / (total_ms * 1e-3) / 1e12
    gold = golden_rmse(w)
    line = {
        "metric": "block SVDs/s", "value": value, "unit": "block-SVDs/s",
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": total_ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None,
        "dtype": {"fp32": "f32", "tf32": "tf32 gram, f32",
                  "bf16": "bf16 gram, f32"}[args.precision],
        "data": "synthetic (seeded MovieLens-1M-shaped ratings, in HBM)",
        "config": {"workload": w.name, "m": w.m, "n": w.n,
                   "nnz_train": int(r.u_train.size),
                   "nnz_test": int(r.u_test.size), "p": w.p, "q": w.q,
                   "k": w.k, "precision": args.precision,
                   "gram": {1: "fp32 simt", 2: "tensor cores, exact",
                            3: "tensor cores, tf32",
                            4: "tensor cores, bf16"}.get(gram_path, "none"),
                   "l2": "flushed (256 MB write) before each step, untimed"},
        "latency_ms": {"p50": float(np.percentile(step_ms, 50)),
                       "p99": float(np.percentile(step_ms, 99))},
        "tflops": tflops,
        "phases_ms": {k: statistics.mean(v) for k, v in phases.items()},
        "rmse": rm, "rmse_oracle": gold,
        "rmse_parity": (gold is not None and abs(rm - gold) <= 1e-4),
        "roofline": roof_panel,
        "roofline_gram": {"kernel": roof["kernel"], "bound": roof["bound"],
                          "achieved": achieved, "peak": roof["peak"],
                          "unit": "TFLOP/s", "frac": achieved / roof["peak"],
                          "traffic": roof["traffic"],
                          "algorithmic_flops_per_launch": gflops,
                          "peak_source": roof["peak_source"]},
        "gpu_launches": int(launches),
        "e2e": {"value": world * nblocks * args.steps / (e2e_total * 1e-3),
                "unit": "block-SVDs/s",
                "h2d_bytes_per_step": int(12 * (r.u_train.size + r.u_test.size)
                                          + (4 * (w.m + w.n) if gridkw else 0)),
                "d2h_bytes_per_step": 8, "rmse": rm_e2e},
        "clocks": clk,
    }
    if world == 1 and not args.no_cpu_baseline:
        cores = min(os.cpu_count() or 1, nblocks)
        dt, nb = oracle_sample(w, r, cores, cores, gridkw)
        line["cpu_baseline"] = {
            "value": nb / dt, "unit": "block-SVDs/s", "cores": cores,
            "kind": "oracle",
            "sample": "oracle partition of all ratings + FP64 Jacobi SVD of "
                      "the %d smallest of %d blocks (one thread each) + their "
                      "held-out RMSE, %.1f s" % (nb, nblocks, dt)}
    rates = [float(v) for v in args.serve_rates.split(",") if v.strip()]
    if world == 1 and rates:
        line["served"] = serve_leg(rates)
    if world == 1 and not args.no_sgd and w.name == synth.MEDIUM.name:
        line["sgd"] = sgd_leg(r, w)
    print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
