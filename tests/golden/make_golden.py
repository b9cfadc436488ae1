"""Write the oracle's results for the synthetic workloads to JSON fixtures
(``served`` selects the served form's request pool; the full-size uneven
workload, large-480189x17770-32x8-k40, takes about half an hour).

Calls only ``oracle`` and the seeded generator ``synth``: no stored value
here comes from the CUDA library. Run from the repository root:

    python tests/golden/make_golden.py [workload names | served]
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
    grid = {}
    if w.grid == "quantile":
        rp, rb = oracle.activity_quantile_cut(r.u_train, w.m, w.p)
        cp, cb = oracle.activity_quantile_cut(r.i_train, w.n, w.q)
        grid = dict(row_bounds=rb, col_bounds=cb, row_perm=rp, col_perm=cp)
    part = oracle.partition(w.m, w.n, r.u_train, r.i_train, r.x_train, w.p,
                            w.q, **grid)
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
        row_bounds=part.grid.row_bounds.tolist(),
        col_bounds=part.grid.col_bounds.tolist(),
        yhat_first_1000=yhat[:1000].tolist(),
        oracle_seconds=time.time() - t0,
    )
    return out


# held-out ratings whose predictions the large fixture stores
LARGE_QUERY_SAMPLE = 10_000
LARGE_QUERY_SEED = 31


def large_golden(w: synth.Workload) -> dict:
    """The full-size uneven workload. Every block through the oracle's FP64
    Gram route (the Jacobi routine would take hours on the largest
    blocks); the 4 smallest and 2 median blocks (by cells) also through
    Jacobi, which must agree. Stores sigma and the gap of every block, the
    held-out RMSE over all held-out ratings and the predictions of a seeded
    sample of them."""
    import concurrent.futures as cf
    r = synth.generate(w)
    t0 = time.time()
    rp, rb = oracle.activity_quantile_cut(r.u_train, w.m, w.p)
    cp, cb = oracle.activity_quantile_cut(r.i_train, w.n, w.q)
    part = oracle.partition(w.m, w.n, r.u_train, r.i_train, r.x_train, w.p,
                            w.q, rb, cb, rp, cp)
    t_part = time.time() - t0
    print("partition %.1f s" % t_part, flush=True)
    nb = w.p * w.q
    threads = os.cpu_count() or 1
    # largest blocks first, so the pool ends evenly
    cost = [min(part.grid.block_shape(b)) ** 2 * max(part.grid.block_shape(b))
            for b in range(nb)]
    order = sorted(range(nb), key=lambda b: -cost[b])
    with cf.ThreadPoolExecutor(max_workers=threads) as ex:
        fs = dict(zip(order, ex.map(
            lambda b: oracle.factor_block_gram(part, b, w.k), order)))
    model = oracle.Model(part, w.k, fs)
    t_gram = time.time() - t0 - t_part
    print("gram route %.1f s" % t_gram, flush=True)
    rmse = oracle.rmse(model, r.u_test, r.i_test, r.x_test)
    rng = np.random.Generator(np.random.PCG64(LARGE_QUERY_SEED))
    qidx = np.sort(rng.choice(r.u_test.size, LARGE_QUERY_SAMPLE,
                              replace=False))
    yhat = oracle.predict(model, r.u_test[qidx], r.i_test[qidx])
    qblock, _, _ = part.grid.locate(r.u_test[qidx], r.i_test[qidx])
    cells = [int(np.prod(part.grid.block_shape(b))) for b in range(nb)]
    by_cells = [int(b) for b in np.argsort(cells, kind="stable")]
    jac_ids = by_cells[:4] + by_cells[nb // 2 - 1:nb // 2 + 1]
    jac = oracle.factor(part, w.k, blocks=jac_ids, threads=threads)
    for b in jac_ids:
        fj, fg = jac.blocks[b], fs[b]
        n = min(fj.keff + 1, fj.sigma.size)
        err = np.max(np.abs(fj.sigma[:n] - fg.sigma[:n])) / fj.sigma[0]
        assert err <= 1e-11, ("Gram and Jacobi routes disagree", b, err)
    return dict(
        workload=w.name, digest=r.digest(), k=w.k, p=w.p, q=w.q,
        route="FP64 Gram + LAPACK symmetric eigensolver (factor_block_gram)",
        row_bounds=part.grid.row_bounds.tolist(),
        col_bounds=part.grid.col_bounds.tolist(),
        shapes=[list(part.grid.block_shape(b)) for b in range(nb)],
        counts=part.counts.tolist(), mu64=part.mu64.tolist(),
        sigma=[fs[b].sigma[:w.k + 1].tolist() for b in range(nb)],
        gap=[fs[b].gap for b in range(nb)],
        rmse=rmse, query_seed=LARGE_QUERY_SEED, query_idx=qidx.tolist(),
        yhat_sample=yhat.tolist(), query_block=qblock.tolist(),
        jacobi_blocks=jac_ids,
        sigma_jacobi=[jac.blocks[b].sigma[:w.k + 1].tolist()
                      for b in jac_ids],
        oracle_seconds=dict(partition=t_part, gram=t_gram,
                            total=time.time() - t0),
    )


SERVED_MAX_COST = 2e9   # m_b * n_b * min(m_b, n_b): the oracle's Jacobi work


def served_golden() -> dict:
    """The oracle on the cheaper requests of the served pool (each a 1 x 1
    grid): predictions for its held-out queries, top singular values and
    the RMSE over those queries."""
    import concurrent.futures as cf
    pool = synth.served_requests(synth.SERVED_POOL_SEED,
                                 synth.SERVED_POOL_SIZE, dense=False)
    ids = [j for j, d in enumerate(pool)
           if d["m"] * d["n"] * min(d["m"], d["n"]) <= SERVED_MAX_COST]
    t0 = time.time()

    def one(j):
        d = pool[j]
        part = oracle.partition(d["m"], d["n"], d["r"], d["c"], d["x"], 1, 1)
        model = oracle.factor(part, d["k"], threads=1)
        f = model.blocks[0]
        return dict(index=j, m=d["m"], n=d["n"], k=d["k"], nnz=len(d["r"]),
                    mu64=float(part.mu64[0]),
                    sigma=f.sigma[:d["k"] + 1].tolist(), gap=f.gap,
                    yhat=oracle.predict(model, d["qr"], d["qc"]).tolist())
    with cf.ThreadPoolExecutor(max_workers=os.cpu_count() or 1) as ex:
        reqs = list(ex.map(one, ids))
    err = np.concatenate([np.array(q["yhat"]) - pool[q["index"]]["qy"]
                          for q in reqs])
    return dict(workload="served-pool-%d" % synth.SERVED_POOL_SIZE,
                seed=synth.SERVED_POOL_SEED, max_cost=SERVED_MAX_COST,
                requests=reqs, rmse=float(np.sqrt(np.mean(err ** 2))),
                oracle_seconds=time.time() - t0)


def main():
    names = sys.argv[1:] or [synth.MEDIUM.name]
    for name in names:
        if name == "served":
            g = served_golden()
            path = os.path.join(HERE, g["workload"] + ".json")
            with open(path, "w") as f:
                json.dump(g, f, indent=1)
            print(path, "rmse", g["rmse"], "%.1fs" % g["oracle_seconds"])
            continue
        w = synth.WORKLOADS[name]
        big = w.nnz >= 10_000_000
        g = large_golden(w) if big else golden(w)
        path = os.path.join(HERE, w.name + ".json")
        with open(path, "w") as f:
            json.dump(g, f, indent=None if big else 1)
        secs = g["oracle_seconds"]
        print(path, "rmse", g["rmse"], "%.1fs" % (
            secs["total"] if isinstance(secs, dict) else secs))


if __name__ == "__main__":
    main()
