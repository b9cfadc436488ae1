"""The served form on the device: requests of mixed shapes and ranks laid
out block-diagonally (bsvd_partition_diag) and factorised in one
bsvd_factor_ks call. Each request's result in a batch must match the same
request run alone and the FP64 oracle run on that request's ratings (a 1 x 1
grid). Bars as on the grid path: singular values relative 1e-5, rank-k
reconstruction relative Frobenius 1e-4 and predictions within 1e-3 where the
block's gap is at least 1e-3; batch against alone within 1e-4."""
import numpy as np
import pytest

import oracle
import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_1907_07410_gb300 as bs  # noqa: E402
from paper_1907_07410_gb300 import serve  # noqa: E402


def requests(seed, count, **kw):
    return [serve.Request(d["m"], d["n"], d["k"], d["r"], d["c"], d["x"],
                          d["qr"], d["qc"])
            for d in synth.served_requests(seed, count, dense=False, **kw)]


def edge_requests():
    """A full-rank tiny block, a single row, a k=0 request and a block with
    every value equal (zero after centring)."""
    rng = np.random.default_rng(11)
    out = []
    d = rng.integers(1, 6, size=(5, 3)).astype(np.float32)
    out.append(serve.Request.from_dense(d, 10, np.array([0, 4], np.int32),
                             np.array([2, 1], np.int32)))
    d = np.zeros((1, 40), np.float32)
    d[0, ::3] = rng.integers(1, 6, size=14)
    out.append(serve.Request.from_dense(d, 4, np.array([0], np.int32),
                             np.array([1], np.int32)))
    d = rng.integers(1, 6, size=(70, 90)).astype(np.float32)
    d[rng.random(d.shape) < 0.5] = 0
    out.append(serve.Request.from_dense(d, 0, np.array([3, 5], np.int32),
                             np.array([7, 8], np.int32)))
    d = np.zeros((60, 50), np.float32)
    d[rng.random(d.shape) < 0.2] = 4.0
    out.append(serve.Request.from_dense(d, 20, np.array([1], np.int32),
                             np.array([2], np.int32)))
    return out


def oracle_request(req):
    part = oracle.partition(req.m, req.n, req.r, req.c, req.x, 1, 1)
    model = oracle.factor(part, req.k, threads=1)
    return model, oracle.predict(model, req.qr, req.qc)


def test_batch_matches_alone_and_oracle():
    reqs = requests(5, 8, rows=(128, 1200), cols=(64, 500)) + edge_requests()
    ctx = bs.Context()
    got = serve.run_batch(ctx, reqs)
    assert ctx.nblocks == len(reqs)
    for b, req in enumerate(reqs):
        alone = serve.run_batch(bs.Context(), [req])[0]
        assert np.max(np.abs(got[b] - alone), initial=0) <= 1e-4, b
        info = ctx.get_block(b)
        m, n = req.m, req.n
        assert (info["mb"], info["nb"]) == (m, n)
        model, yref = oracle_request(req)
        f = model.blocks[0]
        assert len(info["sigma"]) == f.keff == min(req.k, m, n)
        if f.keff:
            ref = f.sigma[:f.keff]
            live = ref > 1e-6 * max(ref[0], 1e-30)
            rel = np.abs(info["sigma"][live] - ref[live]) / ref[live]
            assert np.max(rel, initial=0) <= 1e-5, b
        if f.gap >= 1e-3 and f.keff and f.sigma[0] > 0:
            R_ref = f.P @ f.V.T
            R_got = ctx.reconstruct(b, add_mean=False).astype(np.float64)
            rel = np.linalg.norm(R_got - R_ref) / max(np.linalg.norm(R_ref),
                                                       1e-30)
            assert rel <= 1e-4, (b, rel)
            assert np.max(np.abs(got[b] - yref)) <= 1e-3, b
        if f.keff == 0 or np.all(f.sigma == 0):
            # no factor to add: the prediction is the block mean
            assert np.allclose(got[b], yref, atol=1e-6), b


def test_per_block_rank_reaches_each_block():
    reqs = requests(6, 5, rows=(100, 400), cols=(64, 300), ks=(4, 12, 40))
    ctx = bs.Context()
    serve.run_batch(ctx, reqs)
    for b, req in enumerate(reqs):
        s = ctx.get_block(b)["sigma"]
        assert len(s) == min(req.k, req.m, req.n)
        assert np.all(np.diff(s) <= 0)


def test_off_diagonal_rating_is_rejected():
    ctx = bs.Context()
    rb = np.array([0, 4, 8], np.int64)
    cb = np.array([0, 3, 6], np.int64)
    u = np.array([0, 5, 1], np.int32)
    i = np.array([0, 4, 4], np.int32)      # (1, 4) lies in block (0, 1)
    x = np.array([3, 4, 5], np.float32)
    with pytest.raises(bs.BsvdError) as e:
        ctx.partition_diag(rb, cb, u, i, x)
    assert e.value.status == bs.EINVAL


def test_server_results_match_alone():
    reqs = requests(7, 24, rows=(128, 2048), cols=(64, 1024))
    with serve.Server(workers=3, max_batch=6, hbm_budget=8e9) as srv:
        futs = [srv.submit(r) for r in reqs]
        res = [f.result(timeout=600) for f in futs]
    assert max(len(ids) for ids, _ in srv.batches) > 1
    assert srv.max_held <= srv.budget
    for req, r in zip(reqs, res):
        alone = serve.run_batch(bs.Context(), [req])[0]
        assert np.max(np.abs(r.yhat - alone)) <= 1e-4, req.rid
    pct = serve.latency_percentiles(res)
    assert 0 < pct["p50_ms"] <= pct["p99_ms"]


def test_server_under_a_tight_budget():
    """A budget of about two requests forces small batches and context
    resets; every result is still right."""
    reqs = requests(8, 10, rows=(256, 1024), cols=(128, 512))
    fps = [serve.footprint(r.m, r.n, r.nnz, len(r.qr)) for r in reqs]
    budget = max(fps) * 2
    with serve.Server(workers=3, max_batch=8, hbm_budget=budget) as srv:
        res = [f.result(timeout=600) for f in [srv.submit(r) for r in reqs]]
    assert srv.max_held <= budget
    for req, r in zip(reqs, res):
        alone = serve.run_batch(bs.Context(), [req])[0]
        assert np.max(np.abs(r.yhat - alone)) <= 1e-4


def test_served_pool_against_oracle_fixture():
    """The served form's request pool through the server; the requests the
    oracle fixture covers (Jacobi work m n min(m, n) <= 2e9) against its
    singular values, predictions and held-out RMSE."""
    import json
    import os
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden",
                        "served-pool-%d.json" % synth.SERVED_POOL_SIZE)
    g = json.load(open(path))
    raw = synth.served_requests(synth.SERVED_POOL_SEED,
                                synth.SERVED_POOL_SIZE, dense=False)
    pool = [serve.Request(d["m"], d["n"], d["k"], d["r"], d["c"], d["x"],
                          d["qr"], d["qc"]) for d in raw]
    with serve.Server(workers=4, max_batch=16, hbm_budget=40e9) as srv:
        res = [f.result(timeout=600) for f in [srv.submit(q) for q in pool]]
    err = []
    ctx = bs.Context()
    for ref in g["requests"]:
        j = ref["index"]
        assert (pool[j].m, pool[j].n, pool[j].k) == (ref["m"], ref["n"],
                                                     ref["k"])
        serve.run_batch(ctx, [pool[j]])
        s = ctx.get_block(0)["sigma"]
        sref = np.array(ref["sigma"][:len(s)])
        assert np.max(np.abs(s - sref) / sref) <= 1e-5, j
        if ref["gap"] >= 1e-3:
            assert np.max(np.abs(res[j].yhat - np.array(ref["yhat"]))) <= 1e-3
        err.append(res[j].yhat.astype(np.float64) - raw[j]["qy"])
    got = float(np.sqrt(np.mean(np.concatenate(err) ** 2)))
    print("served pool subset rmse %.9f oracle %.9f" % (got, g["rmse"]))
    assert abs(got - g["rmse"]) <= 1e-4
