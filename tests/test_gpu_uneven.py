"""The batched uneven form against the FP64 oracle's fixtures: a long-tailed
20,000 x 3,000 matrix cut at activity quantiles into an 8 x 4 grid (every
block), and the full 480,189 x 17,770 matrix on its 32 x 8 grid (every
block's singular values, the held-out RMSE and sampled predictions), with
the float32 (exact Gram) and BF16 forms."""
import json
import os

import numpy as np
import pytest

import oracle
import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_1907_07410_gb300 as bs  # noqa: E402
from paper_1907_07410_gb300 import grid  # noqa: E402

HERE = os.path.dirname(os.path.abspath(__file__))


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def run(w, r, kw):
    ctx = bs.Context()
    ctx.partition(w.m, w.n, dev(r.u_train), dev(r.i_train), dev(r.x_train),
                  w.p, w.q, row_bounds=kw["row_bounds"],
                  col_bounds=kw["col_bounds"], row_perm=dev(kw["row_perm"]),
                  col_perm=dev(kw["col_perm"]))
    status = ctx.factor(w.k)
    return ctx, status


def test_uneven_quantile_grid_against_golden():
    w = synth.UNEVEN
    g = json.load(open(os.path.join(HERE, "golden", w.name + ".json")))
    r = synth.generate(w)
    assert r.digest() == g["digest"]
    kw = grid.quantile_grid(r.u_train, r.i_train, w.m, w.n, w.p, w.q)
    assert kw["row_bounds"].tolist() == g["row_bounds"]
    assert kw["col_bounds"].tolist() == g["col_bounds"]
    ctx, status = run(w, r, kw)
    assert status == bs.OK
    counts, mu = ctx.block_stats()
    assert counts.tolist() == g["counts"]
    assert np.array_equal(mu, np.array(g["mu64"]).astype(np.float32))
    for b in range(w.p * w.q):
        s = ctx.get_block(b)["sigma"]
        ref = np.array(g["sigma"][b][:len(s)])
        assert np.max(np.abs(s - ref) / ref) <= 1e-5, b
    got = ctx.rmse(dev(r.u_test), dev(r.i_test), dev(r.x_test))
    assert abs(got - g["rmse"]) <= 1e-4


LARGE_FIXTURE = os.path.join(HERE, "golden", synth.LARGE.name + ".json")
# (precision, sigma bar, reconstruction bar). Sampled predictions stand in
# for the blocks' rank-k reconstructions: over the queries of blocks whose
# gap is at least 1e-2, |yhat - yhat_oracle| relative to |yhat_oracle -
# mu_b| (2-norms over the sample) is held to the reconstruction bar, and
# every such query to that bar in absolute terms times 2 (predictions are
# ratings of 1-5 whose rank-k part stays below 2 in magnitude).
LARGE_FORMS = [(bs.FP32, 1e-5, 1e-4), (bs.BF16, 2e-3, 5e-3)]


@pytest.fixture(scope="module")
def large():
    w = synth.LARGE
    g = json.load(open(LARGE_FIXTURE))
    r = synth.generate(w)
    assert r.digest() == g["digest"], "generator output differs from fixture"
    return w, r, g


def test_full_size_quantile_grid(large):
    """The library's activity-quantile cut of the 480,189 x 17,770 matrix
    equals the oracle's bounds."""
    w, r, g = large
    kw = grid.quantile_grid(dev(r.u_train), dev(r.i_train), w.m, w.n, w.p,
                            w.q)
    assert kw["row_bounds"].tolist() == g["row_bounds"]
    assert kw["col_bounds"].tolist() == g["col_bounds"]


@pytest.mark.parametrize("precision,sig_bar,recon_bar", LARGE_FORMS)
def test_full_size_batched_against_oracle(large, precision, sig_bar,
                                          recon_bar):
    """The full batched workload (256 uneven blocks from 177 x 132 to
    92,840 x 4,619, k = 40) in the launch configuration the benchmark times,
    against the oracle's fixture: bit-exact counts and means, the retained
    singular values of every block, the held-out RMSE over all 10,048,050
    held-out ratings, and the predictions of a seeded sample of 10,000 of
    them."""
    w, r, g = large
    u, i = dev(r.u_train), dev(r.i_train)
    ctx = bs.Context(precision=precision)
    kw = ctx.quantile_grid(w.m, w.n, u, i, w.p, w.q)
    ctx.partition(w.m, w.n, u, i, dev(r.x_train), w.p, w.q, **kw)
    assert ctx.factor(w.k) == bs.OK
    counts, mu = ctx.block_stats()
    assert counts.tolist() == g["counts"]
    assert np.array_equal(mu, np.array(g["mu64"]).astype(np.float32))
    worst = 0.0
    for b in range(w.p * w.q):
        s = ctx.get_block(b)["sigma"]
        ref = np.array(g["sigma"][b][:len(s)])
        worst = max(worst, float(np.max(np.abs(s - ref) / ref)))
    rm = ctx.rmse(dev(r.u_test), dev(r.i_test), dev(r.x_test))
    q = np.array(g["query_idx"])
    yg = ctx.predict(r.u_test[q], r.i_test[q]).astype(np.float64)
    yo = np.array(g["yhat_sample"])
    qb = np.array(g["query_block"])
    gap = np.array(g["gap"], dtype=np.float64)[qb]
    mu_q = np.array(g["mu64"])[qb]
    d = np.abs(yg - yo)
    wide = gap >= 1e-2
    rel = np.linalg.norm(d[wide]) / np.linalg.norm(yo[wide] - mu_q[wide])
    print("precision %d: worst sigma rel %.2e, rmse %.9f (oracle %.9f), "
          "max |dy| %.2e; gap >= 1e-2 (%d queries): max |dy| %.2e, "
          "relative %.2e" % (precision, worst, rm, g["rmse"], d.max(),
                             wide.sum(), d[wide].max(), rel))
    assert worst <= sig_bar
    assert abs(rm - g["rmse"]) <= 1e-4
    assert rel <= recon_bar
    assert d[wide].max() <= 2 * recon_bar
    ctx.close()
