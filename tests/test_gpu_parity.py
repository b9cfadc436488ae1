"""Parity of the CUDA path (through the C ABI) with the FP64 oracle.

Bars (from the method's precision, float32 on the GPU):
  * partition: counts, block means and every dense cell bit-exact;
  * singular values: relative 1e-5 on the retained top-k;
  * rank-k block reconstructions: relative Frobenius 1e-4, compared as
    matrices (so singular-vector signs and rotations inside clusters do not
    matter), for blocks whose gap (sigma_k - sigma_k+1)/sigma_k >= 1e-3;
  * held-out RMSE: |delta| <= 1e-4.
"""
import json
import math
import os

import numpy as np
import pytest

import oracle
import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_1907_07410_gb300 as bs  # noqa: E402

HERE = os.path.dirname(os.path.abspath(__file__))
SIGMA_RTOL = 1e-5
RECON_RTOL = 1e-4
RMSE_ATOL = 1e-4
GAP_MIN = 1e-3


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def gpu_run(r, p, q, k, on_device=True, ctx_kw=None, **grid):
    ctx = bs.Context(**(ctx_kw or {}))
    conv = (lambda a: dev(a)) if on_device else (lambda a: a)
    ctx.partition(r.m, r.n, conv(r.u_train), conv(r.i_train),
                  conv(r.x_train), p, q, **grid)
    ctx.factor(k)
    return ctx


def check_partition(ctx, part):
    counts, mu = ctx.block_stats()
    assert np.array_equal(counts, part.counts)
    assert np.array_equal(mu.view(np.uint32), part.mu32.view(np.uint32))
    for b in range(part.grid.p * part.grid.q):
        got = ctx.get_block(b, want_factors=False, want_dense=True)["dense"]
        want = oracle.dense_block(part, b, fp32=True)
        assert got.shape == want.shape
        assert np.array_equal(got.view(np.uint32), want.view(np.uint32)), b


def check_factors(ctx, model, blocks=None):
    worst = dict(sigma=0.0, recon=0.0)
    for b, f in model.blocks.items():
        if blocks is not None and b not in blocks:
            continue
        g = ctx.get_block(b)
        assert g["keff"] == f.keff, b
        if f.keff == 0:
            continue
        s_ref = f.sigma[:f.keff]
        floor = 1e-6 * max(f.sigma[0], 1e-30)
        err = np.abs(g["sigma"] - s_ref) / np.maximum(s_ref, floor)
        worst["sigma"] = max(worst["sigma"], float(err.max()))
        assert err.max() <= SIGMA_RTOL, (b, err.max())
        if f.gap >= GAP_MIN:
            R_ref = f.P @ f.V.T
            R_got = ctx.reconstruct(b, add_mean=False).astype(np.float64)
            nrm = np.linalg.norm(R_ref)
            if nrm > 0:
                rel = np.linalg.norm(R_got - R_ref) / nrm
                worst["recon"] = max(worst["recon"], float(rel))
                assert rel <= RECON_RTOL, (b, rel)
            # the factor pair returned by get_block rebuilds the same matrix
            R_pv = g["P"].astype(np.float64) @ g["V"].astype(np.float64).T
            assert np.linalg.norm(R_pv - R_got) <= 1e-5 * max(nrm, 1e-30) + 1e-6
    return worst


def check_rmse(ctx, model, r):
    """Held-out RMSE within 1e-4, and the predictions themselves: they are
    entries of the blocks' rank-k reconstructions, so where a block's gap is
    at least 1e-2 they are held to the reconstruction bar (relative 2-norm
    of the differences over |yhat - mu_b| of those queries, and 2e-4 for any
    single query); gap-limited blocks, whose rank-k subspace is not unique,
    only to 1e-3."""
    want = oracle.rmse(model, r.u_test, r.i_test, r.x_test)
    got = ctx.rmse(dev(r.u_test), dev(r.i_test), dev(r.x_test))
    assert abs(got - want) <= RMSE_ATOL, (got, want)
    yg = ctx.predict(dev(r.u_test), dev(r.i_test),
                     torch.zeros(r.u_test.size, dtype=torch.float32,
                                 device="cuda")).cpu().numpy()
    yo = oracle.predict(model, r.u_test, r.i_test)
    d = np.abs(yg.astype(np.float64) - yo)
    b, _, _ = model.part.grid.locate(r.u_test, r.i_test)
    gap = np.array([model.blocks[int(x)].gap for x in b])
    wide = gap >= 1e-2
    if wide.any():
        dev_part = np.linalg.norm(yo[wide] - model.part.mu64[b[wide]])
        # (a full-rank block predicts its mean at held-out cells: nothing
        # to compare relatively there)
        if dev_part > 1e-3 * np.sqrt(wide.sum()):
            assert np.linalg.norm(d[wide]) <= RECON_RTOL * dev_part
        assert d[wide].max() <= 2e-4, d[wide].max()
    assert d.max() <= 1e-3
    return got, want


# ---------------------------------------------------------------------------

def test_small_workload_end_to_end():
    w = synth.SMALL
    r = synth.generate(w)
    part = oracle.partition(w.m, w.n, r.u_train, r.i_train, r.x_train, w.p,
                            w.q)
    model = oracle.factor(part, w.k)
    ctx = gpu_run(r, w.p, w.q, w.k)
    assert ctx.last_status == bs.OK
    check_partition(ctx, part)
    check_factors(ctx, model)
    check_rmse(ctx, model, r)
    iters, conv = ctx.factor_report()
    assert conv.all()


def test_medium_workload_against_golden():
    """4 x 4 grid of 1510 x 988 blocks, k = 20: the benchmark workload."""
    w = synth.MEDIUM
    g = json.load(open(os.path.join(HERE, "golden", w.name + ".json")))
    r = synth.generate(w)
    assert r.digest() == g["digest"], "generator output differs from fixture"
    ctx = gpu_run(r, w.p, w.q, w.k)
    counts, mu = ctx.block_stats()
    assert counts.tolist() == g["counts"]
    assert np.array_equal(mu, np.array(g["mu64"]).astype(np.float32))
    for b in range(w.p * w.q):
        s = ctx.get_block(b)["sigma"]
        ref = np.array(g["sigma"][b][:w.k])
        assert np.max(np.abs(s - ref) / ref) <= SIGMA_RTOL, b
    got = ctx.rmse(dev(r.u_test), dev(r.i_test), dev(r.x_test))
    assert abs(got - g["rmse"]) <= RMSE_ATOL
    yg = ctx.predict(dev(r.u_test[:1000]), dev(r.i_test[:1000]),
                     torch.zeros(1000, dtype=torch.float32, device="cuda"))
    assert np.max(np.abs(yg.cpu().numpy() - np.array(g["yhat_first_1000"]))) < 1e-3
    # one sampled block recomputed by the oracle for the reconstruction bar
    part = oracle.partition(w.m, w.n, r.u_train, r.i_train, r.x_train, w.p,
                            w.q)
    model = oracle.factor(part, w.k, blocks=[5])
    check_factors(ctx, model, blocks=[5])


@pytest.mark.parametrize("case", [
    # (m, n, p, q, k, nnz_train, nnz_test)
    (30, 20, 2, 2, 4, 250, 60),        # s = 10 <= 16: direct eigen path
    (100, 90, 2, 2, 10, 3000, 500),    # s = 45, subspace width 32
    (1000, 777, 3, 5, 12, 40000, 4000),  # ragged tails on both sides
    (257, 129, 1, 1, 20, 9000, 900),   # one block (global truncated SVD)
    (300, 1, 4, 1, 3, 200, 40),        # single item column: s = 1
    (9, 400, 9, 2, 2, 1200, 100),      # one-user block rows
    (80, 60, 2, 3, 40, 2500, 300),     # k >= s in some blocks
])
def test_shapes_and_ragged_edges(case):
    m, n, p, q, k, ntr, nte = case
    r = synth.random_ratings(17 + m, m, n, ntr, nte)
    part = oracle.partition(m, n, r.u_train, r.i_train, r.x_train, p, q)
    model = oracle.factor(part, k)
    ctx = gpu_run(r, p, q, k)
    check_partition(ctx, part)
    check_factors(ctx, model)
    check_rmse(ctx, model, r)


def test_k_zero_and_full_rank_predict_block_means():
    r = synth.random_ratings(5, 60, 50, 900, 200)
    part = oracle.partition(60, 50, r.u_train, r.i_train, r.x_train, 2, 2)
    b, _, _ = part.grid.locate(r.u_test, r.i_test)
    for k in (0, 56):
        ctx = gpu_run(r, 2, 2, k)
        y = ctx.predict(r.u_test, r.i_test)
        assert np.max(np.abs(y - part.mu32[b])) <= 1e-4, k


def test_empty_and_constant_blocks():
    # ratings only in block 0; block 3 has one constant value (B = 0)
    u = np.array([0, 1, 2, 0, 1, 7, 8, 9], np.int32)
    i = np.array([0, 1, 2, 3, 0, 7, 8, 9], np.int32)
    x = np.array([1, 5, 3, 2, 4, 4, 4, 4], np.float32)
    part = oracle.partition(10, 10, u, i, x, 2, 2)
    assert part.counts.tolist() == [5, 0, 0, 3]
    ctx = bs.Context()
    ctx.partition(10, 10, u, i, x, 2, 2)
    assert ctx.factor(3) == bs.OK
    check_partition(ctx, part)
    model = oracle.factor(part, 3)
    uq = np.array([5, 0, 9, 6], np.int32)    # blocks 3, 1 (empty), 2, 3
    iq = np.array([9, 9, 0, 6], np.int32)
    yg = ctx.predict(uq, iq)
    yo = oracle.predict(model, uq, iq)
    assert np.max(np.abs(yg - yo)) < 1e-5
    assert yg[1] == yg[2] == np.float32(part.global_mean)
    assert yg[0] == yg[3] == 4.0


def test_explicit_bounds_and_permutations():
    rng = np.random.default_rng(3)
    m, n = 500, 300
    r = synth.random_ratings(8, m, n, 20000, 2000)
    rb = np.array([0, 37, 37, 300, 500], np.int64)     # includes an empty row
    cb = np.array([0, 100, 101, 300], np.int64)
    rp = rng.permutation(m).astype(np.int32)
    cp = rng.permutation(n).astype(np.int32)
    part = oracle.partition(m, n, r.u_train, r.i_train, r.x_train, 4, 3,
                            rb, cb, rp, cp)
    model = oracle.factor(part, 8)
    ctx = gpu_run(r, 4, 3, 8, row_bounds=rb, col_bounds=cb,
                  row_perm=dev(rp), col_perm=cp)
    check_partition(ctx, part)
    check_factors(ctx, model)
    check_rmse(ctx, model, r)


def test_host_and_device_inputs_agree():
    w = synth.SMALL
    r = synth.generate(w)
    a = gpu_run(r, w.p, w.q, w.k, on_device=True)
    b = gpu_run(r, w.p, w.q, w.k, on_device=False)
    ra = a.rmse(r.u_test, r.i_test, r.x_test)
    rb_ = b.rmse(dev(r.u_test), dev(r.i_test), dev(r.x_test))
    assert ra == rb_
    assert np.array_equal(a.predict(r.u_test, r.i_test),
                          b.predict(r.u_test, r.i_test))


def test_runs_are_bit_identical():
    w = synth.SMALL
    r = synth.generate(w)
    out = []
    for _ in range(2):
        c = gpu_run(r, w.p, w.q, w.k)
        out.append((c.rmse(r.u_test, r.i_test, r.x_test),
                    c.get_block(1)["sigma"].tobytes(),
                    c.predict(r.u_test, r.i_test).tobytes()))
    assert out[0] == out[1]


def test_clamp_option():
    w = synth.SMALL
    r = synth.generate(w)
    raw = gpu_run(r, w.p, w.q, w.k).predict(r.u_test, r.i_test)
    clp = gpu_run(r, w.p, w.q, w.k, ctx_kw=dict(clamp=1)).predict(
        r.u_test, r.i_test)
    assert np.array_equal(clp, np.clip(raw, 1.0, 5.0))


def test_bad_inputs_are_rejected():
    ctx = bs.Context()
    u = np.array([0, 5], np.int32)
    i = np.array([0, 1], np.int32)
    x = np.array([1.0, 2.0], np.float32)
    with pytest.raises(bs.BsvdError) as e:
        ctx.partition(5, 5, u, i, x, 1, 1)
    assert e.value.status == bs.EINVAL
    with pytest.raises(bs.BsvdError) as e:
        ctx.partition(5, 5, u[:1], i[:1], np.array([np.nan], np.float32), 1, 1)
    assert e.value.status == bs.EINVAL
    with pytest.raises(bs.BsvdError) as e:
        ctx.factor(3)
    assert e.value.status == bs.ESTATE
    ctx.partition(5, 5, u[:1], i[:1], x[:1], 1, 1)
    ctx.factor(1)
    with pytest.raises(bs.BsvdError) as e:
        ctx.predict(np.array([7], np.int32), np.array([0], np.int32))
    assert e.value.status == bs.EINVAL
    with pytest.raises(bs.BsvdError) as e:
        ctx.partition(5, 5, u[:1], i[:1], x[:1], 1, 1,
                      row_perm=np.array([0, 1, 2, 3, 3], np.int32))
    assert e.value.status == bs.EINVAL


@pytest.mark.parametrize("path", [1, 2])
def test_gram_paths_match_oracle(path):
    """FP32 SIMT Gram (path 1) and exact tensor-core Gram (path 2)."""
    w = synth.SMALL
    r = synth.generate(w)
    part = oracle.partition(w.m, w.n, r.u_train, r.i_train, r.x_train, w.p,
                            w.q)
    model = oracle.factor(part, w.k)
    ctx = gpu_run(r, w.p, w.q, w.k, ctx_kw=dict(gram_path=path))
    assert ctx.gram_path() == path
    check_factors(ctx, model)
    check_rmse(ctx, model, r)


def test_default_gram_path_uses_tensor_cores_on_integer_ratings():
    w = synth.SMALL
    r = synth.generate(w)
    ctx = gpu_run(r, w.p, w.q, w.k)
    assert ctx.gram_path() == 2


def test_non_integer_ratings_fall_back_to_simt_gram():
    r = synth.random_ratings(21, 300, 200, 6000, 600)
    r.x_train = (r.x_train + np.float32(0.37)).astype(np.float32)
    r.x_test = (r.x_test + np.float32(0.37)).astype(np.float32)
    part = oracle.partition(300, 200, r.u_train, r.i_train, r.x_train, 2, 2)
    model = oracle.factor(part, 6)
    ctx = gpu_run(r, 2, 2, 6)
    assert ctx.gram_path() == 1
    check_factors(ctx, model)
    check_rmse(ctx, model, r)
    forced = bs.Context(gram_path=2)
    forced.partition(300, 200, r.u_train, r.i_train, r.x_train, 2, 2)
    with pytest.raises(bs.BsvdError) as e:
        forced.factor(6)
    assert e.value.status == bs.EINVAL


@pytest.mark.parametrize("panel", [0, 1])
def test_panel_paths_match_oracle(panel):
    """Eigen-solver panel products on the tensor cores (three tf32 passes,
    panel_path 0) and on the FP32 SIMT pipes (panel_path 1), against the
    oracle on the small workload."""
    w = synth.SMALL
    r = synth.generate(w)
    part = oracle.partition(w.m, w.n, r.u_train, r.i_train, r.x_train, w.p,
                            w.q)
    model = oracle.factor(part, w.k)
    ctx = gpu_run(r, w.p, w.q, w.k, ctx_kw=dict(panel_path=panel))
    check_factors(ctx, model)
    check_rmse(ctx, model, r)


@pytest.mark.parametrize("k", [6, 20, 40])
def test_panel_paths_agree_on_medium(k):
    """Both panel paths on the medium matrix, for subspace widths 16, 32 and
    64: singular values within 2e-6 relative, RMSE within 1e-5."""
    w = synth.MEDIUM
    r = synth.generate(w)
    out = []
    for panel in (0, 1):
        ctx = gpu_run(r, w.p, w.q, k, ctx_kw=dict(panel_path=panel))
        assert ctx.last_status == bs.OK
        sig = [ctx.get_block(b)["sigma"] for b in range(w.p * w.q)]
        out.append((sig, ctx.rmse(dev(r.u_test), dev(r.i_test),
                                  dev(r.x_test))))
    for a, b in zip(out[0][0], out[1][0]):
        assert np.max(np.abs(a - b) / b) <= 2e-6
    assert abs(out[0][1] - out[1][1]) <= 1e-5


def test_sign_convention_matches_oracle():
    """Each (P_j, V_j) pair is flipped so that the item-side vector's
    largest-|.| entry is positive; columns with well-separated singular
    values then equal the oracle's canonical vectors."""
    w = synth.SMALL
    r = synth.generate(w)
    part = oracle.partition(w.m, w.n, r.u_train, r.i_train, r.x_train, w.p,
                            w.q)
    model = oracle.factor(part, w.k)
    ctx = gpu_run(r, w.p, w.q, w.k)
    checked = 0
    for b, f in model.blocks.items():
        g = ctx.get_block(b)
        V = g["V"].astype(np.float64)
        for j in range(f.keff):
            col = V[:, j]
            top = int(np.argmax(np.abs(col)))
            assert col[top] > 0, (b, j)
            s = f.sigma
            sep = min(abs(s[j] - s[j - 1]) if j > 0 else np.inf,
                      abs(s[j] - s[j + 1]) if j + 1 < s.size else np.inf)
            if sep >= 1e-2 * s[0]:
                assert np.max(np.abs(col - f.V[:, j])) <= 1e-3, (b, j)
                checked += 1
    assert checked >= 8


@pytest.mark.parametrize("workload", [synth.SMALL, synth.MEDIUM_8x8])
def test_device_driven_loop_matches_host_loop(workload):
    """The eigen loop captured in one CUDA graph (a conditional WHILE node
    that a kernel ends) gives bit-identical factors to the host-driven loop:
    loop = 0 runs the host loop on a layout's first factorisation and the
    graph from the second on; loop = 2 always the graph; loop = 1 never."""
    w = workload
    r = synth.generate(w)

    def run(loop, times):
        ctx = bs.Context(loop=loop)
        forms = []
        for _ in range(times):
            ctx.partition(r.m, r.n, dev(r.u_train), dev(r.i_train),
                          dev(r.x_train), w.p, w.q)
            assert ctx.factor(w.k) == bs.OK
            forms.append(ctx.loop_form())
        sig = [ctx.get_block(b)["sigma"] for b in range(w.p * w.q)]
        y = ctx.predict(r.u_test, r.i_test)
        rm = ctx.rmse(r.u_test, r.i_test, r.x_test)
        iters, _ = ctx.factor_report()
        ctx.close()
        return forms, sig, y, rm, iters

    f1, s1, y1, rm1, it1 = run(1, 1)
    f0, s0, y0, rm0, it0 = run(0, 3)
    f2, s2, y2, rm2, it2 = run(2, 1)
    assert f1 == [1] and f0 == [1, 2, 2] and f2 == [2]
    for a, b in zip(s1, s0):
        assert np.array_equal(a, b)
    for a, b in zip(s1, s2):
        assert np.array_equal(a, b)
    assert np.array_equal(y1, y0) and np.array_equal(y1, y2)
    assert rm1 == rm0 == rm2
    assert np.array_equal(it1, it0) and np.array_equal(it1, it2)


def test_reconstruction_on_tensor_cores_matches_factors():
    """bsvd_reconstruct (128 x 128 tiles, three tf32 products of the factors'
    hi and lo parts) against mu + P V^T computed in float64 from the block's
    own factors, element by element: blocks of both orientations with
    ragged tails across several tiles, host and device outputs, with and
    without the mean. (check_factors holds reconstructions to the
    oracle's.)"""
    w = synth.UNEVEN
    r = synth.generate(w)
    ctx = bs.Context()
    kw = ctx.quantile_grid(w.m, w.n, dev(r.u_train), dev(r.i_train), w.p, w.q)
    ctx.partition(w.m, w.n, dev(r.u_train), dev(r.i_train), dev(r.x_train),
                  w.p, w.q, **kw)
    assert ctx.factor(w.k) == bs.OK
    shapes = [(b, ctx.get_block(b, want_factors=False)) for b in range(w.p * w.q)]
    tall = [b for b, g in shapes if g["mb"] > g["nb"] and g["mb"] % 128]
    wide = [b for b, g in shapes if g["mb"] < g["nb"] and g["nb"] % 128]
    big = max(range(w.p * w.q), key=lambda b: shapes[b][1]["mb"] * shapes[b][1]["nb"])
    picked = sorted({big, tall[0], wide[0]} if tall and wide else {big})
    assert len(picked) >= 2
    for b in picked:
        g = ctx.get_block(b)
        P = g["P"].astype(np.float64)
        V = g["V"].astype(np.float64)
        ref = P @ V.T
        scale = np.abs(P) @ np.abs(V).T      # the dot products' magnitude
        got0 = ctx.reconstruct(b, add_mean=False).astype(np.float64)
        assert got0.shape == (g["mb"], g["nb"])
        assert np.all(np.abs(got0 - ref) <= 4e-6 * scale + 1e-7), b
        got1 = ctx.reconstruct(b, add_mean=True).astype(np.float64)
        mu = float(np.float32(g["mu"]))
        assert np.all(np.abs(got1 - (ref + mu)) <=
                      4e-6 * scale + 1e-6 * abs(mu) + 1e-7), b
        out = torch.full((g["mb"] * g["nb"],), float("nan"),
                         dtype=torch.float32, device="cuda")
        ctx.reconstruct(b, add_mean=True, out=out)
        assert np.array_equal(out.cpu().numpy().reshape(g["mb"], g["nb"]),
                              got1.astype(np.float32)), b
    with pytest.raises(ValueError):
        ctx.reconstruct(picked[0], out=torch.zeros(3, device="cuda"))
    ctx.close()
