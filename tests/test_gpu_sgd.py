"""The paper's own method, blocked SGD (Algorithms 1-2), on the device
against the sequential FP64 oracle. Both sides evaluate every update in the
same order with one rounding per operation, so the bar is bit equality of
the parameters after a fixed number of epochs; the training-RMSE history
is summed in different orders and must agree to 1e-12 relative."""
import numpy as np
import pytest

import oracle
import synth
from oracle import sgd as osgd

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_1907_07410_gb300 as bs  # noqa: E402
from paper_1907_07410_gb300 import grid as qgrid  # noqa: E402


def run_both(r, p, q, k, steps, delta=-1e300, grid_kw=None, rates=None,
             seed=13, on_device=False, f32=False):
    P0, Q0 = synth.sgd_start(r.m, r.n, k, seed)
    grid_kw = grid_kw or {}
    ctx = bs.Context()
    conv = (lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()) \
        if on_device else (lambda a: a)
    gk = dict(grid_kw)
    for key in ("row_perm", "col_perm"):
        if gk.get(key) is not None:
            gk[key] = conv(np.asarray(gk[key], np.int32))
    ctx.partition(r.m, r.n, conv(r.u_train), conv(r.i_train), conv(r.x_train),
                  p, q, **gk)
    ctx.sgd_prepare(conv(r.u_train), conv(r.i_train), conv(r.x_train))
    rk = dict(vars(rates)) if rates else {}
    if f32:
        rk["precision"] = bs.SGD_FP32
    hist, ran = ctx.sgd_train(conv(P0), conv(Q0), max_steps=steps,
                              delta=delta, **rk)
    g = oracle.make_grid(r.m, r.n, p, q, **grid_kw)
    ref = osgd.train(g, r.u_train, r.i_train, r.x_train, P0, Q0, steps,
                     rates=rates, delta=delta,
                     dtype=np.float32 if f32 else np.float64)
    return ctx, hist, ran, ref


def assert_same(ctx, hist, ran, ref):
    P, Q, bu, bi = ctx.sgd_get()
    assert ran == ref.steps_run
    assert np.array_equal(P, ref.P)
    assert np.array_equal(Q, ref.Q)
    assert np.array_equal(bu, ref.bu)
    assert np.array_equal(bi, ref.bi)
    np.testing.assert_allclose(hist, ref.rmse, rtol=1e-12, atol=0)


def test_small_workload_three_epochs_bit_identical():
    w = synth.SMALL
    r = synth.generate(w)
    ctx, hist, ran, ref = run_both(r, w.p, w.q, osgd.K, 3)
    assert_same(ctx, hist, ran, ref)
    assert hist[-1] < hist[0]


@pytest.mark.parametrize("p,q,k", [(3, 2, 7), (2, 5, 1), (1, 1, 32),
                                   (4, 4, 13), (7, 3, 5), (3, 3, 15),
                                   (2, 3, 16)])
def test_grid_shapes_and_ranks(p, q, k):
    r = synth.random_ratings(31, 300, 200, 6000, 0)
    ctx, hist, ran, ref = run_both(r, p, q, k, 2)
    assert_same(ctx, hist, ran, ref)


@pytest.mark.parametrize("f32", [False, True])
def test_quantile_grid_with_permutations_on_device_inputs(f32):
    w = synth.UNEVEN
    r = synth.generate(w)
    kw = qgrid.quantile_grid(r.u_train, r.i_train, w.m, w.n, w.p, w.q)
    ctx, hist, ran, ref = run_both(r, w.p, w.q, osgd.K, 1, grid_kw=kw,
                                   on_device=True, f32=f32)
    assert_same(ctx, hist, ran, ref)


# ---- the float32 form: bit-identical to the float32 oracle ----------------

@pytest.mark.parametrize("p,q,k", [(3, 2, 7), (2, 5, 1), (1, 1, 32),
                                   (4, 4, 13), (7, 3, 5), (2, 3, 16)])
def test_float32_form_grid_shapes_and_ranks(p, q, k):
    """Blocks small enough to stage in shared memory."""
    r = synth.random_ratings(31, 300, 200, 6000, 0)
    ctx, hist, ran, ref = run_both(r, p, q, k, 2, f32=True)
    assert_same(ctx, hist, ran, ref)


def test_float32_form_in_global_memory():
    """One block of 3,000 users and 600 items at k = 32 needs
    3,600 x 34 x 4 = 490 KB, more than a CTA's shared memory: the block
    works on its rows in global memory."""
    r = synth.random_ratings(34, 3000, 600, 30000, 0)
    ctx, hist, ran, ref = run_both(r, 1, 1, 32, 2, f32=True)
    assert_same(ctx, hist, ran, ref)
    ctx, hist, ran, ref = run_both(r, 2, 2, 32, 2, f32=True)
    assert_same(ctx, hist, ran, ref)


def test_float32_form_medium_workload_tracks_float64():
    """The paper's 8 x 8 grid: three epochs equal the float32 oracle bit
    for bit, and stay within float32 rounding of the float64 form."""
    w = synth.MEDIUM_8x8
    r = synth.generate(w)
    ctx, hist, ran, ref = run_both(r, w.p, w.q, osgd.K, 3, f32=True)
    assert_same(ctx, hist, ran, ref)
    _, hist64, _, _ = run_both(r, w.p, w.q, osgd.K, 3)
    np.testing.assert_allclose(hist, hist64, rtol=1e-5)
    assert hist[-1] < hist[0]
    got = ctx.sgd_predict(r.u_test, r.i_test)
    want = osgd.predict(ref.P, ref.Q, ref.bu, ref.bi, r.u_test, r.i_test)
    assert np.array_equal(got, want)


def test_medium_workload_stops_where_the_oracle_stops():
    """Section 5 hyper-parameters and delta = 1e-4 on the 8 x 8 grid the
    paper's CPU experiment used for MovieLens 1M."""
    w = synth.MEDIUM_8x8
    r = synth.generate(w)
    ctx, hist, ran, ref = run_both(r, w.p, w.q, osgd.K, 60,
                                   delta=osgd.DELTA)
    assert_same(ctx, hist, ran, ref)
    print("medium 8x8: %d epochs, train rmse %.6f -> %.6f"
          % (ran, hist[0], hist[-1]))


def test_early_stop_at_the_same_epoch():
    w = synth.SMALL
    r = synth.generate(w)
    ctx, hist, ran, ref = run_both(r, w.p, w.q, osgd.K, 100, delta=2e-3)
    assert_same(ctx, hist, ran, ref)
    assert 1 < ran < 100
    assert hist[-2] - hist[-1] < 2e-3 <= hist[-3] - hist[-2]


def test_predictions_bit_identical():
    w = synth.SMALL
    r = synth.generate(w)
    ctx, hist, ran, ref = run_both(r, w.p, w.q, 9, 2)
    got = ctx.sgd_predict(r.u_test, r.i_test)
    want = osgd.predict(ref.P, ref.Q, ref.bu, ref.bi, r.u_test, r.i_test)
    assert np.array_equal(got, want)
    # on device arrays too
    dev = torch.zeros(len(r.u_test), dtype=torch.float64, device="cuda")
    ctx.sgd_predict(torch.from_numpy(r.u_test).cuda(),
                    torch.from_numpy(r.i_test).cuda(), dev)
    assert np.array_equal(dev.cpu().numpy(), want)


def test_block_diagonal_batch_is_one_step():
    rng = np.random.default_rng(5)
    rb = np.array([0, 40, 70, 130], np.int64)
    cb = np.array([0, 25, 60, 80], np.int64)
    us, is_, xs = [], [], []
    for b in range(3):
        cells = rng.choice((rb[b + 1] - rb[b]) * (cb[b + 1] - cb[b]), 300,
                           replace=False)
        us.append(rb[b] + cells // (cb[b + 1] - cb[b]))
        is_.append(cb[b] + cells % (cb[b + 1] - cb[b]))
        xs.append(rng.integers(1, 6, 300))
    u = np.concatenate(us).astype(np.int32)
    i = np.concatenate(is_).astype(np.int32)
    x = np.concatenate(xs).astype(np.float32)
    P0, Q0 = synth.sgd_start(130, 80, 6)
    ctx = bs.Context()
    ctx.partition_diag(rb, cb, u, i, x)
    ctx.sgd_prepare(u, i, x)
    hist, ran = ctx.sgd_train(P0, Q0, max_steps=3, delta=-1e300)
    g = oracle.make_grid(130, 80, 3, 3, row_bounds=rb, col_bounds=cb)
    ref = osgd.train(g, u, i, x, P0, Q0, 3, delta=-1e300)
    assert_same(ctx, hist, ran, ref)
    hist, ran = ctx.sgd_train(P0, Q0, max_steps=3, delta=-1e300,
                              precision=bs.SGD_FP32)
    ref = osgd.train(g, u, i, x, P0, Q0, 3, delta=-1e300, dtype=np.float32)
    assert_same(ctx, hist, ran, ref)


def test_call_order_and_bad_arguments():
    r = synth.random_ratings(32, 50, 40, 400, 0)
    P0, Q0 = synth.sgd_start(50, 40, 4)
    ctx = bs.Context()
    with pytest.raises(bs.BsvdError) as e:
        ctx.sgd_prepare(r.u_train, r.i_train, r.x_train)
    assert e.value.status == bs.ESTATE
    ctx.partition(50, 40, r.u_train, r.i_train, r.x_train, 2, 2)
    with pytest.raises(bs.BsvdError) as e:
        ctx.sgd_train(P0, Q0)
    assert e.value.status == bs.ESTATE
    bad = r.u_train.copy()
    bad[3] = 50
    with pytest.raises(bs.BsvdError) as e:
        ctx.sgd_prepare(bad, r.i_train, r.x_train)
    assert e.value.status == bs.EINVAL
    ctx.sgd_prepare(r.u_train, r.i_train, r.x_train)
    for kk in (0, 33):
        with pytest.raises(bs.BsvdError) as e:
            ctx.sgd_train(np.zeros((50, max(kk, 1))), np.zeros((40, max(kk, 1))),
                          k=kk)
        assert e.value.status == bs.EINVAL
    with pytest.raises(bs.BsvdError) as e:
        ctx.sgd_train(P0, Q0, precision=2)
    assert e.value.status == bs.EINVAL
    with pytest.raises(bs.BsvdError) as e:
        ctx.sgd_predict(r.u_test, r.i_test)
    assert e.value.status == bs.ESTATE
    hist, ran = ctx.sgd_train(P0, Q0, max_steps=0)
    assert ran == 0 and len(hist) == 1


def test_equal_grid_with_empty_trailing_block_rows():
    """300 users on 32 block rows of ceil(300 / 32) = 10: block row 31 lies
    wholly past the last user, and so do its blocks in every step."""
    r = synth.random_ratings(33, 300, 200, 5000, 0)
    ctx, hist, ran, ref = run_both(r, 32, 32, 5, 2)
    assert_same(ctx, hist, ran, ref)
    ctx, hist, ran, ref = run_both(r, 32, 7, 5, 2)
    assert_same(ctx, hist, ran, ref)
