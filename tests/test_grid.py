"""Activity-quantile grids (the batched form's uneven cut): the oracle's cut
against a hand-worked example and brute force (CPU), and the library's
bsvd_quantile_grid against the oracle bit for bit (GPU)."""
import numpy as np
import pytest

import oracle


def _library_cut(ids, size, parts):
    """One side of bsvd_quantile_grid: the ids as users of a size x 1
    matrix, cut into parts block rows (one block column)."""
    torch = pytest.importorskip("torch")
    import paper_1907_07410_gb300 as bs
    ids = np.ascontiguousarray(ids, np.int32)
    zeros = np.zeros(ids.size, np.int32)
    with bs.Context() as ctx:
        kw = ctx.quantile_grid(size, 1, torch.from_numpy(ids).cuda(),
                               torch.from_numpy(zeros).cuda(), parts, 1)
    return kw["row_perm"].cpu().numpy(), kw["row_bounds"]


@pytest.mark.gpu
def test_library_hand_example():
    # counts per id: [5, 1, 3, 0, 3] -> order 0, 2, 4, 1, 3 (ties by id)
    ids = np.array([0] * 5 + [1] + [2] * 3 + [4] * 3)
    perm, bounds = _library_cut(ids, 5, 2)
    assert perm.tolist() == [0, 3, 1, 4, 2]
    # ratings before positions 0..5: 0, 5, 8, 11, 12, 12; half of 12 is
    # first reached before position 2
    assert bounds.tolist() == [0, 2, 5]
    perm3, bounds3 = _library_cut(ids, 5, 3)
    # thirds: 4 and 8 ratings -> positions 1 (5 >= 4) and 2 (8 >= 8)
    assert bounds3.tolist() == [0, 1, 2, 5]


@pytest.mark.gpu
@pytest.mark.parametrize("seed,size,parts", [(1, 50, 4), (2, 1000, 8),
                                             (3, 300, 32), (4, 17, 17),
                                             (7, 5000, 1), (8, 9000, 31)])
def test_library_matches_oracle(seed, size, parts):
    """bsvd_quantile_grid against the oracle's cut, bit for bit; sizes on
    both sides of the 4096-key sorting tile."""
    rng = np.random.default_rng(seed)
    w = (np.arange(size) + 1.0) ** -1.1
    ids = rng.choice(size, size=20 * size, p=w / w.sum())
    perm, bounds = _library_cut(ids, size, parts)
    operm, obounds = oracle.activity_quantile_cut(ids, size, parts)
    assert np.array_equal(perm, operm)
    assert np.array_equal(bounds, obounds)


@pytest.mark.gpu
def test_library_grid_both_sides_and_errors():
    torch = pytest.importorskip("torch")
    import paper_1907_07410_gb300 as bs
    rng = np.random.default_rng(9)
    m, n = 700, 300
    u = rng.integers(0, m, 6000).astype(np.int32)
    i = (rng.integers(0, n, 6000) ** 2 % n).astype(np.int32)
    with bs.Context() as ctx:
        kw = ctx.quantile_grid(m, n, u, i, 5, 3)       # host arrays
        rp, rb = oracle.activity_quantile_cut(u, m, 5)
        cp, cb = oracle.activity_quantile_cut(i, n, 3)
        assert np.array_equal(kw["row_perm"], rp)
        assert np.array_equal(kw["col_perm"], cp)
        assert np.array_equal(kw["row_bounds"], rb)
        assert np.array_equal(kw["col_bounds"], cb)
        bad = u.copy()
        bad[17] = m
        with pytest.raises(bs.BsvdError) as e:
            ctx.quantile_grid(m, n, bad, i, 5, 3)
        assert e.value.status == bs.EINVAL
        with pytest.raises(bs.BsvdError):
            ctx.quantile_grid(m, n, u, i, m + 1, 3)


@pytest.mark.gpu
def test_partition_quantile_matches_the_two_calls():
    """bsvd_partition_quantile (the grid cut and the partition in one call,
    host ratings uploaded once) gives the oracle's bounds and the same
    counts, means and factors as bsvd_quantile_grid + bsvd_partition, from
    host and from device inputs; a bad id is rejected."""
    torch = pytest.importorskip("torch")
    import paper_1907_07410_gb300 as bs
    import synth
    w = synth.UNEVEN
    r = synth.generate(w)
    _, orb = oracle.activity_quantile_cut(r.u_train, w.m, w.p)
    _, ocb = oracle.activity_quantile_cut(r.i_train, w.n, w.q)

    def run(one_call, on_device):
        conv = (lambda a: torch.from_numpy(a).cuda()) if on_device else (lambda a: a)
        u, i, x = conv(r.u_train), conv(r.i_train), conv(r.x_train)
        with bs.Context() as ctx:
            if one_call:
                rb, cb = ctx.partition_quantile(w.m, w.n, u, i, x, w.p, w.q)
            else:
                kw = ctx.quantile_grid(w.m, w.n, u, i, w.p, w.q)
                ctx.partition(w.m, w.n, u, i, x, w.p, w.q, **kw)
                rb, cb = kw["row_bounds"], kw["col_bounds"]
            counts, mu = ctx.block_stats()
            assert ctx.factor(w.k) == bs.OK
            sig = [ctx.get_block(b)["sigma"] for b in range(w.p * w.q)]
            rm = ctx.rmse(r.u_test, r.i_test, r.x_test)
        return rb, cb, counts, mu, sig, rm

    ref = run(False, True)
    assert np.array_equal(ref[0], orb) and np.array_equal(ref[1], ocb)
    for on_device in (True, False):
        got = run(True, on_device)
        assert np.array_equal(got[0], ref[0]) and np.array_equal(got[1], ref[1])
        assert np.array_equal(got[2], ref[2]) and np.array_equal(got[3], ref[3])
        for a, b in zip(got[4], ref[4]):
            assert np.array_equal(a, b)
        assert got[5] == ref[5]
    bad = r.u_train.copy()
    bad[5] = w.m
    with bs.Context() as ctx:
        with pytest.raises(bs.BsvdError) as e:
            ctx.partition_quantile(w.m, w.n, bad, r.i_train, r.x_train, w.p, w.q)
        assert e.value.status == bs.EINVAL


def test_oracle_cut_hand_example():
    ids = np.array([0] * 5 + [1] + [2] * 3 + [4] * 3)
    perm, bounds = oracle.activity_quantile_cut(ids, 5, 2)
    assert perm.tolist() == [0, 3, 1, 4, 2]
    assert bounds.tolist() == [0, 2, 5]
    assert oracle.activity_quantile_cut(ids, 5, 3)[1].tolist() == [0, 1, 2, 5]


@pytest.mark.parametrize("seed,size,parts", [(5, 40, 3), (6, 200, 7)])
def test_oracle_cut_brute_force(seed, size, parts):
    """Each bound is the first position whose preceding ids hold at least
    g / parts of the ratings, checked by trying every position; the order is
    by count descending, ids ascending on ties."""
    rng = np.random.default_rng(seed)
    ids = rng.integers(0, size, size=15 * size) ** 2 % size
    perm, bounds = oracle.activity_quantile_cut(ids, size, parts)
    counts = np.bincount(ids, minlength=size)
    order = np.argsort(perm)
    for a, b in zip(order[:-1], order[1:]):
        assert (counts[a], -a) > (counts[b], -b)
    total = len(ids)
    for g in range(1, parts):
        first = next(j for j in range(size + 1)
                     if parts * counts[order[:j]].sum() >= g * total)
        assert bounds[g] == first
