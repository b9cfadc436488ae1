"""Pins of the blocked-SGD oracle (Algorithms 1-2) against facts that do not
come from the oracle itself: the gradient of the per-rating loss (finite
differences), the independence of a schedule step's blocks, a hand-worked
processing order, monotone descent on an exact low-rank matrix, and the
stopping rule."""
import numpy as np
import pytest

import oracle
from oracle import sgd


def loss(x, p, q, bu, bi, r: sgd.Rates):
    """Per-rating regularised loss whose half-gradient the updates follow:
    err^2 + b_user |p|^2 + b_item |q|^2 + b_ubias bu^2 + b_ibias bi^2
    (Section 2.2, the regularised objective, restricted to one rating)."""
    err = x - bu - bi - float(np.dot(p, q))
    return (err * err + r.b_user * float(np.dot(p, p))
            + r.b_item * float(np.dot(q, q)) + r.b_ubias * bu * bu
            + r.b_ibias * bi * bi)


def test_single_update_is_a_gradient_step():
    rng = np.random.default_rng(0)
    k = 5
    r = sgd.Rates(a_user=0.02, b_user=0.03, a_item=0.01, b_item=0.05,
                  a_ubias=0.007, b_ubias=0.11, a_ibias=0.013, b_ibias=0.17)
    P = rng.normal(0, 0.4, (3, k))
    Q = rng.normal(0, 0.4, (2, k))
    bu = rng.normal(0, 0.2, 3)
    bi = rng.normal(0, 0.2, 2)
    u, i, x = 2, 1, 4.0
    P1, Q1, bu1, bi1 = P.copy(), Q.copy(), bu.copy(), bi.copy()
    sgd.sgd_pass([u], [i], [x], P1, Q1, bu1, bi1, r)
    h = 1e-6

    def grad(fn, v):
        g = np.zeros_like(v)
        for t in range(v.size):
            e = np.zeros_like(v)
            e.flat[t] = h
            g.flat[t] = (fn(v + e) - fn(v - e)) / (2 * h)
        return g
    gp = grad(lambda v: loss(x, v, Q[i], bu[u], bi[i], r), P[u])
    gq = grad(lambda v: loss(x, P[u], v, bu[u], bi[i], r), Q[i])
    gbu = grad(lambda v: loss(x, P[u], Q[i], v[0], bi[i], r), bu[u:u + 1])
    gbi = grad(lambda v: loss(x, P[u], Q[i], bu[u], v[0], r), bi[i:i + 1])
    np.testing.assert_allclose(P1[u] - P[u], -0.5 * r.a_user * gp, rtol=1e-6,
                               atol=1e-10)
    np.testing.assert_allclose(Q1[i] - Q[i], -0.5 * r.a_item * gq, rtol=1e-6,
                               atol=1e-10)
    np.testing.assert_allclose(bu1[u] - bu[u], -0.5 * r.a_ubias * gbu[0],
                               rtol=1e-6)
    np.testing.assert_allclose(bi1[i] - bi[i], -0.5 * r.a_ibias * gbi[0],
                               rtol=1e-6)
    # nothing else moved
    for a, b in ((P1, P), (Q1, Q), (bu1, bu), (bi1, bi)):
        mask = np.ones(len(a), bool)
        mask[u if a is P1 or a is bu1 else i] = False
        assert np.array_equal(a[mask], b[mask])


def test_zero_rates_change_nothing():
    rng = np.random.default_rng(1)
    P, Q = rng.normal(size=(4, 3)), rng.normal(size=(5, 3))
    bu, bi = rng.normal(size=4), rng.normal(size=5)
    P0, Q0, bu0, bi0 = P.copy(), Q.copy(), bu.copy(), bi.copy()
    z = sgd.Rates(0, 0.3, 0, 0.3, 0, 0.3, 0, 0.3)
    sgd.sgd_pass([0, 3, 1], [4, 0, 2], [5, 1, 3], P, Q, bu, bi, z)
    for a, b in ((P, P0), (Q, Q0), (bu, bu0), (bi, bi0)):
        assert np.array_equal(a, b)


@pytest.mark.parametrize("p,q", [(1, 1), (2, 2), (4, 4), (3, 2), (2, 5),
                                 (8, 3)])
def test_schedule_steps_are_independent_and_cover_the_grid(p, q):
    steps = sgd.schedule(p, q)
    assert len(steps) == max(p, q)
    seen = []
    for step in steps:
        rows = [b // q for b in step]
        cols = [b % q for b in step]
        assert len(set(rows)) == len(rows) and len(set(cols)) == len(cols)
        assert len(step) == min(p, q)
        seen += step
    assert sorted(seen) == list(range(p * q))
    # the first step is the main diagonal
    assert steps[0] == [d * q + d for d in range(min(p, q))]


def test_order_within_a_step_does_not_matter():
    """Blocks of one step touch disjoint parameters, so processing them in
    reverse order gives bit-identical results."""
    rng = np.random.default_rng(2)
    m, n, p, q, k = 40, 30, 4, 3, 4
    cells = rng.choice(m * n, size=500, replace=False)
    u, i = (cells // n).astype(np.int32), (cells % n).astype(np.int32)
    x = rng.integers(1, 6, 500).astype(np.float32)
    grid = oracle.make_grid(m, n, p, q)
    b, r, c = grid.locate(u, i)
    P0 = rng.normal(0, 0.1, (m, k))
    Q0 = rng.normal(0, 0.1, (n, k))
    outs = []
    for reverse in (False, True):
        pos = {}
        t = 0
        for step in sgd.schedule(p, q):
            for blk in (step[::-1] if reverse else step):
                pos[blk] = t
                t += 1
        order = np.lexsort((c, r, np.array([pos[v] for v in b])))
        P, Q = P0.copy(), Q0.copy()
        bu, bi = np.zeros(m), np.zeros(n)
        sgd.sgd_pass(u[order], i[order], x[order], P, Q, bu, bi, sgd.Rates())
        outs.append((P, Q, bu, bi))
    for a, b_ in zip(*outs):
        assert np.array_equal(a, b_)


def test_processing_order_hand_example():
    # 4 users x 4 items, 2 x 2 grid of 2 x 2 blocks; steps: {(0,0),(1,1)},
    # then {(1,0),(0,1)}
    u = np.array([3, 0, 1, 0, 2, 3, 1, 2], np.int32)
    i = np.array([3, 1, 0, 0, 1, 0, 3, 2], np.int32)
    grid = oracle.make_grid(4, 4, 2, 2)
    order = sgd.processing_order(grid, u, i)
    got = [(int(u[t]), int(i[t])) for t in order]
    # block (0,0): (0,0) (0,1) (1,0); block (1,1): (2,2) (3,3);
    # block (1,0): (2,1) (3,0); block (0,1): (1,3)
    assert got == [(0, 0), (0, 1), (1, 0), (2, 2), (3, 3), (2, 1), (3, 0),
                   (1, 3)]


def test_training_descends_on_an_exact_low_rank_matrix():
    rng = np.random.default_rng(3)
    m, n, k = 30, 20, 2
    A = rng.normal(0, 0.6, (m, k)) @ rng.normal(0, 0.6, (n, k)).T
    X = A + rng.normal(0, 0.3, m)[:, None] + rng.normal(0, 0.3, n)[None, :]
    u, i = np.nonzero(np.ones((m, n)))
    x = X[u, i].astype(np.float32)
    grid = oracle.make_grid(m, n, 3, 2)
    r = sgd.Rates(0.02, 0.001, 0.02, 0.001, 0.02, 0.001, 0.02, 0.001)
    t = sgd.train(grid, u, i, x, rng.normal(0, 0.1, (m, k)),
                  rng.normal(0, 0.1, (n, k)), steps=60, rates=r, delta=-1.0)
    h = np.array(t.rmse)
    assert t.steps_run == 60
    assert np.all(np.diff(h) < 0)
    assert h[-1] < 0.1 * h[0]


def test_stopping_rule():
    rng = np.random.default_rng(4)
    m, n = 12, 10
    u, i = np.nonzero(rng.random((m, n)) < 0.5)
    x = rng.integers(1, 6, len(u)).astype(np.float32)
    grid = oracle.make_grid(m, n, 2, 2)
    P0, Q0 = rng.normal(0, 0.1, (m, 3)), rng.normal(0, 0.1, (n, 3))
    # an improvement can never reach 10: one epoch, then stop
    t = sgd.train(grid, u, i, x, P0, Q0, steps=20, delta=10.0)
    assert t.steps_run == 1 and len(t.rmse) == 2
    # delta <= 0 with descent: all steps run
    t = sgd.train(grid, u, i, x, P0, Q0, steps=5, delta=-1e9)
    assert t.steps_run == 5 and len(t.rmse) == 6


def test_float32_pass_is_exact_where_float32_is():
    """With power-of-two rates and values of a few significant bits, no
    operation of two updates (one per user and item) rounds in float32, so the float32 pass must
    equal the float64 pass (pinned above) bit for bit: a dropped term, a
    wrong sign or a swapped operand in the float32 code would show."""
    r = sgd.Rates(a_user=2.0 ** -4, b_user=2.0 ** -3, a_item=2.0 ** -5,
                  b_item=2.0 ** -2, a_ubias=2.0 ** -3, b_ubias=2.0 ** -4,
                  a_ibias=2.0 ** -2, b_ibias=2.0 ** -5)
    P = np.array([[0.5, -0.25, 0.75], [0.125, 0.5, -0.5]])
    Q = np.array([[-0.5, 0.25, 0.5], [0.75, -0.125, 0.25], [0.5, 0.5, 0.5]])
    u, i, x = [0, 1], [2, 0], [4.0, 2.0]
    P64, Q64 = P.copy(), Q.copy()
    bu64, bi64 = np.zeros(2), np.zeros(3)
    sgd.sgd_pass(u, i, x, P64, Q64, bu64, bi64, r)
    P32, Q32 = P.astype(np.float32), Q.astype(np.float32)
    bu32, bi32 = np.zeros(2, np.float32), np.zeros(3, np.float32)
    sgd.sgd_pass(u, i, x, P32, Q32, bu32, bi32, r)
    # the float64 results still fit in float32 exactly
    for a in (P64, Q64, bu64, bi64):
        assert np.array_equal(a.astype(np.float32).astype(np.float64), a)
    assert not np.array_equal(P64, P) and not np.array_equal(bi64, 0 * bi64)
    for a, b in ((P32, P64), (Q32, Q64), (bu32, bu64), (bi32, bi64)):
        assert np.array_equal(a.astype(np.float64), b)


def test_float32_training_tracks_float64():
    """Float32 training from the same start stays within float32 rounding
    of the float64 run: each update perturbs a parameter by about 2^-24 of
    its size and the updates contract, so after three epochs on a few
    thousand ratings the parameters agree to ~1e-5 and the RMSE history to
    ~1e-6, while a mistake in the float32 pass would move them by the size
    of an update (~1e-2)."""
    rng = np.random.default_rng(5)
    m, n, k = 60, 40, 6
    u, i = np.nonzero(rng.random((m, n)) < 0.6)
    x = rng.integers(1, 6, len(u)).astype(np.float32)
    grid = oracle.make_grid(m, n, 3, 2)
    P0, Q0 = rng.normal(0, 0.1, (m, k)), rng.normal(0, 0.1, (n, k))
    t64 = sgd.train(grid, u, i, x, P0, Q0, steps=3, delta=-1e300)
    t32 = sgd.train(grid, u, i, x, P0, Q0, steps=3, delta=-1e300,
                    dtype=np.float32)
    assert t32.steps_run == 3 and t32.P.dtype == np.float64
    for a in (t32.P, t32.Q, t32.bu, t32.bi):
        assert np.array_equal(a.astype(np.float32).astype(np.float64), a)
    for a, b in ((t32.P, t64.P), (t32.Q, t64.Q), (t32.bu, t64.bu),
                 (t32.bi, t64.bi)):
        d = np.max(np.abs(a - b))
        assert 0 < d < 2e-5
    np.testing.assert_allclose(t32.rmse, t64.rmse, rtol=2e-6)
    assert t32.rmse[-1] < t32.rmse[0]
