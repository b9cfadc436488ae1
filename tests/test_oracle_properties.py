"""Property tests of the oracle's partition (Section 3, Eq. "datax") over
random shapes and grids, including grids with more block rows or columns
than the matrix has rows or columns (empty blocks). Each property is
checked against a direct recount, not against the oracle itself."""
import collections
import math

import numpy as np
import pytest

hypothesis = pytest.importorskip("hypothesis")
from hypothesis import given, settings, strategies as st  # noqa: E402

import oracle  # noqa: E402
import synth  # noqa: E402


@st.composite
def grids(draw):
    m = draw(st.integers(1, 40))
    n = draw(st.integers(1, 40))
    p = draw(st.integers(1, m + 3))
    q = draw(st.integers(1, n + 3))
    nnz = draw(st.integers(1, max(1, m * n // 2)))
    seed = draw(st.integers(0, 2**31 - 1))
    return m, n, p, q, nnz, seed


@settings(max_examples=150, deadline=None)
@given(grids())
def test_partition_properties(g):
    m, n, p, q, nnz, seed = g
    r = synth.random_ratings(seed, m, n, nnz, 0)
    part = oracle.partition(m, n, r.u_train, r.i_train, r.x_train, p, q)
    rb = np.asarray(part.grid.row_bounds)
    cb = np.asarray(part.grid.col_bounds)
    # the bounds tile [0, m) and [0, n): equal blocks of ceil(m/p), ceil(n/q)
    # with the remainder in the last non-empty one
    assert rb[0] == 0 and rb[-1] == m and np.all(np.diff(rb) >= 0)
    assert cb[0] == 0 and cb[-1] == n and np.all(np.diff(cb) >= 0)
    br, bc = -(-m // p), -(-n // q)
    assert np.all(np.diff(rb) <= br) and np.all(np.diff(cb) <= bc)
    # every rating in exactly one block, at in-range local coordinates that
    # map back to its global cell
    blk = np.asarray(part.block)
    lr = np.asarray(part.r)
    lc = np.asarray(part.c)
    bi, bj = blk // q, blk % q
    assert np.all((0 <= blk) & (blk < p * q))
    assert np.array_equal(rb[bi] + lr, r.u_train)
    assert np.array_equal(cb[bj] + lc, r.i_train)
    assert np.all(lr < rb[bi + 1] - rb[bi]) and np.all(lc < cb[bj + 1] - cb[bj])
    # counts and block means: a direct recount, the mean as an exact sum
    cells = collections.defaultdict(list)
    for b, x in zip(blk.tolist(), r.x_train.tolist()):
        cells[b].append(x)
    assert int(np.sum(part.counts)) == nnz
    for b in range(p * q):
        vals = cells.get(b, [])
        assert part.counts[b] == len(vals)
        if vals:
            assert part.mu32[b] == np.float32(math.fsum(vals) / len(vals))
