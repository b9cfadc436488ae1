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


@st.composite
def matrices(draw):
    m = draw(st.integers(1, 12))
    n = draw(st.integers(1, 12))
    seed = draw(st.integers(0, 2**31 - 1))
    kind = draw(st.sampled_from(["gauss", "small_ints", "dup_cols", "zero"]))
    rng = np.random.default_rng(seed)
    if kind == "gauss":
        a = rng.normal(size=(m, n))
    elif kind == "small_ints":          # many zeros and repeats, often rank-deficient
        a = rng.integers(-3, 4, size=(m, n)).astype(np.float64)
    elif kind == "dup_cols":            # repeated columns: exact rank deficiency
        base = rng.normal(size=(m, max(1, n // 2)))
        a = base[:, rng.integers(0, base.shape[1], size=n)]
    else:
        a = np.zeros((m, n))
    return a


@settings(max_examples=200, deadline=None)
@given(matrices())
def test_jacobi_svd_properties(a):
    """Eq. 1 for any shape: A = U S V^T, descending non-negative S equal to
    numpy's singular values, sum S^2 = ||A||_F^2. The short side's factor
    (the accumulated rotations: V when m >= n, U otherwise) is orthonormal;
    the long side's columns are orthonormal wherever the singular value is
    not negligible (zero columns elsewhere)."""
    m, n = a.shape
    U, s, V = oracle.svd(a)
    r = min(m, n)
    assert U.shape == (m, r) and s.shape == (r,) and V.shape == (n, r)
    assert np.all(s >= 0) and np.all(np.diff(s) <= 0)
    scale = max(1.0, float(np.abs(a).max()))
    ref = np.linalg.svd(a, compute_uv=False)
    assert np.allclose(s, ref, rtol=0, atol=1e-12 * scale * (m + n))
    assert np.allclose(U @ np.diag(s) @ V.T, a, rtol=0,
                       atol=1e-12 * scale * (m + n))
    fro2 = float(np.sum(a * a))
    assert abs(float(np.sum(s * s)) - fro2) <= 1e-12 * max(1.0, fro2) * (m + n)
    short, long_ = (V, U) if m >= n else (U, V)
    assert np.allclose(short.T @ short, np.eye(r), rtol=0,
                       atol=1e-12 * (m + n))
    live = s > 1e-10 * max(s[0] if r else 0.0, 1e-300)
    Ll = long_[:, live]
    assert np.allclose(Ll.T @ Ll, np.eye(int(live.sum())), rtol=0,
                       atol=1e-10 * (m + n))
