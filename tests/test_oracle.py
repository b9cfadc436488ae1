"""Pins for the FP64 oracle: every check here comes from mathematics or a
library routine, never from the oracle itself.

Each test is chosen so that a plausible slip in the oracle (a dropped mean,
a swapped U/V, a wrong rotation sign, a missing sort, an off-by-one block
bound) fails at least one of them.
"""
import collections
import math

import numpy as np
import pytest

import oracle
import synth

RTOL = 1e-12


def _rel(a, b):
    return np.max(np.abs(np.asarray(a) - np.asarray(b))) / max(
        1e-300, np.max(np.abs(b)))


# --- the Jacobi SVD (Section 2, Eq. 1) ------------------------------------

@pytest.mark.parametrize("seed", range(8))
def test_closed_form_2x2(seed):
    A = np.random.default_rng(seed).standard_normal((2, 2))
    S = np.sum(A * A)
    det = np.linalg.det(A)
    root = math.sqrt(max(S * S - 4 * det * det, 0.0))
    expect = [math.sqrt((S + root) / 2), math.sqrt(max((S - root) / 2, 0))]
    U, s, V = oracle.svd(A)
    assert _rel(s, expect) < 1e-13
    assert np.allclose(U @ np.diag(s) @ V.T, A, atol=1e-14)


def test_diagonal_rectangular():
    d = np.array([0.5, -3.0, 0.0, 2.0, -2.0])
    A = np.zeros((7, 5))
    A[np.arange(5), np.arange(5)] = d
    U, s, V = oracle.svd(A)
    assert np.array_equal(s, np.sort(np.abs(d))[::-1])
    # ties (|-2| == |2|) keep original column order: column 3 before 4
    assert abs(V[3, 1]) == 1.0 and abs(V[4, 2]) == 1.0
    U2, s2, V2 = oracle.svd(A.T)
    assert np.array_equal(s2, s)


def test_rank_one_and_factor_sides():
    rng = np.random.default_rng(1)
    u = rng.standard_normal(9)
    v = rng.standard_normal(4)
    A = np.outer(u, v)
    U, s, V = oracle.svd(A)
    assert abs(s[0] - np.linalg.norm(u) * np.linalg.norm(v)) < 1e-13 * s[0]
    assert np.all(s[1:] < 1e-13 * s[0])
    # U holds the row (length-9) side, V the column side
    assert U.shape == (9, 4) and V.shape == (4, 4)
    assert abs(abs(U[:, 0] @ u) - np.linalg.norm(u)) < 1e-12 * np.linalg.norm(u)
    assert abs(abs(V[:, 0] @ v) - np.linalg.norm(v)) < 1e-12 * np.linalg.norm(v)


@pytest.mark.parametrize("shape", [(40, 25), (25, 40), (30, 30)])
def test_prescribed_spectrum(shape):
    """Q diag(sigma) P^T with orthogonal Q, P and chosen sigma, including
    clustered, repeated and zero values."""
    rng = np.random.default_rng(7)
    m, n = shape
    r = min(m, n)
    sig = np.linspace(10.0, 1.0, r)
    sig[3] = sig[2] * (1 + 1e-9)       # a tight cluster
    sig[6] = sig[5]                    # an exact repeat
    sig[-3:] = 0.0                     # rank deficiency
    sig = np.sort(sig)[::-1]
    Q, _ = np.linalg.qr(rng.standard_normal((m, r)))
    P, _ = np.linalg.qr(rng.standard_normal((n, r)))
    A = (Q * sig) @ P.T
    U, s, V = oracle.svd(A)
    assert np.max(np.abs(s - sig)) < 1e-13 * sig[0]


@pytest.mark.parametrize("shape", [(60, 35), (35, 60), (1, 9), (9, 1), (1, 1),
                                   (17, 17)])
def test_invariants_and_numpy(shape):
    rng = np.random.default_rng(3)
    A = rng.standard_normal(shape) * (rng.random(shape) < 0.3)
    U, s, V = oracle.svd(A)
    r = min(shape)
    assert abs(np.sum(A * A) - np.sum(s * s)) <= 1e-12 * max(1.0, np.sum(s * s))
    assert np.allclose(U.T @ U, np.eye(r), atol=1e-12) or np.any(s == 0)
    assert np.allclose(V.T @ V, np.eye(r), atol=1e-12)
    assert np.allclose(A @ V, U * s, atol=1e-12)
    ref = np.linalg.svd(A, compute_uv=False)
    assert np.max(np.abs(s - ref)) <= 1e-12 * max(1.0, ref[0])
    assert np.all(np.diff(s) <= 0)


def test_transpose_permutation_padding_invariance():
    rng = np.random.default_rng(5)
    A = rng.standard_normal((23, 14)) * (rng.random((23, 14)) < 0.4)
    s = oracle.svd(A)[1]
    assert np.max(np.abs(oracle.svd(A.T)[1] - s)) < 1e-12 * s[0]
    Ap = A[rng.permutation(23)][:, rng.permutation(14)]
    assert np.max(np.abs(oracle.svd(Ap)[1] - s)) < 1e-12 * s[0]
    Z = np.zeros((30, 20))
    Z[:23, :14] = A
    sz = oracle.svd(Z)[1]
    assert np.max(np.abs(sz[:14] - s)) < 1e-12 * s[0]
    assert np.all(sz[14:] < 1e-12 * s[0])


def test_truncation_eckart_young():
    """|B - R_k|_F^2 equals the sum of the dropped sigma^2 (Section 2)."""
    rng = np.random.default_rng(11)
    B = rng.standard_normal((30, 18))
    f = oracle.factor_block(B, 5)
    R = f.P @ f.V.T
    assert abs(np.sum((B - R) ** 2) - np.sum(f.sigma[5:] ** 2)) < 1e-10
    assert f.keff == 5 and f.P.shape == (30, 5) and f.V.shape == (18, 5)
    # canonical sign: largest |entry| of each item-side vector is positive
    for j in range(5):
        assert f.V[np.argmax(np.abs(f.V[:, j])), j] > 0


# --- partition and means (Section 3, Eq. "datax") --------------------------

def _brute_partition(m, n, p, q, u, i, x):
    br, bc = -(-m // p), -(-n // q)
    cells = collections.defaultdict(list)
    where = []
    for uu, ii, xx in zip(u.tolist(), i.tolist(), x.tolist()):
        b = (uu // br) * q + (ii // bc)
        cells[b].append(xx)
        where.append((b, uu % br, ii % bc))
    return cells, where


@pytest.mark.parametrize("m,n,p,q", [(37, 23, 3, 4), (10, 10, 1, 1),
                                     (9, 31, 9, 2), (6040, 3952, 16, 16)])
def test_partition_bruteforce(m, n, p, q):
    r = synth.random_ratings(2, m, n, min(m * n // 3, 20000), 10)
    part = oracle.partition(m, n, r.u_train, r.i_train, r.x_train, p, q)
    cells, where = _brute_partition(m, n, p, q, r.u_train, r.i_train,
                                    r.x_train)
    assert [tuple(t) for t in zip(part.block.tolist(), part.r.tolist(),
                                  part.c.tolist())] == where
    for b in range(p * q):
        vals = cells.get(b, [])
        assert part.counts[b] == len(vals)
        if vals:
            assert part.mu32[b] == np.float32(math.fsum(vals) / len(vals))
    if (m, p) == (6040, 16):
        # 16 block rows of ceil(6040/16) = 378; the last holds 370
        sizes = np.diff(part.grid.row_bounds)
        assert sizes.tolist() == [378] * 15 + [370]


def test_mean_is_exact_sum():
    # naive left-to-right float sum loses the 1.0 entirely
    x = np.array([2.0 ** 24, 1.0, -(2.0 ** 24), 1.0, 1.0], np.float32)
    part = oracle.partition(1, 5, np.zeros(5, np.int32),
                            np.arange(5, dtype=np.int32), x, 1, 1)
    assert part.mu64[0] == 3.0 / 5.0
    assert part.mu32[0] == np.float32(0.6)


def test_empty_block_takes_global_mean():
    u = np.array([0, 0, 1], np.int32)
    i = np.array([0, 1, 0], np.int32)
    x = np.array([1.0, 2.0, 4.0], np.float32)
    part = oracle.partition(4, 4, u, i, x, 2, 2)
    assert part.counts.tolist() == [3, 0, 0, 0]
    assert part.mu64.tolist() == [7 / 3] * 4
    model = oracle.factor(part, 2)
    yhat = oracle.predict(model, np.array([3]), np.array([3]))
    assert yhat[0] == 7 / 3


def test_dense_block_values_and_padding():
    r = synth.random_ratings(4, 11, 7, 30, 0)
    part = oracle.partition(11, 7, r.u_train, r.i_train, r.x_train, 2, 2)
    # equal bounds: ceil(11/2) = 6 rows, last block row holds 5
    assert part.grid.block_shape(2) == (5, 4)
    assert part.grid.block_shape(3) == (5, 3)
    for b in range(4):
        B = oracle.dense_block(part, b)
        B32 = oracle.dense_block(part, b, fp32=True)
        r0 = part.grid.row_bounds[b // 2]
        c0 = part.grid.col_bounds[b % 2]
        for uu, ii, xx in zip(r.u_train, r.i_train, r.x_train):
            if part.grid.row_bounds[b // 2] <= uu < part.grid.row_bounds[
                    b // 2 + 1] and part.grid.col_bounds[b % 2] <= ii < \
                    part.grid.col_bounds[b % 2 + 1]:
                assert B[uu - r0, ii - c0] == float(xx) - part.mu64[b]
                assert B32[uu - r0, ii - c0] == np.float32(xx) - part.mu32[b]
        assert np.count_nonzero(B == 0) + part.counts[b] >= B.size


# --- whole-pipeline special cases -------------------------------------------

def test_one_block_is_global_truncated_svd():
    """With a 1 x 1 grid the method is the mean-centred rank-k SVD of the
    whole matrix (Section 3: MF is BMF with a single block)."""
    w = synth.SMALL
    r = synth.generate(w)
    part = oracle.partition(w.m, w.n, r.u_train, r.i_train, r.x_train, 1, 1)
    model = oracle.factor(part, w.k)
    x = r.x_train.astype(np.float64)
    mu = x.sum() / x.size
    X = np.zeros((w.m, w.n))
    X[r.u_train, r.i_train] = x - mu
    Un, sn, Vtn = np.linalg.svd(X, full_matrices=False)
    f = model.blocks[0]
    assert np.max(np.abs(f.sigma - sn)) < 1e-10 * sn[0]
    R = (Un[:, :w.k] * sn[:w.k]) @ Vtn[:w.k]
    pred = mu + R[r.u_test, r.i_test]
    assert np.max(np.abs(oracle.predict(model, r.u_test, r.i_test) - pred)) \
        < 1e-9


@pytest.mark.parametrize("k", [0, 10_000])
def test_zero_or_full_rank_predicts_block_mean(k):
    """k = 0 keeps nothing; k >= min(m_b, n_b) reconstructs B exactly, and
    a held-out cell is 0 in B. Both predict mu_b for every held-out cell,
    so the RMSE is the block-mean predictor's."""
    r = synth.random_ratings(9, 40, 30, 300, 80)
    part = oracle.partition(40, 30, r.u_train, r.i_train, r.x_train, 2, 3)
    model = oracle.factor(part, k)
    yhat = oracle.predict(model, r.u_test, r.i_test)
    b, _, _ = part.grid.locate(r.u_test, r.i_test)
    assert np.max(np.abs(yhat - part.mu64[b])) < 1e-12
    err = [(part.mu64[bb] - float(y)) ** 2 for bb, y in zip(b, r.x_test)]
    assert abs(oracle.rmse(model, r.u_test, r.i_test, r.x_test)
               - math.sqrt(sum(err) / len(err))) < 1e-12


def test_exact_rank_block_reconstructs():
    """A fully observed block of rank 3 around its mean is recovered."""
    rng = np.random.default_rng(12)
    half = rng.integers(-1, 2, (6, 3)).astype(float)
    L = np.vstack([half, -half])    # zero column sums: block mean exactly 3
    Rm = rng.integers(-1, 2, (3, 9)).astype(float)
    X = 3.0 + L @ Rm
    u, i = np.nonzero(np.ones_like(X))
    part = oracle.partition(12, 9, u.astype(np.int32), i.astype(np.int32),
                            X[u, i].astype(np.float32), 1, 1)
    assert part.mu64[0] == 3.0
    model = oracle.factor(part, 3)
    assert np.max(np.abs(oracle.reconstruct(model, 0) - X)) < 1e-12
    assert model.blocks[0].sigma[3] < 1e-12


def test_rmse_hand_example():
    # one block, k = 0: predictions are the mean 2.0
    u = np.array([0, 1], np.int32)
    i = np.array([0, 1], np.int32)
    part = oracle.partition(2, 2, u, i, np.array([1.0, 3.0], np.float32),
                            1, 1)
    model = oracle.factor(part, 0)
    got = oracle.rmse(model, np.array([0, 1]), np.array([1, 0]),
                      np.array([5.0, 2.0], np.float32))
    assert got == math.sqrt((9.0 + 0.0) / 2)


def test_out_of_range_ids_rejected():
    with pytest.raises(ValueError):
        oracle.partition(3, 3, np.array([3], np.int32),
                         np.array([0], np.int32),
                         np.array([1.0], np.float32), 1, 1)


def test_generator_shapes():
    w = synth.SMALL
    r = synth.generate(w)
    assert r.u_train.size + r.u_test.size == w.nnz
    assert r.u_test.size == w.nnz // 10
    keys = np.concatenate([r.u_train.astype(np.int64) * w.n + r.i_train,
                           r.u_test.astype(np.int64) * w.n + r.i_test])
    assert np.unique(keys).size == keys.size
    per_user = np.bincount(np.concatenate([r.u_train, r.u_test]),
                           minlength=w.m)
    assert per_user.min() >= 20 and per_user.max() <= w.n
    assert set(np.unique(r.x_train).tolist()) <= {1.0, 2.0, 3.0, 4.0, 5.0}


def test_oracle_is_usable_from_threads():
    """The reference arm runs the oracle on a thread pool: loading the C
    library from several threads at once, and running SVDs concurrently
    (the C routine releases the GIL), gives the serial results."""
    import concurrent.futures as cf
    rng = np.random.default_rng(11)
    mats = [rng.normal(size=(40 + 3 * t, 25 + t)) for t in range(8)]
    serial = [oracle.svd(a) for a in mats]
    oracle._lib = None                 # make the workers race to load it
    with cf.ThreadPoolExecutor(max_workers=8) as ex:
        threaded = list(ex.map(oracle.svd, mats))
    for (u0, s0, v0), (u1, s1, v1) in zip(serial, threaded):
        assert np.array_equal(s0, s1)
        assert np.array_equal(u0, u1) and np.array_equal(v0, v1)


# --- the Gram route for blocks too large for Jacobi (Eq. 1) -----------------

def _gram_route_agrees(part, k, blocks):
    jac = oracle.factor(part, k, blocks=blocks)
    gram = oracle.factor_gram(part, k, blocks=blocks)
    for b in blocks:
        fj, fg = jac.blocks[b], gram.blocks[b]
        assert fg.keff == fj.keff
        n = min(fj.keff + 1, fj.sigma.size)
        # absolute error of the Gram route is about eps * sigma_1^2 / sigma_i
        assert np.max(np.abs(fg.sigma[:n] - fj.sigma[:n])) <= 1e-11 * fj.sigma[0]
        if fj.keff and fj.gap >= 1e-3:
            Rj, Rg = fj.P @ fj.V.T, fg.P @ fg.V.T
            assert np.linalg.norm(Rg - Rj) <= 1e-8 * np.linalg.norm(Rj)
    return jac, gram


@pytest.mark.parametrize("workload,k", [(synth.SMALL, 10), (synth.SMALL, 40)])
def test_gram_route_matches_jacobi_users_side(workload, k):
    """2 x 2 small grid: 472 x 841 blocks, the users side is shorter."""
    w = workload
    r = synth.generate(w)
    part = oracle.partition(w.m, w.n, r.u_train, r.i_train, r.x_train, w.p,
                            w.q)
    _gram_route_agrees(part, k, [0, 3])


def test_gram_route_matches_jacobi_items_side_and_predictions():
    """A 4 x 12 cut of the medium matrix: 1510 x 330 blocks, the items side
    is shorter; predictions of their held-out ratings agree too."""
    w = synth.MEDIUM
    r = synth.generate(w)
    part = oracle.partition(w.m, w.n, r.u_train, r.i_train, r.x_train, 4, 12)
    blocks = [0, 17, 47]
    jac, gram = _gram_route_agrees(part, 20, blocks)
    b, _, _ = part.grid.locate(r.u_test, r.i_test)
    sel = np.isin(b, blocks)
    yj = oracle.predict(jac, r.u_test[sel], r.i_test[sel])
    yg = oracle.predict(gram, r.u_test[sel], r.i_test[sel])
    gaps = np.array([jac.blocks[int(x)].gap for x in b[sel]])
    ok = gaps >= 1e-3
    assert ok.any()
    assert np.max(np.abs(yj[ok] - yg[ok])) < 1e-8


def test_gram_route_closed_forms():
    """A diagonal block (only diagonal cells observed) has sigma = sorted
    |x - mu|; a fully observed block 3 + u v^T with sum(u) = 0 has the one
    singular value |u| |v|."""
    d = np.array([1.0, 5.0, 2.0, 4.0, 4.0, 3.0], np.float32)
    idx = np.arange(d.size, dtype=np.int32)
    part = oracle.partition(8, 6, idx, idx, d, 1, 1)
    mu = float(d.astype(np.float64).mean())
    f = oracle.factor_block_gram(part, 0, 3)
    want = np.sort(np.abs(d.astype(np.float64) - mu))[::-1]
    assert np.max(np.abs(f.sigma[:4] - want[:4])) < 1e-13
    # 9 x 5 rank one around the mean 3 (users side longer: items side G)
    u = np.array([1, -1, 2, -2, 0, 3, -3, 1, -1], float)
    v = np.array([1, 2, 0, -1, 3], float)
    X = 3.0 + np.outer(u, v)
    uu, ii = np.nonzero(np.ones_like(X))
    for shape, (a, c) in (((9, 5), (uu, ii)), ((5, 9), (ii, uu))):
        vals = X[uu, ii].astype(np.float32)
        part = oracle.partition(shape[0], shape[1], a.astype(np.int32),
                                c.astype(np.int32), vals, 1, 1)
        assert part.mu64[0] == 3.0
        f = oracle.factor_block_gram(part, 0, 2)
        s1 = np.linalg.norm(u) * np.linalg.norm(v)
        assert abs(f.sigma[0] - s1) < 1e-12 * s1
        assert f.sigma[1] < 1e-6 * s1
        R = f.P @ f.V.T
        want = np.outer(u, v) if shape == (9, 5) else np.outer(u, v).T
        assert np.max(np.abs(R[:, :] - want)) < 1e-10 * s1
