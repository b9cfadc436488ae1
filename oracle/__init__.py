"""Plain FP64 CPU oracle for the block-SVD recommender hot path.

TEST INFRASTRUCTURE ONLY. Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this package. The CUDA library
never calls it, and the two share no code: no kernels, headers, helpers or
constants. The only shared module is ``synth``, which generates seeded inputs
and holds none of the method's arithmetic.

What it computes, step by step, with the passage each step follows:

1. Partition (Section 3, Eq. "datax"). X (m users x n items) is cut into a
   p x q grid of blocks. The paper uses equal blocks and zero-pads X up to a
   multiple of the block size, so block rows hold ceil(m/p) users and block
   columns ceil(n/q) items; the last block row/column holds what remains.
   Explicit bounds (and a user/item permutation) may replace the equal cut.
2. Block mean (the reading taken here; the paper defines no imputation).
   mu_b = (sum of the block's training ratings) / (their count). The sum is
   exact (math.fsum), so mu_b in float32 is fl32(fl64(sum) / count). An
   empty block takes the global training mean.
3. Impute and centre. Missing cells take mu_b; then mu_b is subtracted, so
   B_b[r, c] = x - mu_b on observed cells and 0 elsewhere. Zero padding is
   therefore exact: padded rows and columns of zeros change neither the
   singular values nor the reconstruction on real cells.
4. Truncated SVD (Section 2, Eq. 1 and the rank-k truncation that follows).
   The full SVD B_b = U S V^T comes from FP64 one-sided Jacobi
   (``jacobi_svd.c``). Only the k_eff = min(k, min(m_b, n_b)) largest values
   are kept. P = U_k S_k (users x k) and V_k (items x k).
   Blocks too large for Jacobi (the large uneven workload's biggest are
   92,840 x 4,619) take the same truncated SVD through the FP64 symmetric
   eigenproblem of the shorter side's Gram matrix (``factor_block_gram``),
   pinned against the Jacobi route on blocks small enough for both.
5. Predict (Section 2.1, Eq. 2 with S merged into the user factor):
   y_hat(u, i) = mu_b + P[r, :] . V_k[c, :].
6. Score (Section 5, Table 1 "Test RMSE"):
   RMSE = sqrt(sum (y_hat - y)^2 / |held-out|), summed exactly.

Sign convention: singular vectors are only defined up to sign, so each pair
is flipped until the largest-magnitude entry of the item-side vector is
positive (lowest index on ties).
"""
from __future__ import annotations

import concurrent.futures as _cf
import ctypes
import dataclasses
import math
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "jacobi_svd.c")
_LIB = os.path.join(_HERE, "liboracle_jacobi.so")
_lib = None
_lock = threading.Lock()   # builds and loads from worker threads

MAX_SWEEPS = 60


def build(force: bool = False) -> str:
    """Compile the C Jacobi routine (plain gcc, no architecture flags), and
    the blocked-SGD pass of ``oracle.sgd``."""
    with _lock:
        if force or not os.path.exists(_LIB) or (
                os.path.getmtime(_LIB) < os.path.getmtime(_SRC)):
            tmp = _LIB + ".tmp%d.%d" % (os.getpid(), threading.get_ident())
            subprocess.check_call(["gcc", "-O2", "-fPIC", "-shared",
                                   "-std=c99", "-o", tmp, _SRC, "-lm"])
            os.replace(tmp, _LIB)
    from . import sgd
    sgd.build(force)
    return _LIB


def _load():
    global _lib
    if _lib is not None:
        return _lib
    path = build()
    with _lock:
        if _lib is not None:
            return _lib
        lib = ctypes.CDLL(path)
        f = lib.oracle_jacobi_svd
        f.restype = ctypes.c_int
        dp = ctypes.POINTER(ctypes.c_double)
        f.argtypes = [dp, ctypes.c_int64, ctypes.c_int64, dp, dp, dp,
                      ctypes.c_int]
        _lib = lib
    return _lib


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def svd(A: np.ndarray, max_sweeps: int = MAX_SWEEPS):
    """Thin SVD of a real matrix by FP64 one-sided Jacobi (Eq. 1).

    Returns (U, s, V) with A = U diag(s) V^T, s descending, U m x r and
    V n x r where r = min(m, n). Raises if Jacobi did not converge.
    """
    A = np.asarray(A, dtype=np.float64)
    m, n = A.shape
    if m >= n:
        work = np.array(A, dtype=np.float64, order="F")     # columns of A
        rows, cols = m, n
    else:
        work = np.array(A.T, dtype=np.float64, order="F")   # columns of A^T
        rows, cols = n, m
    U = np.zeros((rows, cols), order="F")
    s = np.zeros(cols)
    V = np.zeros((cols, cols), order="F")
    rc = _load().oracle_jacobi_svd(_ptr(work), rows, cols, _ptr(U), _ptr(s),
                                   _ptr(V), max_sweeps)
    if rc < 0:
        raise RuntimeError("one-sided Jacobi did not converge (rc=%d)" % rc)
    if m >= n:
        return np.ascontiguousarray(U), s, np.ascontiguousarray(V)
    # A^T = U s V^T  =>  A = V s U^T
    return np.ascontiguousarray(V), s, np.ascontiguousarray(U)


@dataclasses.dataclass
class Grid:
    """Block bounds in permuted row/column positions (Eq. "datax")."""
    m: int
    n: int
    p: int
    q: int
    row_bounds: np.ndarray          # int64, p + 1
    col_bounds: np.ndarray          # int64, q + 1
    row_perm: np.ndarray | None     # user id -> row position, or None
    col_perm: np.ndarray | None     # item id -> column position, or None

    def block_shape(self, b: int) -> tuple[int, int]:
        bi, bj = divmod(b, self.q)
        return (int(self.row_bounds[bi + 1] - self.row_bounds[bi]),
                int(self.col_bounds[bj + 1] - self.col_bounds[bj]))

    def locate(self, u: np.ndarray, i: np.ndarray):
        """Block id and local (row, col) of each (user, item) pair."""
        u = np.asarray(u, np.int64)
        i = np.asarray(i, np.int64)
        if u.size and (u.min() < 0 or u.max() >= self.m or i.min() < 0
                       or i.max() >= self.n):
            raise ValueError("rating index out of range")
        ru = self.row_perm[u] if self.row_perm is not None else u
        ci = self.col_perm[i] if self.col_perm is not None else i
        bi = np.searchsorted(self.row_bounds, ru, side="right") - 1
        bj = np.searchsorted(self.col_bounds, ci, side="right") - 1
        return (bi * self.q + bj, ru - self.row_bounds[bi],
                ci - self.col_bounds[bj])


def equal_bounds(total: int, parts: int) -> np.ndarray:
    """Equal blocks of ceil(total/parts); the last one holds the rest."""
    size = -(-total // parts) if parts > 0 else 0
    b = np.minimum(np.arange(parts + 1, dtype=np.int64) * size, total)
    return b


def make_grid(m, n, p, q, row_bounds=None, col_bounds=None, row_perm=None,
              col_perm=None) -> Grid:
    if p < 1 or q < 1:
        raise ValueError("grid must be at least 1 x 1")
    rb = equal_bounds(m, p) if row_bounds is None else np.asarray(
        row_bounds, np.int64)
    cb = equal_bounds(n, q) if col_bounds is None else np.asarray(
        col_bounds, np.int64)
    if (rb.size != p + 1 or cb.size != q + 1 or rb[0] != 0 or rb[-1] != m
            or cb[0] != 0 or cb[-1] != n or np.any(np.diff(rb) < 0)
            or np.any(np.diff(cb) < 0)):
        raise ValueError("bad block bounds")
    for perm, size in ((row_perm, m), (col_perm, n)):
        if perm is not None and not np.array_equal(
                np.sort(np.asarray(perm)), np.arange(size)):
            raise ValueError("not a permutation")
    return Grid(m, n, p, q, rb, cb,
                None if row_perm is None else np.asarray(row_perm, np.int64),
                None if col_perm is None else np.asarray(col_perm, np.int64))


def activity_quantile_cut(ids, size: int, parts: int):
    """Uneven grid side for the batched form (reading of "split at activity
    quantiles"): order ids by training-rating count, busiest first, ties by
    lower id; cut where the ratings before the cut first reach g/parts of
    all ratings (exact integer comparison parts * before >= g * total).
    Returns (perm: id -> position, bounds: parts + 1 positions)."""
    ids = np.asarray(ids, np.int64)
    if ids.size and (ids.min() < 0 or ids.max() >= size):
        raise ValueError("id out of range")
    counts = np.bincount(ids, minlength=size).tolist()   # ratings per id
    order = sorted(range(size), key=lambda x: (-counts[x], x))
    perm = np.empty(size, np.int64)
    for pos, x in enumerate(order):
        perm[x] = pos
    total = sum(counts)
    bounds = [0]
    before = 0
    pos = 0
    for g in range(1, parts):
        while pos < size and parts * before < g * total:
            before += counts[order[pos]]
            pos += 1
        bounds.append(pos)
    bounds.append(size)
    return perm, np.array(bounds, np.int64)


@dataclasses.dataclass
class Partition:
    grid: Grid
    block: np.ndarray        # block id per training rating
    r: np.ndarray            # local row
    c: np.ndarray            # local column
    x: np.ndarray            # rating (float64 copy of the float32 input)
    counts: np.ndarray       # int64 per block
    mu64: np.ndarray         # exact sum / count, float64
    mu32: np.ndarray         # float32 rounding of mu64
    global_mean: float


def partition(m, n, u, i, x, p, q, row_bounds=None, col_bounds=None,
              row_perm=None, col_perm=None) -> Partition:
    """Steps 1-2: block ids, local indices, counts and block means."""
    g = make_grid(m, n, p, q, row_bounds, col_bounds, row_perm, col_perm)
    x = np.asarray(x, np.float32).astype(np.float64)
    if not np.all(np.isfinite(x)):
        raise ValueError("non-finite rating")
    b, r, c = g.locate(u, i)
    nb = p * q
    counts = np.bincount(b, minlength=nb).astype(np.int64)
    gm = math.fsum(x.tolist()) / x.size if x.size else 0.0
    mu64 = np.full(nb, gm)
    order = np.argsort(b, kind="stable")
    starts = np.searchsorted(b[order], np.arange(nb + 1))
    for blk in range(nb):
        if counts[blk]:
            vals = x[order[starts[blk]:starts[blk + 1]]]
            mu64[blk] = math.fsum(vals.tolist()) / counts[blk]
    return Partition(g, b, r, c, x, counts, mu64, mu64.astype(np.float32),
                     gm)


def dense_block(part: Partition, b: int, fp32: bool = False) -> np.ndarray:
    """Step 3: the imputed, centred block B_b.

    fp32=False gives the FP64 matrix x - mu64 that the SVD runs on.
    fp32=True gives fl32(x - mu32), one float32 subtraction per cell: the
    exact values a float32 dense block must hold.
    """
    mb, nb = part.grid.block_shape(b)
    sel = part.block == b
    if fp32:
        B = np.zeros((mb, nb), np.float32)
        B[part.r[sel], part.c[sel]] = (part.x[sel].astype(np.float32)
                                       - part.mu32[b])
    else:
        B = np.zeros((mb, nb))
        B[part.r[sel], part.c[sel]] = part.x[sel] - part.mu64[b]
    return B


@dataclasses.dataclass
class BlockFactors:
    keff: int
    sigma: np.ndarray        # all min(m_b, n_b) singular values, descending
    P: np.ndarray            # m_b x keff, U_k S_k
    V: np.ndarray            # n_b x keff
    sweeps_ok: bool = True

    @property
    def gap(self) -> float:
        """(sigma_k - sigma_{k+1}) / sigma_k, or inf at full rank."""
        k = self.keff
        if k == 0 or k >= self.sigma.size or self.sigma[k - 1] == 0:
            return math.inf
        return float((self.sigma[k - 1] - self.sigma[k]) / self.sigma[k - 1])


def canonical_signs(P: np.ndarray, V: np.ndarray):
    """Flip each (P_i, V_i) pair so V_i's largest-|.| entry is positive."""
    P = P.copy()
    V = V.copy()
    for j in range(V.shape[1]):
        idx = int(np.argmax(np.abs(V[:, j])))     # first index on ties
        if V[idx, j] < 0:
            V[:, j] = -V[:, j]
            P[:, j] = -P[:, j]
    return P, V


def factor_block(B: np.ndarray, k: int) -> BlockFactors:
    """Step 4: full SVD by Jacobi, then keep the k largest (Eq. 1)."""
    mb, nb = B.shape
    s_b = min(mb, nb)
    keff = max(0, min(k, s_b))
    if s_b == 0:
        return BlockFactors(0, np.zeros(0), np.zeros((mb, 0)),
                            np.zeros((nb, 0)))
    U, s, V = svd(B)
    P = U[:, :keff] * s[:keff]
    P, Vk = canonical_signs(P, V[:, :keff])
    return BlockFactors(keff, s, P, Vk)


def block_entries(part: Partition, b: int):
    """Local rows, columns and FP64 centred values x - mu_b of block b's
    training ratings (step 3 without forming the dense matrix)."""
    sel = part.block == b
    return part.r[sel], part.c[sel], part.x[sel] - part.mu64[b]


def factor_block_gram(part: Partition, b: int, k: int) -> BlockFactors:
    """Step 4 for blocks too large for the Jacobi routine (a 92,840 x 4,619
    block would take hours): the same truncated SVD (Eq. 1) through the
    symmetric eigenproblem of the block's shorter side. The squared singular
    values of B are the eigenvalues of G = B^T B (items side, when
    n_b <= m_b) or G = B B^T (users side), and the eigenvectors of G are the
    singular vectors of that side.

    Steps, all in float64: G from the block's observed entries (a sparse
    product; unobserved cells are 0 after centring); the k_eff + 1 largest
    eigenpairs of G by LAPACK's symmetric eigensolver; sigma_i =
    sqrt(max(lambda_i, 0)), descending; the other side's factor by one
    product with B (P = B V when V is the eigenvector side, else
    P = U S and V = B^T U S^-1). A singular value sigma_i has absolute error
    about eps * sigma_1^2 / sigma_i, far below the tolerances the GPU path
    is held to for the retained values. ``sigma`` holds only the k_eff + 1
    largest values (enough for the gap), not all min(m_b, n_b).
    """
    import scipy.linalg
    import scipy.sparse
    mb, nb = part.grid.block_shape(b)
    s_b = min(mb, nb)
    keff = max(0, min(k, s_b))
    if s_b == 0:
        return BlockFactors(0, np.zeros(0), np.zeros((mb, 0)),
                            np.zeros((nb, 0)))
    r, c, v = block_entries(part, b)
    B = scipy.sparse.csr_matrix((v, (r, c)), shape=(mb, nb))
    items_side = nb <= mb
    G = (B.T @ B) if items_side else (B @ B.T)
    G = np.asarray(G.toarray(), np.float64)
    want = min(keff + 1, s_b)
    lam, W = scipy.linalg.eigh(G, subset_by_index=[s_b - want, s_b - 1])
    lam, W = lam[::-1], W[:, ::-1]          # descending
    sigma = np.sqrt(np.maximum(lam, 0.0))
    Ws = W[:, :keff]
    if items_side:
        V = Ws
        P = np.asarray(B @ V)
    else:
        sk = sigma[:keff]
        P = Ws * sk
        V = np.asarray(B.T @ Ws)
        nz = sk > 0
        V[:, nz] /= sk[nz]
        V[:, ~nz] = 0.0
    P, V = canonical_signs(P, V)
    return BlockFactors(keff, sigma, P, V)


def factor_gram(part: Partition, k: int, blocks=None,
                threads: int | None = None) -> Model:
    """factor_block_gram for every block (or the listed ones)."""
    ids = list(range(part.grid.p * part.grid.q)) if blocks is None else list(
        blocks)
    threads = threads or os.cpu_count() or 1
    out = {}
    if threads == 1 or len(ids) == 1:
        for b in ids:
            out[b] = factor_block_gram(part, b, k)
    else:
        with _cf.ThreadPoolExecutor(max_workers=threads) as ex:
            for b, f in zip(ids, ex.map(
                    lambda b: factor_block_gram(part, b, k), ids)):
                out[b] = f
    return Model(part, k, out)


@dataclasses.dataclass
class Model:
    part: Partition
    k: int
    blocks: dict             # block id -> BlockFactors


def factor(part: Partition, k: int, blocks=None, threads: int | None = None
           ) -> Model:
    """Step 4 for every block (or the listed ones), blocks in parallel."""
    ids = list(range(part.grid.p * part.grid.q)) if blocks is None else list(
        blocks)
    threads = threads or os.cpu_count() or 1

    def one(b):
        return b, factor_block(dense_block(part, b), k)
    out = {}
    if threads == 1 or len(ids) == 1:
        for b in ids:
            out[b] = one(b)[1]
    else:
        # ctypes drops the GIL during the C call, so threads run in parallel
        with _cf.ThreadPoolExecutor(max_workers=threads) as ex:
            for b, f in ex.map(one, ids):
                out[b] = f
    return Model(part, k, out)


def predict(model: Model, u, i, clamp: tuple[float, float] | None = None
            ) -> np.ndarray:
    """Step 5: y_hat = mu_b + P[r] . V[c] for each query (Eq. 2)."""
    b, r, c = model.part.grid.locate(u, i)
    y = model.part.mu64[b].copy()
    for blk in np.unique(b):
        if int(blk) not in model.blocks:
            raise KeyError("block %d was not factorised" % blk)
        f = model.blocks[int(blk)]
        sel = b == blk
        y[sel] += np.einsum("ij,ij->i", f.P[r[sel]], f.V[c[sel]])
    if clamp is not None:
        y = np.clip(y, clamp[0], clamp[1])
    return y


def reconstruct(model: Model, b: int, add_mean: bool = True) -> np.ndarray:
    """Rank-k reconstruction P V^T of block b (+ mu_b)."""
    f = model.blocks[b]
    R = f.P @ f.V.T
    return R + model.part.mu64[b] if add_mean else R


def rmse(model: Model, u, i, y, clamp=None) -> float:
    """Step 6: sqrt(sum (y_hat - y)^2 / count), the sum taken exactly."""
    y = np.asarray(y, np.float32).astype(np.float64)
    if y.size == 0:
        raise ValueError("RMSE of an empty set")
    d = predict(model, u, i, clamp) - y
    return math.sqrt(math.fsum((d * d).tolist()) / y.size)
