"""Seeded synthetic rating workloads shaped like the paper's datasets.

This module is shared by the tests, the benchmark and the oracle. It holds
only input generation: no step of the block-SVD method (no partition, no
mean, no factorisation) lives here.

The paper evaluates on MovieLens-100K/1M/10M/20M and Jester (Section 5).
Those datasets are not available, so these generators stand in for them with
the same shapes, rating scale and long-tailed user/item activity:

  * users are ranked in a random order and user r gets weight r^-s_user;
    every user has at least ``min_per_user`` ratings and the rest are shared
    in proportion to the weights (largest-remainder rounding), capped at n
    per user by water-filling;
  * each user's items are drawn without replacement with probability
    proportional to an item popularity weight (uniform, or rank^-s_item over
    a random item order);
  * rating = clamp(round_half_away(3.5 + u.v + eps), 1, 5) with latent
    u, v ~ N(0, 0.3^2 I_d) and eps ~ N(0, 0.8^2);
  * a seeded permutation puts the first floor(held_out_frac * N) ratings in
    the held-out set.

Everything is drawn from numpy's PCG64 with a fixed seed per workload.
"""
from __future__ import annotations

import dataclasses
import hashlib
import math
import os
import tempfile

import numpy as np

SEED_BASE = 1907074100


@dataclasses.dataclass(frozen=True)
class Workload:
    """Shape of one synthetic rating matrix and its block grid."""
    name: str
    m: int                 # users
    n: int                 # items
    nnz: int               # total ratings (train + held-out)
    d: int                 # latent rank of the generating model
    s_user: float          # Zipf exponent of user activity
    s_item: float | None   # Zipf exponent of item popularity (None = uniform)
    p: int                 # block rows
    q: int                 # block columns
    k: int                 # retained rank
    seed_index: int
    min_per_user: int = 20
    held_out_frac: float = 0.1
    grid: str = "equal"    # "equal" blocks or "quantile" (activity) cuts

    @property
    def seed(self) -> int:
        return SEED_BASE + self.seed_index


# The workloads. "small" is MovieLens-100K shaped, "medium" MovieLens-1M
# shaped; the precision grids reuse the medium matrix; "large" is
# Netflix-prize shaped.
SMALL = Workload("small-943x1682-2x2-k10", 943, 1682, 100_000, 10, 1.1, None,
                 2, 2, 10, 0)
MEDIUM = Workload("medium-6040x3952-4x4-k20", 6040, 3952, 1_000_209, 20, 1.0,
                  1.0, 4, 4, 20, 1)
MEDIUM_8x8 = dataclasses.replace(MEDIUM, name="medium-6040x3952-8x8-k20",
                                 p=8, q=8)
MEDIUM_16x16 = dataclasses.replace(MEDIUM, name="medium-6040x3952-16x16-k20",
                                   p=16, q=16)
LARGE = Workload("large-480189x17770-32x8-k40", 480_189, 17_770, 100_480_507,
                 40, 1.2, 0.9, 32, 8, 40, 3, grid="quantile")

# A mid-size long-tailed matrix for the uneven (activity-quantile) grid,
# small enough for the oracle to factorise every block.
UNEVEN = Workload("uneven-20000x3000-8x4-k40", 20_000, 3_000, 1_500_000, 40,
                  1.2, 0.9, 8, 4, 40, 4, grid="quantile")

# The large workload's generator at a tenth of its ratings, for kernel
# profiles that must fit a few GB of device memory (blocks up to about
# 30,000 x 5,000; every Gram and dense copy still exceeds the 129 MB L2).
MID = Workload("mid-120000x8000-16x4-k40", 120_000, 8_000, 12_000_000, 40,
               1.2, 0.9, 16, 4, 40, 5, grid="quantile")

WORKLOADS = {w.name: w for w in (SMALL, MEDIUM, MEDIUM_8x8, MEDIUM_16x16,
                                 LARGE, UNEVEN, MID)}


@dataclasses.dataclass
class Ratings:
    """COO ratings split into train and held-out parts (0-based ids)."""
    m: int
    n: int
    u_train: np.ndarray    # int32
    i_train: np.ndarray    # int32
    x_train: np.ndarray    # float32
    u_test: np.ndarray
    i_test: np.ndarray
    x_test: np.ndarray

    def digest(self) -> str:
        h = hashlib.sha256()
        for a in (self.u_train, self.i_train, self.x_train, self.u_test,
                  self.i_test, self.x_test):
            h.update(np.ascontiguousarray(a).tobytes())
        return h.hexdigest()


def _largest_remainder(total: int, weights: np.ndarray) -> np.ndarray:
    """Integer shares of ``total`` proportional to ``weights``."""
    if total <= 0 or weights.size == 0:
        return np.zeros(weights.shape, np.int64)
    exact = total * (weights / weights.sum())
    base = np.floor(exact).astype(np.int64)
    rest = total - int(base.sum())
    if rest > 0:
        frac = exact - base
        # stable: ties go to the lower index
        order = np.argsort(-frac, kind="stable")[:rest]
        base[order] += 1
    return base


def user_counts(rng: np.random.Generator, m: int, n: int, nnz: int,
                s_user: float, min_per_user: int) -> np.ndarray:
    """Ratings per user: Zipf over a random user ranking, floor and cap."""
    if min_per_user * m > nnz or nnz > m * n:
        raise ValueError("infeasible workload shape")
    rank_of_user = rng.permutation(m)           # user -> rank 0..m-1
    w = (rank_of_user + 1.0) ** (-s_user)
    floor = min(min_per_user, n)
    counts = np.full(m, floor, np.int64)
    remaining = nnz - int(counts.sum())
    free = np.ones(m, bool)
    # water-filling: share, cap at n, re-share the excess among the rest
    while remaining > 0:
        share = _largest_remainder(remaining, np.where(free, w, 0.0))
        new = counts + share
        over = new > n
        if not over.any():
            counts = new
            remaining = 0
            break
        remaining -= int((n - counts[over]).sum())
        counts[over] = n
        free &= ~over
        # users not capped keep their old counts; redo the share next round
    return counts


def _item_weights(rng: np.random.Generator, n: int,
                  s_item: float | None) -> np.ndarray:
    if s_item is None:
        return np.ones(n)
    rank_of_item = rng.permutation(n)
    return (rank_of_item + 1.0) ** (-s_item)


def _sorted_unique(a: np.ndarray) -> np.ndarray:
    a = np.sort(a)
    if a.size == 0:
        return a
    return a[np.concatenate([[True], a[1:] != a[:-1]])]


def sample_items(rng: np.random.Generator, counts: np.ndarray, n: int,
                 w_item: np.ndarray) -> tuple[np.ndarray, np.ndarray]:
    """Distinct items per user, drawn with probability proportional to w_item.

    Users with count <= n/8 draw with replacement and drop repeats until they
    have enough (dropping repeats is sampling without replacement); denser
    users take the ``count`` smallest exponential keys -log(U)/w.
    """
    m = counts.size
    prob = w_item / w_item.sum()
    cdf = np.cumsum(prob)
    cdf[-1] = 1.0
    users_out, items_out = [], []

    dense = np.nonzero(counts > n // 8)[0]
    for u in dense:
        c = int(counts[u])
        if c == n:
            it = np.arange(n, dtype=np.int64)
        else:
            keys = -np.log(rng.random(n)) / w_item
            it = np.sort(np.argpartition(keys, c - 1)[:c])
        users_out.append(np.full(c, u, np.int64))
        items_out.append(it)

    active = np.nonzero(counts <= n // 8)[0]
    need = counts[active].copy()
    rounds = []            # sorted, disjoint key sets, one per round
    while active.size:
        draw_u = np.repeat(active, need)
        draw_i = np.searchsorted(cdf, rng.random(draw_u.size), side="right")
        key = draw_u * n + np.minimum(draw_i, n - 1)
        key = _sorted_unique(key)
        # each user drew `need` times, so it cannot overshoot its deficit
        for h in rounds:
            if key.size == 0 or h.size == 0:
                continue
            pos = np.searchsorted(h, key)
            pos[pos == h.size] = 0
            key = key[h[pos] != key]
        rounds.append(key)
        got = np.bincount(key // n, minlength=m)
        need = need - got[active]
        keep = need > 0
        active, need = active[keep], need[keep]
    have = (np.sort(np.concatenate(rounds)) if rounds
            else np.zeros(0, np.int64))
    users_out.append(have // n)
    items_out.append(have % n)
    uu = np.concatenate(users_out)
    ii = np.concatenate(items_out)
    order = np.lexsort((ii, uu))
    return uu[order], ii[order]


def _round_half_away(v: np.ndarray) -> np.ndarray:
    return np.sign(v) * np.floor(np.abs(v) + 0.5)


def ratings_from_latent(rng: np.random.Generator, m: int, n: int, d: int,
                        uu: np.ndarray, ii: np.ndarray,
                        chunk: int = 1 << 22) -> np.ndarray:
    """clamp(round_half_away(3.5 + u.v + eps), 1, 5) per (user, item) pair."""
    U = rng.normal(0.0, 0.3, size=(m, d))
    V = rng.normal(0.0, 0.3, size=(n, d))
    x = np.empty(uu.size, np.float32)
    sub = 1 << 16          # gather rows in small pieces (less temporary memory)
    for s in range(0, uu.size, chunk):
        e = min(uu.size, s + chunk)
        dots = np.empty(e - s)
        for a in range(s, e, sub):
            z = min(e, a + sub)
            dots[a - s:z - s] = np.einsum("ij,ij->i", U[uu[a:z]], V[ii[a:z]])
        eps = rng.normal(0.0, 0.8, size=e - s)
        x[s:e] = np.clip(_round_half_away(3.5 + dots + eps), 1, 5)
    return x


# Workloads at least this large are cached on disk between processes.
CACHE_MIN_NNZ = 10_000_000


def _cache_path(w: Workload) -> str:
    root = os.environ.get("BSVD_SYNTH_CACHE") or os.path.join(
        tempfile.gettempdir(), "bsvd_synth_cache")
    with open(__file__, "rb") as f:
        tag = hashlib.sha256(f.read()).hexdigest()[:16]
    return os.path.join(root, "%s-%s.npz" % (w.name, tag))


def generate(w: Workload, cache: bool = True) -> Ratings:
    """The full seeded COO for a workload, split into train and held-out.

    Workloads of CACHE_MIN_NNZ ratings or more are kept in a cache directory
    (``BSVD_SYNTH_CACHE``, else a folder in the system's temporary
    directory), keyed by the workload's name and this file's contents, so
    processes after the first load them instead of drawing them again."""
    path = _cache_path(w) if cache and w.nnz >= CACHE_MIN_NNZ else None
    if path and os.path.exists(path):
        try:
            with np.load(path) as z:
                return Ratings(w.m, w.n, z["u_train"], z["i_train"],
                               z["x_train"], z["u_test"], z["i_test"],
                               z["x_test"])
        except (OSError, KeyError, ValueError):
            pass
    r = _generate(w)
    if path:
        try:
            os.makedirs(os.path.dirname(path), exist_ok=True)
            tmp = path + ".tmp%d.npz" % os.getpid()
            np.savez(tmp, u_train=r.u_train, i_train=r.i_train,
                     x_train=r.x_train, u_test=r.u_test, i_test=r.i_test,
                     x_test=r.x_test)
            os.replace(tmp, path)
        except OSError:
            pass
    return r


def _generate(w: Workload) -> Ratings:
    rng = np.random.Generator(np.random.PCG64(w.seed))
    counts = user_counts(rng, w.m, w.n, w.nnz, w.s_user, w.min_per_user)
    w_item = _item_weights(rng, w.n, w.s_item)
    uu, ii = sample_items(rng, counts, w.n, w_item)
    x = ratings_from_latent(rng, w.m, w.n, w.d, uu, ii)
    perm = rng.permutation(uu.size)
    n_test = int(math.floor(w.held_out_frac * uu.size))
    te, tr = perm[:n_test], perm[n_test:]
    return Ratings(w.m, w.n,
                   uu[tr].astype(np.int32), ii[tr].astype(np.int32), x[tr],
                   uu[te].astype(np.int32), ii[te].astype(np.int32), x[te])


def random_ratings(seed: int, m: int, n: int, nnz_train: int,
                   nnz_test: int, levels: int = 5) -> Ratings:
    """Small uniform random COO without repeated pairs (for edge cases)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    total = nnz_train + nnz_test
    if total > m * n:
        raise ValueError("more ratings than cells")
    cells = rng.choice(m * n, size=total, replace=False)
    uu = (cells // n).astype(np.int32)
    ii = (cells % n).astype(np.int32)
    x = rng.integers(1, levels + 1, size=total).astype(np.float32)
    return Ratings(m, n, uu[:nnz_train], ii[:nnz_train], x[:nnz_train],
                   uu[nnz_train:], ii[nnz_train:], x[nnz_train:])


# The request pool of the served form: 32 requests drawn by served_requests
# with this seed (shapes rows ~U[128, 8192], cols ~U[64, 2048]).
SERVED_POOL_SEED = 20190717
SERVED_POOL_SIZE = 32


def served_requests(seed: int, count: int,
                    ks: tuple[int, ...] = (10, 20, 40),
                    rows: tuple[int, int] = (128, 8192),
                    cols: tuple[int, int] = (64, 2048),
                    density: tuple[float, float] = (0.03, 0.10),
                    d: int = 10, queries: int = 64,
                    dense: bool = True) -> list[dict]:
    """Dense single-block requests for the served form.

    Each request is an m_b x n_b float32 matrix whose zeros mean "missing"
    (``dense``; the same cells as COO in ``r``, ``c``, ``x``), a rank k and
    ``queries`` held-out (row, col, rating) triples taken out of the
    observed cells. Ratings follow the same latent model as ``generate``.
    ``dense=False`` leaves the dense matrix out (None).
    """
    rng = np.random.Generator(np.random.PCG64(seed))
    out = []
    for _ in range(count):
        mb = int(rng.integers(rows[0], rows[1] + 1))
        nb = int(rng.integers(cols[0], cols[1] + 1))
        dens = float(rng.uniform(*density))
        k = int(ks[int(rng.integers(0, len(ks)))])
        nobs = max(queries + 1, int(round(dens * mb * nb)))
        cells = rng.choice(mb * nb, size=nobs, replace=False)
        r = cells // nb
        c = cells % nb
        U = rng.normal(0.0, 0.3, size=(mb, d))
        V = rng.normal(0.0, 0.3, size=(nb, d))
        val = np.clip(_round_half_away(
            3.5 + np.einsum("ij,ij->i", U[r], V[c])
            + rng.normal(0.0, 0.8, size=nobs)), 1, 5).astype(np.float32)
        q = rng.permutation(nobs)[:queries]
        keep = np.ones(nobs, bool)
        keep[q] = False
        full = None
        if dense:
            full = np.zeros((mb, nb), np.float32)
            full[r[keep], c[keep]] = val[keep]
        out.append(dict(m=mb, n=nb, k=k, dense=full,
                        r=r[keep].astype(np.int32), c=c[keep].astype(np.int32),
                        x=val[keep],
                        qr=r[q].astype(np.int32), qc=c[q].astype(np.int32),
                        qy=val[q]))
    return out


def sgd_start(m: int, n: int, k: int, seed: int = 13):
    """Starting factors of the blocked SGD: P0 (m x k) and Q0 (n x k), float64,
    entries N(0, 0.1^2). The paper only says the latent feature matrices
    start from random values; the distribution and scale are this module's
    choice."""
    rng = np.random.Generator(np.random.PCG64(seed))
    return (rng.normal(0.0, 0.1, size=(m, k)),
            rng.normal(0.0, 0.1, size=(n, k)))
