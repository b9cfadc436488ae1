"""Uneven block grids cut at rating-activity quantiles (host side).

The paper's grid uses equal blocks (Section 3, Eq. "datax"). On long-tailed
data that leaves a few blocks holding most ratings. The batched form
instead orders users (items) by their number of training ratings,
busiest first (ties: lower id first), and cuts the order where the running
count of ratings crosses g/p (g/q) of the total. Each block row (column)
then holds about the same number of ratings, and the blocks have uneven
shapes. The result plugs into bsvd_partition as row_perm + row_bounds and
col_perm + col_bounds.
"""
from __future__ import annotations

import numpy as np


def quantile_split(ids: np.ndarray, size: int, parts: int):
    """Permutation (id -> position) and parts + 1 bounds for one side.

    Bound g (0 < g < parts) is the first position j whose preceding
    positions hold at least g / parts of the ratings, i.e. the smallest j
    with parts * C_j >= g * N in exact integers, where C_j is the number of
    ratings of the first j ids in the order.
    """
    if parts < 1 or size < parts:
        raise ValueError("need 1 <= parts <= size")
    counts = np.bincount(np.asarray(ids, np.int64), minlength=size)
    order = np.lexsort((np.arange(size), -counts))     # busiest first
    perm = np.empty(size, np.int32)
    perm[order] = np.arange(size, dtype=np.int32)
    cum = np.concatenate([[0], np.cumsum(counts[order], dtype=np.int64)])
    total = int(cum[-1])
    bounds = np.empty(parts + 1, np.int64)
    bounds[0], bounds[parts] = 0, size
    for g in range(1, parts):
        j = int(np.searchsorted(cum * parts, g * total, side="left"))
        bounds[g] = min(max(j, bounds[g - 1]), size)
    return perm, bounds


def quantile_grid(u: np.ndarray, i: np.ndarray, m: int, n: int, p: int,
                  q: int) -> dict:
    """Keyword arguments for bsvd_partition / Context.partition."""
    row_perm, row_bounds = quantile_split(u, m, p)
    col_perm, col_bounds = quantile_split(i, n, q)
    return dict(row_bounds=row_bounds, col_bounds=col_bounds,
                row_perm=row_perm, col_perm=col_perm)
