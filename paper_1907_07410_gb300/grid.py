"""Uneven block grids cut at rating-activity quantiles.

The paper's grid uses equal blocks (Section 3, Eq. "datax"). On long-tailed
data that leaves a few blocks holding most ratings. The batched form
instead orders users (items) by their number of training ratings, busiest
first (ties: lower id first), and cuts the order where the running count of
ratings first reaches g/p (g/q) of the total. Each block row (column) then
holds about the same number of ratings, and the blocks have uneven shapes.

The cut runs in the CUDA library (bsvd_quantile_grid); this module only
wraps the call. The result plugs into bsvd_partition as row_perm +
row_bounds and col_perm + col_bounds.
"""
from __future__ import annotations


def quantile_grid(u, i, m: int, n: int, p: int, q: int, ctx=None) -> dict:
    """Keyword arguments for bsvd_partition / Context.partition, computed by
    the library on the current CUDA device. ``ctx``: a Context to run on
    (a temporary one when None)."""
    import paper_1907_07410_gb300 as bs
    own = ctx is None
    if own:
        ctx = bs.Context()
    try:
        return ctx.quantile_grid(m, n, u, i, p, q)
    finally:
        if own:
            ctx.close()
