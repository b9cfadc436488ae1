"""Multi-GPU helpers for the block-SVD path (host side).

Blocks are independent on this path: a block's factorisation needs only its
own ratings. So blocks shard across ranks with no data exchange: each rank
holds its longest-processing-time share of the blocks (bsvd_set_owned), and
the library partitions and factorises only those. The only cross-rank
reductions are the held-out error (the RMSE of Section 5 sums squared
errors over every block's held-out ratings: one all-reduce of the sum and
the count) and the benchmark's max-over-ranks time. Everything here uses
torch.distributed collectives on whatever backend the caller initialised
(NCCL on GPUs, gloo on CPUs).
"""
from __future__ import annotations

import math

import torch


def block_costs(shapes) -> list:
    """Work of each block's Gram: L s^2 for a block with sides s <= L."""
    return [float(L) * s * s for (s, L) in shapes]


def assign_blocks(costs, world: int) -> list:
    """Longest-processing-time-first assignment of blocks to ranks.

    Blocks are taken by decreasing cost (ties: lower id first) and each
    goes to the currently least loaded rank (ties: lower rank). Returns one
    sorted list of block ids per rank.
    """
    if world < 1:
        raise ValueError("world must be >= 1")
    order = sorted(range(len(costs)), key=lambda b: (-costs[b], b))
    load = [0.0] * world
    parts = [[] for _ in range(world)]
    for b in order:
        r = min(range(world), key=lambda j: (load[j], j))
        parts[r].append(b)
        load[r] += costs[b]
    return [sorted(p) for p in parts]


def owned_mask(costs, world: int, rank: int):
    """This rank's blocks under assign_blocks, as a 0/1 list (one flag per
    block) for Context.set_owned."""
    mine = set(assign_blocks(costs, world)[rank])
    return [1 if b in mine else 0 for b in range(len(costs))]


def _device(group=None):
    backend = torch.distributed.get_backend(group)
    return torch.device("cuda", torch.cuda.current_device()) \
        if backend == "nccl" else torch.device("cpu")


def max_over_ranks(value: float, group=None) -> float:
    t = torch.tensor([value], dtype=torch.float64, device=_device(group))
    torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX,
                                 group=group)
    return float(t.item())


def rmse_from_parts(sqerr_sum: float, count: int, group=None) -> float:
    """sqrt(sum of every rank's squared errors / total held-out count)."""
    dev = _device(group)
    s = torch.tensor([sqerr_sum], dtype=torch.float64, device=dev)
    n = torch.tensor([count], dtype=torch.int64, device=dev)
    torch.distributed.all_reduce(s, group=group)
    torch.distributed.all_reduce(n, group=group)
    total = int(n.item())
    if total == 0:
        raise ValueError("RMSE of an empty set")
    return math.sqrt(float(s.item()) / total)


def sharded_rmse(ctx, u, i, y, group=None) -> float:
    """RMSE over all ranks' held-out ratings: each rank sums the squared
    errors of the queries in its own blocks (Context.sqerr), then one
    all-reduce combines the sums and the counts."""
    s, n = ctx.sqerr(u, i, y)
    return rmse_from_parts(s, n, group)
