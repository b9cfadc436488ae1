"""Multi-GPU helpers for the block-SVD path (host side).

Blocks are independent on this path: a block's factorisation needs only its
own ratings. So blocks shard across ranks with no data exchange. The only
cross-rank reductions are the held-out error (the RMSE of Section 5 sums
squared errors over every block's held-out ratings) and the benchmark's
max-over-ranks time. Everything here uses torch.distributed collectives on
whatever backend the caller initialised (NCCL on GPUs, gloo on CPUs).
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
