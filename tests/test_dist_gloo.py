"""Multi-rank host logic with gloo on CPU (world size 2).

Blocks shard across ranks with no data exchange; the held-out RMSE is the
only cross-rank reduction. A sharded run (each rank factorises its blocks
with the FP64 oracle and sums the squared errors of the held-out ratings in
those blocks) must give the single-process RMSE, and the benchmark's
max-over-ranks time must be the largest rank time.
"""
import math
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

import oracle
import synth
from paper_1907_07410_gb300 import dist as bdist


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        w = synth.SMALL
        r = synth.generate(w)
        part = oracle.partition(w.m, w.n, r.u_train, r.i_train, r.x_train,
                                w.p, w.q)
        shapes = []
        for b in range(w.p * w.q):
            mb, nb = part.grid.block_shape(b)
            shapes.append((min(mb, nb), max(mb, nb)))
        mine = bdist.assign_blocks(bdist.block_costs(shapes), world)[rank]
        model = oracle.factor(part, w.k, blocks=mine, threads=2)
        b, _, _ = part.grid.locate(r.u_test, r.i_test)
        sel = np.isin(b, mine)
        yhat = oracle.predict(model, r.u_test[sel], r.i_test[sel])
        d = yhat - r.x_test[sel].astype(np.float64)
        sq = math.fsum((d * d).tolist())
        rmse = bdist.rmse_from_parts(sq, int(sel.sum()))
        t_max = bdist.max_over_ranks(float(rank + 1))
        out[rank] = (mine, rmse, t_max)
    finally:
        dist.destroy_process_group()


def test_sharded_rmse_and_timing_with_gloo():
    world = 2
    port = _free_port()
    manager = mp.get_context("spawn").Manager()
    out = manager.dict()
    mp.start_processes(_worker, args=(world, port, out), nprocs=world,
                       join=True, start_method="spawn")
    w = synth.SMALL
    r = synth.generate(w)
    part = oracle.partition(w.m, w.n, r.u_train, r.i_train, r.x_train, w.p,
                            w.q)
    want = oracle.rmse(oracle.factor(part, w.k), r.u_test, r.i_test,
                       r.x_test)
    blocks = sorted(out[0][0] + out[1][0])
    assert blocks == list(range(w.p * w.q))
    for rank in range(world):
        assert abs(out[rank][1] - want) < 1e-12
        assert out[rank][2] == float(world)


def test_assign_blocks_balances_and_covers():
    costs = [5.0, 1.0, 4.0, 4.0, 3.0, 2.0, 2.0, 1.0]
    parts = bdist.assign_blocks(costs, 3)
    flat = sorted(b for p in parts for b in p)
    assert flat == list(range(len(costs)))
    loads = [sum(costs[b] for b in p) for p in parts]
    # LPT bound: max load <= 4/3 - 1/(3m) of the optimum (>= total / m)
    assert max(loads) <= (4 / 3 - 1 / 9) * max(sum(costs) / 3, max(costs)) + 1e-9
    with pytest.raises(ValueError):
        bdist.assign_blocks(costs, 0)


def _gpu_worker(rank, world, port, out):
    """One shard on cuda:0: the library holds and factorises this rank's
    LPT share of the uneven workload's 32 blocks."""
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import paper_1907_07410_gb300 as bs
        torch.cuda.set_device(0)
        w = synth.UNEVEN
        r = synth.generate(w)
        ctx = bs.Context()
        kw = ctx.quantile_grid(w.m, w.n, r.u_train, r.i_train, w.p, w.q)
        rb, cb = kw["row_bounds"], kw["col_bounds"]
        shapes = [(min(rb[b // w.q + 1] - rb[b // w.q],
                       cb[b % w.q + 1] - cb[b % w.q]),
                   max(rb[b // w.q + 1] - rb[b // w.q],
                       cb[b % w.q + 1] - cb[b % w.q]))
                  for b in range(w.p * w.q)]
        mask = bdist.owned_mask(bdist.block_costs(shapes), world, rank)
        ctx.set_owned(mask)
        ctx.partition(w.m, w.n, r.u_train, r.i_train, r.x_train, w.p, w.q,
                      **kw)
        assert ctx.factor(w.k) == bs.OK
        rmse = bdist.sharded_rmse(ctx, r.u_test, r.i_test, r.x_test)
        mine = [b for b in range(w.p * w.q) if mask[b]]
        sig = {b: ctx.get_block(b)["sigma"].tolist() for b in mine}
        other = next(b for b in range(w.p * w.q) if not mask[b])
        out[rank] = (mine, rmse, sig, ctx.get_block(other)["keff"])
        ctx.close()
    finally:
        dist.destroy_process_group()


@pytest.mark.gpu
def test_sharded_library_on_one_gpu_with_gloo():
    """Two gloo ranks share cuda:0, each factorising its own blocks through
    libbsvd (no kernel of one rank waits on the other). Every block lands on
    exactly one rank, each block's singular values equal the single-process
    run's bit for bit, and the combined RMSE equals the single-process RMSE
    within 1e-12."""
    import paper_1907_07410_gb300 as bs
    world = 2
    port = _free_port()
    manager = mp.get_context("spawn").Manager()
    out = manager.dict()
    mp.start_processes(_gpu_worker, args=(world, port, out), nprocs=world,
                       join=True, start_method="spawn")
    w = synth.UNEVEN
    r = synth.generate(w)
    ctx = bs.Context()
    kw = ctx.quantile_grid(w.m, w.n, r.u_train, r.i_train, w.p, w.q)
    ctx.partition(w.m, w.n, r.u_train, r.i_train, r.x_train, w.p, w.q, **kw)
    assert ctx.factor(w.k) == bs.OK
    want = ctx.rmse(r.u_test, r.i_test, r.x_test)
    s_all, n_all = ctx.sqerr(r.u_test, r.i_test, r.x_test)
    assert n_all == r.u_test.size
    assert abs(np.sqrt(s_all / n_all) - want) <= 1e-15 * want
    blocks = sorted(out[0][0] + out[1][0])
    assert blocks == list(range(w.p * w.q))
    for rank in range(world):
        mine, rmse, sig, keff_other = out[rank]
        assert abs(rmse - want) <= 1e-12
        assert keff_other == 0
        for b in mine:
            assert sig[b] == ctx.get_block(b)["sigma"].tolist(), b
    ctx.close()
