"""The allocation-free block-means entry point against bsvd_partition and
the oracle.

bsvd_block_means_noalloc serves callers that cannot allocate device memory
during a call (a process whose device memory all belongs to its own pool,
or a loop whose memory is fixed up front): its scratch is a fixed device
array inside the library. Its counts and means must equal, bit for bit,
what the context-based partition reports and what the FP64 oracle's
partition computes (exact sums over float64, rounded to float32), on
consecutive calls (a later call must not see an earlier call's sums).
"""
import numpy as np
import pytest

import oracle
import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_1907_07410_gb300 as bs  # noqa: E402


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def via_noalloc(r, p, q):
    counts = torch.full((p * q,), -1, dtype=torch.int64, device="cuda")
    mu = torch.full((p * q,), -1.0, dtype=torch.float32, device="cuda")
    st = bs.bsvd_block_means_noalloc(r.m, r.n, dev(r.u_train),
                                     dev(r.i_train), dev(r.x_train), p, q,
                                     counts, mu,
                                     torch.cuda.current_stream())
    assert st == bs.OK
    return counts.cpu().numpy(), mu.cpu().numpy()


def via_partition(r, p, q):
    ctx = bs.Context()
    ctx.partition(r.m, r.n, dev(r.u_train), dev(r.i_train), dev(r.x_train),
                  p, q)
    counts, mu = ctx.block_stats()
    ctx.close()
    return counts, mu


def test_noalloc_matches_partition_on_consecutive_calls():
    cases = [(synth.generate(synth.MEDIUM), 4, 4),
             (synth.generate(synth.SMALL), 2, 2),
             (synth.random_ratings(3, 500, 300, 20000, 0), 40, 30),
             (synth.random_ratings(5, 600, 500, 30000, 0), 60, 50)]
    for r, p, q in cases:
        c1, m1 = via_noalloc(r, p, q)
        c2, m2 = via_partition(r, p, q)
        assert np.array_equal(c1, c2)
        assert np.array_equal(m1.view(np.uint32), m2.view(np.uint32))
        part = oracle.partition(r.m, r.n, r.u_train, r.i_train, r.x_train,
                                p, q)
        assert np.array_equal(c1, part.counts)
        assert np.array_equal(m1.view(np.uint32), part.mu32.view(np.uint32))


def test_noalloc_rejects_oversized_grid_and_host_memory():
    r = synth.random_ratings(4, 200, 200, 1000, 0)
    counts = torch.zeros(65 * 65, dtype=torch.int64, device="cuda")
    mu = torch.zeros(65 * 65, dtype=torch.float32, device="cuda")
    assert bs.bsvd_block_means_noalloc(r.m, r.n, dev(r.u_train),
                                       dev(r.i_train), dev(r.x_train), 65,
                                       65, counts, mu) == bs.EINVAL
    assert bs.bsvd_block_means_noalloc(r.m, r.n, r.u_train, r.i_train,
                                       r.x_train, 2, 2, counts[:4],
                                       mu[:4]) == bs.EINVAL
    # outputs shorter than p * q are refused before the library is called
    with pytest.raises(ValueError):
        bs.bsvd_block_means_noalloc(r.m, r.n, dev(r.u_train), dev(r.i_train),
                                    dev(r.x_train), 2, 2, counts[:3], mu[:4])
