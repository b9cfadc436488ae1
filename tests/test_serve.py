"""Admission and batching logic of the continuous-batching server, on the
CPU with a fake backend (no device): FIFO order, the batch cap, the memory
budget counted over what every worker's context holds, context resets under
memory pressure, oversized requests and errors handed to the caller."""
import threading
import time

import numpy as np
import pytest

from paper_1907_07410_gb300 import serve


class FakeCtx:
    made = 0
    lock = threading.Lock()

    def __init__(self):
        with FakeCtx.lock:
            FakeCtx.made += 1
        self.closed = False

    def close(self):
        self.closed = True


class Recorder:
    """Runner that checks the budget invariant while batches run."""

    def __init__(self, server_ref, delay=0.01, fail_on=None):
        self.server_ref = server_ref
        self.delay = delay
        self.fail_on = fail_on
        self.active = 0
        self.max_active = 0
        self.lock = threading.Lock()
        self.violations = []

    def __call__(self, ctx, reqs):
        assert not ctx.closed
        srv = self.server_ref[0]
        with self.lock:
            self.active += 1
            self.max_active = max(self.max_active, self.active)
            if sum(srv.held) > srv.budget:
                self.violations.append(sum(srv.held))
        time.sleep(self.delay)
        with self.lock:
            self.active -= 1
        if self.fail_on is not None and any(r.rid == self.fail_on
                                            for r in reqs):
            raise RuntimeError("planted failure")
        return [np.full(len(r.qr), r.rid, np.float32) for r in reqs]


def request(m, n, nnz=10, nq=3):
    cells = np.arange(nnz)
    return serve.Request(m, n, 10, (cells // n).astype(np.int32),
                         (cells % n).astype(np.int32),
                         np.full(nnz, 3.0, np.float32),
                         np.zeros(nq, np.int32), np.zeros(nq, np.int32))


def make(workers, max_batch, budget, **kw):
    ref = [None]
    rec = Recorder(ref, **kw)
    srv = serve.Server(workers=workers, max_batch=max_batch,
                       hbm_budget=budget, context_factory=FakeCtx,
                       runner=rec)
    ref[0] = srv
    return srv, rec


def test_results_fifo_and_batch_cap():
    fp = serve.footprint(100, 50, 10, 3)
    srv, rec = make(workers=3, max_batch=4, budget=1000 * fp)
    futs = [srv.submit(request(100, 50)) for _ in range(40)]
    res = [f.result(timeout=30) for f in futs]
    srv.close()
    for k, r in enumerate(res):
        assert r.rid == k
        assert np.all(r.yhat == k)
        assert r.latency >= 0
    order = [rid for ids, _ in srv.batches for rid in ids]
    assert order == list(range(40))
    assert max(len(ids) for ids, _ in srv.batches) <= 4
    assert sum(len(ids) for ids, _ in srv.batches) == 40
    assert not rec.violations


def test_budget_bounds_what_contexts_hold():
    fp = serve.footprint(100, 50, 10, 3)
    srv, rec = make(workers=4, max_batch=8, budget=int(2.5 * fp))
    futs = [srv.submit(request(100, 50)) for _ in range(30)]
    for f in futs:
        f.result(timeout=30)
    srv.close()
    assert srv.max_held <= srv.budget
    assert not rec.violations
    # at most two requests' worth of memory can be held at once
    assert max(len(ids) for ids, _ in srv.batches) <= 2
    for ids, need in srv.batches:
        assert need == fp * len(ids)


def test_idle_workers_release_memory_for_a_large_request():
    small = serve.footprint(100, 50, 10, 3)
    big = serve.footprint(2000, 1000, 10, 3)
    budget = big + small // 2
    FakeCtx.made = 0
    srv, rec = make(workers=3, max_batch=1, budget=budget, delay=0.02)
    # warm every worker with small requests, then ask for the large one
    warm = [srv.submit(request(100, 50)) for _ in range(6)]
    for f in warm:
        f.result(timeout=30)
    fb = srv.submit(request(2000, 1000))
    fb.result(timeout=30)
    srv.close()
    assert not rec.violations
    assert srv.max_held <= budget
    assert srv.resets >= 1
    assert FakeCtx.made == 3 + srv.resets


def test_oversized_request_fails_at_submit():
    srv, _ = make(workers=1, max_batch=4, budget=1000)
    f = srv.submit(request(100, 50))
    with pytest.raises(ValueError, match="budget"):
        f.result(timeout=5)
    srv.close()
    assert srv.batches == []


def test_runner_error_reaches_every_caller_in_the_batch():
    fp = serve.footprint(100, 50, 10, 3)
    srv, _ = make(workers=1, max_batch=64, budget=1000 * fp, delay=0.05,
                  fail_on=2)
    futs = [srv.submit(request(100, 50)) for _ in range(6)]
    errs = 0
    for f in futs:
        try:
            f.result(timeout=30)
        except RuntimeError:
            errs += 1
    srv.close()
    failing = [ids for ids, _ in srv.batches if 2 in ids][0]
    assert errs == len(failing)


def test_footprint_grows_with_the_block():
    a = serve.footprint(100, 50, 10)
    assert serve.footprint(200, 50, 10) > a
    assert serve.footprint(100, 100, 10) > a
    assert serve.footprint(100, 50, 1000) == a + 12 * 990
    # shape, not orientation, decides
    assert serve.footprint(50, 100, 10) == a


def test_request_from_dense():
    d = np.zeros((3, 4), np.float32)
    d[0, 1], d[2, 3], d[1, 0] = 5, 2, 4
    q = serve.Request.from_dense(d, 2, [0], [0])
    assert (q.m, q.n, q.k, q.nnz) == (3, 4, 2, 3)
    assert q.r.tolist() == [0, 1, 2] and q.c.tolist() == [1, 0, 3]
    assert q.x.tolist() == [5, 4, 2]
    assert q.qr.dtype == np.int32
