"""Continuous-batching server for factorise-then-predict requests.

A request is one rating block (its observed cells as COO), a rank k and a
list of held-out (row, col) cells to predict. The method is the same as the
grid path, with each request as one block: centre on the block mean, rank-k
truncated SVD, predict mu + P[r] . V[c].

Scheduling:
  * worker threads, each with its own library context on its own CUDA
    stream, so batches run concurrently on the device (the library's calls
    release the GIL and synchronise only their own stream);
  * requests wait in one FIFO queue. A free worker takes the longest prefix
    of the queue (at most max_batch requests) whose device footprint fits
    the memory budget next to what the other workers' contexts hold.
    Requests that arrive while batches run join the next batch a worker
    starts, which is what continuous batching means here;
  * a batch is laid out block-diagonally (bsvd_partition_diag) and
    factorised in one bsvd_factor_ks call with each request's own k, so all
    its blocks share every kernel launch;
  * a request larger than the whole budget fails at submit.
Latency = completion time - arrival time (host clock).
"""
from __future__ import annotations

import collections
import concurrent.futures as cf
import dataclasses
import threading
import time

import numpy as np

from . import Context


@dataclasses.dataclass
class Request:
    m: int
    n: int
    k: int
    r: np.ndarray              # observed cells: rows (int32)
    c: np.ndarray              # columns (int32)
    x: np.ndarray              # ratings (float32)
    qr: np.ndarray             # held-out rows to predict (int32)
    qc: np.ndarray             # held-out columns (int32)
    rid: int = 0
    arrival: float = 0.0

    @classmethod
    def from_dense(cls, dense, k, qr, qc):
        """A request from an m x n float32 matrix whose zeros mean
        "missing"."""
        r, c = np.nonzero(dense)
        return cls(dense.shape[0], dense.shape[1], k, r.astype(np.int32),
                   c.astype(np.int32), dense[r, c].astype(np.float32),
                   np.asarray(qr, np.int32), np.asarray(qc, np.int32))

    @property
    def nnz(self):
        return len(self.r)


@dataclasses.dataclass
class Result:
    rid: int
    yhat: np.ndarray
    latency: float             # seconds from arrival to completion
    batch_size: int


def _round_up(v, m):
    return (v + m - 1) // m * m


def footprint(m: int, n: int, nnz: int, nq: int = 0) -> int:
    """Upper bound on the device bytes one m x n request with nnz observed
    cells adds to a batch: the float32 block (32-padded), the two bf16
    planes (128-padded rows), the Gram, two 64-wide subspace panels, their
    split (hi, lo) copies for the tensor cores and their per-row-tile
    partials, the Rayleigh-Ritz matrix, both factors at the widest k, and
    the staged COO triples and queries. The batch's subspace width and
    factor width are its largest request's, so the widest ones are
    assumed."""
    s, L = min(m, n), max(m, n)
    sp, Lp, s128 = _round_up(s, 32), _round_up(L, 32), _round_up(s, 128)
    B, kp = 64, 56
    return (4 * sp * Lp + 4 * s128 * Lp + 4 * sp * sp + 8 * sp * B
            + 16 * sp * B + 8 * B * B * (sp // 64 + 1) + 4 * B * B
            + 4 * (sp + Lp) * kp + 12 * (nnz + nq) + (1 << 12))


class Server:
    """Continuous batching over worker threads with HBM-budget admission.

    A worker's context keeps its device buffers at the largest batch it has
    run (they only grow), so the budget is charged with what every context
    holds: worker w may start a batch needing F bytes only if the other
    workers' holdings plus max(holding_w, F) fit. When the oldest waiting
    request does not fit, idle workers drop and recreate their contexts,
    which frees what they hold. The queue is strict FIFO: a request that
    does not fit yet blocks the ones behind it, so none starves.
    """

    def __init__(self, workers: int = 4, max_batch: int = 64,
                 hbm_budget: float = 120e9, precision: int = 0,
                 context_factory=None, runner=None):
        """context_factory() -> a new per-worker context (default: a library
        Context on a new CUDA stream); runner(ctx, requests) -> list of
        prediction arrays (default: run_batch)."""
        self.max_batch = max_batch
        self.budget = int(hbm_budget)
        self.held = [0] * workers  # bytes each worker's context holds
        self.max_held = 0
        self.in_flight = 0
        self.max_in_flight = 0
        self.resets = 0
        self.batches = []          # (request ids, bytes) per batch
        self._q = collections.deque()
        self._cv = threading.Condition()
        self._stop = False
        self._next_id = 0
        self._run = runner or run_batch
        if context_factory is None:
            def context_factory():
                import torch
                return Context(stream=torch.cuda.Stream(),
                               precision=precision)
        self._factory = context_factory
        self._threads = []
        for w in range(workers):
            t = threading.Thread(target=self._worker,
                                 args=(w, context_factory()), daemon=True)
            t.start()
            self._threads.append(t)

    # ---- client side ----------------------------------------------------
    def submit(self, req: Request) -> cf.Future:
        fut = cf.Future()
        fp = footprint(req.m, req.n, req.nnz, len(req.qr))
        if fp > self.budget:
            fut.set_exception(ValueError(
                "request needs %d bytes, budget is %d" % (fp, self.budget)))
            return fut
        with self._cv:
            if self._stop:
                raise RuntimeError("server is closed")
            req.rid = self._next_id
            self._next_id += 1
            req.arrival = time.perf_counter()
            self._q.append((req, fut, fp))
            self._cv.notify_all()
        return fut

    def close(self):
        with self._cv:
            self._stop = True
            self._cv.notify_all()
        for t in self._threads:
            t.join()

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    # ---- workers --------------------------------------------------------
    def _fits(self, w, need):
        others = sum(self.held) - self.held[w]
        return others + max(self.held[w], need) <= self.budget

    def _take(self, w, ctx):
        """Block until worker w can start a batch; return (batch, ctx)."""
        with self._cv:
            while True:
                if self._stop and not self._q:
                    return None, ctx
                if self._q and self._fits(w, self._q[0][2]):
                    batch, need = [], 0
                    while (self._q and len(batch) < self.max_batch
                           and self._fits(w, need + self._q[0][2])):
                        item = self._q.popleft()
                        batch.append(item)
                        need += item[2]
                    self.held[w] = max(self.held[w], need)
                    self.max_held = max(self.max_held, sum(self.held))
                    self.in_flight += 1
                    self.max_in_flight = max(self.max_in_flight,
                                             self.in_flight)
                    self.batches.append(([b[0].rid for b in batch], need))
                    return batch, ctx
                if self._q and self.held[w] > 0:
                    # memory pressure: give back what this idle worker holds
                    if hasattr(ctx, "close"):
                        ctx.close()
                    ctx = self._factory()
                    self.held[w] = 0
                    self.resets += 1
                    self._cv.notify_all()
                    continue
                self._cv.wait()

    def _done(self):
        with self._cv:
            self.in_flight -= 1
            self._cv.notify_all()

    def _worker(self, w, ctx):
        while True:
            batch, ctx = self._take(w, ctx)
            if batch is None:
                if hasattr(ctx, "close"):
                    ctx.close()
                return
            try:
                results = self._run(ctx, [b[0] for b in batch])
                done = time.perf_counter()
                for (req, fut, _), y in zip(batch, results):
                    fut.set_result(Result(req.rid, y, done - req.arrival,
                                          len(batch)))
            except Exception as e:  # noqa: BLE001 - handed to the caller
                for _, fut, _ in batch:
                    if not fut.done():
                        fut.set_exception(e)
            finally:
                self._done()


def run_batch(ctx: Context, reqs) -> list:
    """Factorise a batch of requests as one block-diagonal partition and
    return each request's predictions."""
    nb = len(reqs)
    rb = np.zeros(nb + 1, np.int64)
    cb = np.zeros(nb + 1, np.int64)
    us, is_, xs, qu, qi = [], [], [], [], []
    for b, req in enumerate(reqs):
        rb[b + 1] = rb[b] + req.m
        cb[b + 1] = cb[b] + req.n
        us.append(np.asarray(req.r, np.int32) + np.int32(rb[b]))
        is_.append(np.asarray(req.c, np.int32) + np.int32(cb[b]))
        xs.append(np.asarray(req.x, np.float32))
        qu.append(np.asarray(req.qr, np.int32) + np.int32(rb[b]))
        qi.append(np.asarray(req.qc, np.int32) + np.int32(cb[b]))
    u = np.concatenate(us)
    i = np.concatenate(is_)
    x = np.concatenate(xs)
    ctx.partition_diag(rb, cb, u, i, x)
    ctx.factor([req.k for req in reqs], warn=False)
    yq = ctx.predict(np.concatenate(qu), np.concatenate(qi))
    out, off = [], 0
    for req in reqs:
        nq = len(req.qr)
        out.append(yq[off:off + nq].copy())
        off += nq
    return out


def latency_percentiles(results) -> dict:
    lat = np.array([r.latency for r in results])
    return {"p50_ms": float(np.percentile(lat, 50) * 1e3),
            "p99_ms": float(np.percentile(lat, 99) * 1e3)}
