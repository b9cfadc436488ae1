"""Plain FP64 CPU oracle for the paper's own blocked SGD (Algorithms 1-2).

TEST INFRASTRUCTURE ONLY. Only ``tests/``, ``__graft_entry__`` and the
CPU-baseline leg of ``bench.py`` may import this module. It shares no code
with the CUDA library.

What it computes, with the passage each step follows:

1. Blocks (Algorithm 1, lines on the I x J block matrix): the ratings are
   cut into the same p x q grid as the SVD path (``oracle.make_grid``).
2. Schedule (Section 3, "Parallelism", Figure 2): blocks are visited in
   steps; a step holds blocks that share no block row and no block column,
   so their updates touch disjoint user and item parameters. Step s holds
   the blocks ((j + s) mod p, j) for j < q when p >= q, else
   (i, (i + s) mod q) for i < p; the first step is the main diagonal and
   each later step moves one block down every column, wrapping around.
   Within a step the blocks are taken in increasing column (row) order.
   Because they are independent, any order within a step gives the same
   result; that is what lets a GPU run a step's blocks at once.
3. Block pass (Algorithm 2): each block's ratings row by row, then column
   by column; the update of one rating is ``sgd.c``.
4. Epochs (Algorithm 1): one pass over every block per step of STEPS;
   after each epoch the training RMSE is measured and the loop ends when
   it improved by less than delta (the first comparison is against the
   RMSE of the starting point).
5. Predict (Eq. 3): y_hat = p_u . q_i + bu_u + bi_i, the dot product summed
   over f = 0 .. k-1 in order, then the biases added left to right.

Precision: float64. ``train(..., dtype=np.float32)`` runs the same steps
with float32 parameters and float32 arithmetic in each update, the
reference for the library's float32 form; its pins compare it with the
float64 run.

Readings: see ``sgd.c`` for the update; the starting factors are inputs
(the paper only says "random values"); biases start at zero; the RMSE of
the stopping rule is the training RMSE, since Algorithm 1 sees only X.
"""
from __future__ import annotations

import ctypes
import dataclasses
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "sgd.c")
_LIB = os.path.join(_HERE, "liboracle_sgd.so")
_lib = None
_lock = threading.Lock()   # builds and loads from worker threads


def build(force: bool = False) -> str:
    """Compile ``sgd.c``: plain gcc, no architecture flags, and no
    floating-point contraction, so each operation rounds once."""
    with _lock:
        if force or not os.path.exists(_LIB) or (
                os.path.getmtime(_LIB) < os.path.getmtime(_SRC)):
            tmp = _LIB + ".tmp%d.%d" % (os.getpid(), threading.get_ident())
            subprocess.check_call(["gcc", "-O2", "-ffp-contract=off", "-fPIC",
                                   "-shared", "-std=c99", "-o", tmp, _SRC])
            os.replace(tmp, _LIB)
    return _LIB


class _Rates(ctypes.Structure):
    _fields_ = [(n, ctypes.c_double) for n in (
        "a_user", "b_user", "a_item", "b_item", "a_ubias", "b_ubias",
        "a_ibias", "b_ibias")]


def _load():
    global _lib
    if _lib is not None:
        return _lib
    path = build()
    with _lock:
        if _lib is not None:
            return _lib
        lib = ctypes.CDLL(path)
        for f in (lib.oracle_sgd_pass, lib.oracle_sgd_pass_f32):
            f.restype = None
            f.argtypes = [ctypes.c_int64, ctypes.c_void_p, ctypes.c_void_p,
                          ctypes.c_void_p, ctypes.c_int32, ctypes.c_void_p,
                          ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                          ctypes.POINTER(_Rates)]
        _lib = lib
    return _lib


@dataclasses.dataclass
class Rates:
    """Learning rates (a_*) and regularisation factors (b_*) per parameter
    group. Defaults: the values of the experiments section (Section 5,
    "Hyper-parameters") for the SVD model."""
    a_user: float = 0.019
    b_user: float = 0.019
    a_item: float = 0.004
    b_item: float = 0.019
    a_ubias: float = 0.004
    b_ubias: float = 0.019
    a_ibias: float = 0.013
    b_ibias: float = 0.007

    def c(self) -> _Rates:
        return _Rates(self.a_user, self.b_user, self.a_item, self.b_item,
                      self.a_ubias, self.b_ubias, self.a_ibias, self.b_ibias)


DELTA = 1e-4        # Section 5: minimum RMSE improvement between steps
K = 13              # Section 5: number of latent factors


def schedule(p: int, q: int) -> list[list[int]]:
    """Block ids (bi * q + bj) of each step of the diagonal schedule."""
    steps = []
    if p >= q:
        for s in range(p):
            steps.append([((j + s) % p) * q + j for j in range(q)])
    else:
        for s in range(q):
            steps.append([i * q + (i + s) % q for i in range(p)])
    return steps


def processing_order(grid, u, i) -> np.ndarray:
    """Permutation of the ratings into the order of one epoch: schedule
    step, block within the step, then the block's local row, then its local
    column (Algorithm 2's loops). Ties (repeated cells) keep input order."""
    b, r, c = grid.locate(np.asarray(u), np.asarray(i))
    rank = np.empty(grid.p * grid.q, np.int64)
    pos = 0
    for step in schedule(grid.p, grid.q):
        for blk in step:
            rank[blk] = pos
            pos += 1
    return np.lexsort((np.arange(len(b)), c, r, rank[b]))


def sgd_pass(u, i, x, P, Q, bu, bi, rates: Rates) -> None:
    """One pass over ratings in the given order, in place (``sgd.c``). The
    parameters' dtype picks the arithmetic: all float64, or all float32
    (the same pass with every operation rounded to float32)."""
    u = np.ascontiguousarray(u, np.int32)
    i = np.ascontiguousarray(i, np.int32)
    x = np.ascontiguousarray(x, np.float32)
    dt = P.dtype
    assert dt in (np.float64, np.float32)
    for a in (P, Q, bu, bi):
        assert a.dtype == dt and a.flags.c_contiguous
    r = rates.c()
    lib = _load()
    f = lib.oracle_sgd_pass if dt == np.float64 else lib.oracle_sgd_pass_f32
    f(len(u), u.ctypes.data, i.ctypes.data, x.ctypes.data, P.shape[1],
      P.ctypes.data, Q.ctypes.data, bu.ctypes.data, bi.ctypes.data,
      ctypes.byref(r))


def predict(P, Q, bu, bi, u, i) -> np.ndarray:
    """Eq. 3, summed in the stated order (float64)."""
    u = np.asarray(u)
    i = np.asarray(i)
    dot = np.zeros(len(u))
    for f in range(P.shape[1]):
        dot = dot + P[u, f] * Q[i, f]
    return (dot + bu[u]) + bi[i]


def rmse(P, Q, bu, bi, u, i, x) -> float:
    d = np.asarray(x, np.float64) - predict(P, Q, bu, bi, u, i)
    return float(np.sqrt(np.mean(d * d)))


@dataclasses.dataclass
class Trained:
    P: np.ndarray
    Q: np.ndarray
    bu: np.ndarray
    bi: np.ndarray
    rmse: list          # training RMSE before the first epoch and after each
    steps_run: int


def train(grid, u, i, x, P0, Q0, steps: int, rates: Rates | None = None,
          delta: float = DELTA, dtype=np.float64) -> Trained:
    """Algorithm 1 over the grid's blocks, from factors P0 (m x k) and
    Q0 (n x k) and zero biases, for at most `steps` epochs. With dtype
    float32 the parameters are P0, Q0 rounded to float32 and every update
    is float32 arithmetic; the RMSE (and so the stopping rule) is float64
    over the parameters' values either way. The returned arrays are
    float64 (exact copies of float32 ones)."""
    rates = rates or Rates()
    order = processing_order(grid, u, i)
    uo, io, xo = (np.asarray(a)[order] for a in (u, i, x))
    P = np.array(P0, dtype, order="C")
    Q = np.array(Q0, dtype, order="C")
    bu = np.zeros(P.shape[0], dtype)
    bi = np.zeros(Q.shape[0], dtype)

    def wide():
        return tuple(np.asarray(a, np.float64) for a in (P, Q, bu, bi))

    hist = [rmse(*wide(), u, i, x)]
    ran = 0
    for _ in range(steps):
        sgd_pass(uo, io, xo, P, Q, bu, bi, rates)
        ran += 1
        hist.append(rmse(*wide(), u, i, x))
        if hist[-2] - hist[-1] < delta:
            break
    return Trained(*wide(), hist, ran)
