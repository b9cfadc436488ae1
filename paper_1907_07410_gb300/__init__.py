"""Python binding of libbsvd, the block-SVD recommender library for GB300.

The functions named ``bsvd_*`` mirror the C ABI in ``include/bsvd.h`` one to
one and only marshal arguments: every step of the method runs in the CUDA
library. ``Context`` wraps them for convenience. Arrays may be numpy arrays
(host memory) or torch tensors (host or CUDA); their dtypes must already be
int32 for ids and float32 for ratings.

There is no CPU fallback: if libbsvd.so cannot be loaded, every call raises.
"""
from __future__ import annotations

import ctypes
import os
import warnings

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libbsvd.so")

OK, EINVAL, ENOMEM, ECUDA, ENOTCONV, ETIMEOUT, ESTATE = range(7)
FP32, TF32, BF16 = range(3)           # bsvd_precision
SGD_FP64, SGD_FP32 = range(2)         # bsvd_sgd_precision
STATUS_NAMES = {OK: "OK", EINVAL: "EINVAL", ENOMEM: "ENOMEM", ECUDA: "ECUDA",
                ENOTCONV: "ENOTCONV", ETIMEOUT: "ETIMEOUT", ESTATE: "ESTATE"}

# every symbol the header declares
EXPORTS = ("bsvd_config_default", "bsvd_create", "bsvd_destroy",
           "bsvd_last_error", "bsvd_partition", "bsvd_factor", "bsvd_predict",
           "bsvd_rmse", "bsvd_block_stats", "bsvd_get_block",
           "bsvd_reconstruct", "bsvd_factor_report", "bsvd_phase_times",
           "bsvd_kernel_launches", "bsvd_block_means_noalloc",
           "bsvd_gram_path", "bsvd_partition_diag", "bsvd_factor_ks",
           "bsvd_sgd_params_default", "bsvd_sgd_prepare", "bsvd_sgd_train",
           "bsvd_sgd_predict", "bsvd_sgd_get", "bsvd_quantile_grid",
           "bsvd_partition_quantile",
           "bsvd_set_owned", "bsvd_sqerr", "bsvd_loop_form",
           "bsvd_panel_launches")


class BsvdError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__("%s: %s" % (STATUS_NAMES.get(status, status), message))
        self.status = status


class Config(ctypes.Structure):
    _fields_ = [("precision", ctypes.c_int32), ("clamp", ctypes.c_int32),
                ("clamp_lo", ctypes.c_float), ("clamp_hi", ctypes.c_float),
                ("oversample", ctypes.c_int32),
                ("cheb_degree", ctypes.c_int32),
                ("max_iters", ctypes.c_int32), ("max_sweeps", ctypes.c_int32),
                ("profile", ctypes.c_int32), ("gram_path", ctypes.c_int32),
                ("tol", ctypes.c_double), ("seed", ctypes.c_uint64),
                ("stream", ctypes.c_void_p), ("panel_path", ctypes.c_int32),
                ("loop", ctypes.c_int32)]


class SgdParams(ctypes.Structure):
    """bsvd_sgd_params: rates named by the parameter they update."""
    _fields_ = [("a_user", ctypes.c_double), ("b_user", ctypes.c_double),
                ("a_item", ctypes.c_double), ("b_item", ctypes.c_double),
                ("a_ubias", ctypes.c_double), ("b_ubias", ctypes.c_double),
                ("a_ibias", ctypes.c_double), ("b_ibias", ctypes.c_double),
                ("delta", ctypes.c_double), ("k", ctypes.c_int32),
                ("max_steps", ctypes.c_int32), ("precision", ctypes.c_int32)]


_lib = None


def load(build_if_missing: bool = True) -> ctypes.CDLL:
    """Load libbsvd.so (compiling it first when it is missing or stale)."""
    global _lib
    if _lib is not None:
        return _lib
    if build_if_missing:
        from . import build as _build
        if _build.stale():
            _build.build()
    if not os.path.exists(LIB_PATH):
        raise RuntimeError("libbsvd.so is not built (run __graft_entry__.build())")
    lib = ctypes.CDLL(LIB_PATH)
    vp, i32, i64 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64
    sig = {
        "bsvd_config_default": (None, [ctypes.POINTER(Config)]),
        "bsvd_create": (i32, [ctypes.POINTER(Config), ctypes.POINTER(vp)]),
        "bsvd_destroy": (None, [vp]),
        "bsvd_last_error": (ctypes.c_char_p, [vp]),
        "bsvd_partition": (i32, [vp, i64, i64, i64, vp, vp, vp, i32, i32, vp,
                                 vp, vp, vp]),
        "bsvd_factor": (i32, [vp, i32]),
        "bsvd_partition_diag": (i32, [vp, i32, vp, vp, i64, vp, vp, vp]),
        "bsvd_factor_ks": (i32, [vp, vp]),
        "bsvd_predict": (i32, [vp, i64, vp, vp, vp]),
        "bsvd_rmse": (i32, [vp, i64, vp, vp, vp, ctypes.POINTER(ctypes.c_double)]),
        "bsvd_block_stats": (i32, [vp, ctypes.POINTER(i32), vp, vp]),
        "bsvd_get_block": (i32, [vp, i32, ctypes.POINTER(i32), ctypes.POINTER(i32),
                                 ctypes.POINTER(i32), ctypes.POINTER(ctypes.c_float),
                                 vp, vp, vp, vp]),
        "bsvd_reconstruct": (i32, [vp, i32, i32, vp]),
        "bsvd_factor_report": (i32, [vp, vp, vp, vp, vp, vp, vp]),
        "bsvd_phase_times": (i32, [vp, vp]),
        "bsvd_kernel_launches": (i64, [vp]),
        "bsvd_gram_path": (i32, [vp]),
        "bsvd_block_means_noalloc": (i32, [i64, i64, i64, vp, vp, vp, i32,
                                           i32, vp, vp, vp]),
        "bsvd_sgd_params_default": (None, [ctypes.POINTER(SgdParams)]),
        "bsvd_sgd_prepare": (i32, [vp, i64, vp, vp, vp]),
        "bsvd_sgd_train": (i32, [vp, ctypes.POINTER(SgdParams), vp, vp, vp,
                                 ctypes.POINTER(i32)]),
        "bsvd_sgd_predict": (i32, [vp, i64, vp, vp, vp]),
        "bsvd_sgd_get": (i32, [vp, vp, vp, vp, vp]),
        "bsvd_partition_quantile": (i32, [vp, i64, i64, i64, vp, vp, vp, i32,
                                          i32, vp, vp]),
        "bsvd_quantile_grid": (i32, [vp, i64, i64, i64, vp, vp, i32, i32, vp,
                                     vp, vp, vp]),
        "bsvd_set_owned": (i32, [vp, i32, vp]),
        "bsvd_loop_form": (i32, [vp]),
        "bsvd_panel_launches": (i64, [vp]),
        "bsvd_sqerr": (i32, [vp, i64, vp, vp, vp,
                             ctypes.POINTER(ctypes.c_double),
                             ctypes.POINTER(ctypes.c_int64)]),
    }
    for name, (res, args) in sig.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    _lib = lib
    return lib


# ---- argument marshalling ------------------------------------------------

def _ptr(a, dtype, name):
    """Address of a contiguous array (numpy or torch, host or device)."""
    if a is None:
        return None
    if isinstance(a, np.ndarray):
        if a.dtype != dtype:
            raise TypeError("%s must be %s, got %s" % (name, dtype, a.dtype))
        if not a.flags.c_contiguous:
            raise ValueError("%s must be contiguous" % name)
        return a.ctypes.data
    try:
        import torch
    except ImportError:  # pragma: no cover
        torch = None
    if torch is not None and isinstance(a, torch.Tensor):
        want = {np.dtype(np.int32): torch.int32, np.dtype(np.float32): torch.float32,
                np.dtype(np.int64): torch.int64, np.dtype(np.float64): torch.float64}[np.dtype(dtype)]
        if a.dtype != want:
            raise TypeError("%s must be %s, got %s" % (name, want, a.dtype))
        if not a.is_contiguous():
            raise ValueError("%s must be contiguous" % name)
        return a.data_ptr()
    raise TypeError("%s must be a numpy array or torch tensor" % name)


def _len(a):
    return int(a.shape[0]) if a is not None else 0


def _check(ctx, status, allow=()):
    if status != OK and status not in allow:
        msg = load().bsvd_last_error(ctx)
        raise BsvdError(status, msg.decode() if msg else "")
    return status


# ---- the C ABI, one function per entry point ------------------------------

def bsvd_config_default() -> Config:
    cfg = Config()
    load().bsvd_config_default(ctypes.byref(cfg))
    return cfg


def bsvd_create(cfg: Config | None = None) -> int:
    h = ctypes.c_void_p()
    st = load().bsvd_create(ctypes.byref(cfg) if cfg is not None else None,
                            ctypes.byref(h))
    if st != OK:
        raise BsvdError(st, "bsvd_create failed")
    return h.value


def bsvd_destroy(ctx) -> None:
    load().bsvd_destroy(ctx)


def bsvd_last_error(ctx) -> str:
    return load().bsvd_last_error(ctx).decode()


def bsvd_partition(ctx, m, n, u, i, x, p, q, row_bounds=None, col_bounds=None,
                   row_perm=None, col_perm=None) -> int:
    nnz = _len(u)
    if _len(i) != nnz or _len(x) != nnz:
        raise ValueError("u, i, x must have the same length")
    rb = None if row_bounds is None else np.ascontiguousarray(row_bounds, np.int64)
    cb = None if col_bounds is None else np.ascontiguousarray(col_bounds, np.int64)
    if rb is not None and rb.size != p + 1:
        raise ValueError("row_bounds must have p + 1 entries")
    if cb is not None and cb.size != q + 1:
        raise ValueError("col_bounds must have q + 1 entries")
    if row_perm is not None and _len(row_perm) != m:
        raise ValueError("row_perm must have m entries")
    if col_perm is not None and _len(col_perm) != n:
        raise ValueError("col_perm must have n entries")
    st = load().bsvd_partition(
        ctx, m, n, nnz, _ptr(u, np.int32, "u"), _ptr(i, np.int32, "i"),
        _ptr(x, np.float32, "x"), p, q, _ptr(rb, np.int64, "row_bounds"),
        _ptr(cb, np.int64, "col_bounds"), _ptr(row_perm, np.int32, "row_perm"),
        _ptr(col_perm, np.int32, "col_perm"))
    return _check(ctx, st)


def bsvd_quantile_grid(ctx, m, n, u, i, p, q, row_perm, col_perm):
    """Activity-quantile grid; fills row_perm (m) and col_perm (n), host or
    device int32 arrays, and returns (row_bounds, col_bounds) as numpy."""
    nnz = _len(u)
    if _len(i) != nnz:
        raise ValueError("u, i must have the same length")
    if _len(row_perm) != m or _len(col_perm) != n:
        raise ValueError("row_perm needs m entries and col_perm n entries")
    rb = np.zeros(p + 1, np.int64)
    cb = np.zeros(q + 1, np.int64)
    st = load().bsvd_quantile_grid(
        ctx, m, n, nnz, _ptr(u, np.int32, "u"), _ptr(i, np.int32, "i"), p, q,
        _ptr(row_perm, np.int32, "row_perm"),
        _ptr(col_perm, np.int32, "col_perm"), rb.ctypes.data, cb.ctypes.data)
    _check(ctx, st)
    return rb, cb


def bsvd_partition_quantile(ctx, m, n, u, i, x, p, q):
    """The activity-quantile grid and the partition on it in one call;
    returns (row_bounds, col_bounds) as numpy."""
    nnz = _len(u)
    if _len(i) != nnz or _len(x) != nnz:
        raise ValueError("u, i, x must have the same length")
    rb = np.zeros(p + 1, np.int64)
    cb = np.zeros(q + 1, np.int64)
    st = load().bsvd_partition_quantile(
        ctx, m, n, nnz, _ptr(u, np.int32, "u"), _ptr(i, np.int32, "i"),
        _ptr(x, np.float32, "x"), p, q, rb.ctypes.data, cb.ctypes.data)
    _check(ctx, st)
    return rb, cb


def bsvd_partition_diag(ctx, row_bounds, col_bounds, u, i, x) -> int:
    rb = np.ascontiguousarray(row_bounds, np.int64)
    cb = np.ascontiguousarray(col_bounds, np.int64)
    if rb.size != cb.size or rb.size < 2:
        raise ValueError("row_bounds and col_bounds need nb + 1 entries")
    nnz = _len(u)
    if _len(i) != nnz or _len(x) != nnz:
        raise ValueError("u, i, x must have the same length")
    st = load().bsvd_partition_diag(
        ctx, rb.size - 1, rb.ctypes.data, cb.ctypes.data, nnz,
        _ptr(u, np.int32, "u"), _ptr(i, np.int32, "i"),
        _ptr(x, np.float32, "x"))
    return _check(ctx, st)


def bsvd_factor_ks(ctx, ks) -> int:
    ks = np.ascontiguousarray(ks, np.int32)
    st = load().bsvd_factor_ks(ctx, ks.ctypes.data)
    return _check(ctx, st, allow=(ENOTCONV,))


def bsvd_factor(ctx, k) -> int:
    st = load().bsvd_factor(ctx, k)
    return _check(ctx, st, allow=(ENOTCONV,))


def bsvd_predict(ctx, u, i, yhat) -> int:
    nq = _len(u)
    if _len(i) != nq or _len(yhat) != nq:
        raise ValueError("u, i, yhat must have the same length")
    st = load().bsvd_predict(ctx, nq, _ptr(u, np.int32, "u"),
                             _ptr(i, np.int32, "i"),
                             _ptr(yhat, np.float32, "yhat"))
    return _check(ctx, st)


def bsvd_rmse(ctx, u, i, y) -> float:
    nq = _len(u)
    if _len(i) != nq or _len(y) != nq:
        raise ValueError("u, i, y must have the same length")
    out = ctypes.c_double()
    st = load().bsvd_rmse(ctx, nq, _ptr(u, np.int32, "u"),
                          _ptr(i, np.int32, "i"), _ptr(y, np.float32, "y"),
                          ctypes.byref(out))
    _check(ctx, st)
    return out.value


def bsvd_set_owned(ctx, owned=None) -> int:
    """Hold only the blocks flagged in `owned` (one entry per block of the
    next partition); None holds all of them again."""
    if owned is None:
        return _check(ctx, load().bsvd_set_owned(ctx, 0, None))
    mask = np.ascontiguousarray(np.asarray(owned) != 0, np.uint8)
    return _check(ctx, load().bsvd_set_owned(ctx, mask.size, mask.ctypes.data))


def bsvd_sqerr(ctx, u, i, y):
    """(sum of squared errors, count) over the queries of held blocks."""
    nq = _len(u)
    if _len(i) != nq or _len(y) != nq:
        raise ValueError("u, i, y must have the same length")
    out = ctypes.c_double()
    cnt = ctypes.c_int64()
    st = load().bsvd_sqerr(ctx, nq, _ptr(u, np.int32, "u"),
                           _ptr(i, np.int32, "i"), _ptr(y, np.float32, "y"),
                           ctypes.byref(out), ctypes.byref(cnt))
    _check(ctx, st)
    return out.value, cnt.value


def bsvd_block_stats(ctx, nblocks: int):
    counts = np.zeros(nblocks, np.int64)
    mu = np.zeros(nblocks, np.float32)
    nb = ctypes.c_int32()
    st = load().bsvd_block_stats(ctx, ctypes.byref(nb), counts.ctypes.data,
                                 mu.ctypes.data)
    _check(ctx, st)
    return counts[:nb.value], mu[:nb.value]


def bsvd_get_block(ctx, b, want_factors=True, want_dense=False):
    mb, nb, keff = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int32()
    mu = ctypes.c_float()
    lib = load()
    st = lib.bsvd_get_block(ctx, b, ctypes.byref(mb), ctypes.byref(nb),
                            ctypes.byref(keff), ctypes.byref(mu), None, None,
                            None, None)
    _check(ctx, st)
    out = dict(mb=mb.value, nb=nb.value, keff=keff.value, mu=mu.value)
    sigma = P = V = dense = None
    if want_factors:
        sigma = np.zeros(max(keff.value, 1), np.float64)
        P = np.zeros((mb.value, keff.value), np.float32)
        V = np.zeros((nb.value, keff.value), np.float32)
    if want_dense:
        dense = np.zeros((mb.value, nb.value), np.float32)
    st = lib.bsvd_get_block(ctx, b, None, None, None, None,
                            sigma.ctypes.data if sigma is not None else None,
                            P.ctypes.data if P is not None else None,
                            V.ctypes.data if V is not None else None,
                            dense.ctypes.data if dense is not None else None)
    _check(ctx, st)
    if want_factors:
        out.update(sigma=sigma[:keff.value], P=P, V=V)
    if want_dense:
        out["dense"] = dense
    return out


def bsvd_reconstruct(ctx, b, out, add_mean=True) -> int:
    st = load().bsvd_reconstruct(ctx, b, 1 if add_mean else 0,
                                 _ptr(out, np.float32, "out"))
    return _check(ctx, st)


def bsvd_factor_report(ctx, nblocks: int, full: bool = False):
    iters = np.zeros(nblocks, np.int32)
    conv = np.zeros(nblocks, np.int32)
    sweeps = np.zeros(nblocks, np.int32)
    cycles = np.zeros((nblocks, 3), np.int64)
    resid = np.zeros(nblocks, np.float32)
    products = np.zeros(nblocks, np.int32)
    st = load().bsvd_factor_report(ctx, iters.ctypes.data, conv.ctypes.data,
                                   sweeps.ctypes.data, cycles.ctypes.data,
                                   resid.ctypes.data, products.ctypes.data)
    _check(ctx, st)
    if full:
        return dict(iters=iters, converged=conv, sweeps=sweeps, cycles=cycles,
                    resid=resid, products=products)
    return iters, conv


def bsvd_phase_times(ctx) -> np.ndarray:
    ms = np.zeros(8, np.float64)
    _check(ctx, load().bsvd_phase_times(ctx, ms.ctypes.data))
    return ms


def bsvd_kernel_launches(ctx) -> int:
    return int(load().bsvd_kernel_launches(ctx))


def bsvd_gram_path(ctx) -> int:
    return int(load().bsvd_gram_path(ctx))


def bsvd_loop_form(ctx) -> int:
    return int(load().bsvd_loop_form(ctx))


def bsvd_panel_launches(ctx) -> int:
    return int(load().bsvd_panel_launches(ctx))


PHASES = ("partition", "gram", "eigen", "project", "predict", "eigen_filter",
          "eigen_rr", "eigen_other")


def bsvd_sgd_params_default() -> SgdParams:
    prm = SgdParams()
    load().bsvd_sgd_params_default(ctypes.byref(prm))
    return prm


def bsvd_sgd_prepare(ctx, u, i, x) -> int:
    nnz = _len(u)
    if _len(i) != nnz or _len(x) != nnz:
        raise ValueError("u, i, x must have the same length")
    st = load().bsvd_sgd_prepare(ctx, nnz, _ptr(u, np.int32, "u"),
                                 _ptr(i, np.int32, "i"),
                                 _ptr(x, np.float32, "x"))
    return _check(ctx, st)


def bsvd_sgd_train(ctx, prm: SgdParams, P0, Q0):
    """Returns (training RMSE history, epochs run)."""
    hist = np.zeros(prm.max_steps + 1, np.float64)
    ran = ctypes.c_int32(0)
    st = load().bsvd_sgd_train(ctx, ctypes.byref(prm),
                               _ptr(P0, np.float64, "P0"),
                               _ptr(Q0, np.float64, "Q0"), hist.ctypes.data,
                               ctypes.byref(ran))
    _check(ctx, st)
    return hist[:ran.value + 1].copy(), ran.value


def bsvd_sgd_predict(ctx, u, i, yhat) -> int:
    nq = _len(u)
    if _len(i) != nq or _len(yhat) != nq:
        raise ValueError("u, i, yhat must have the same length")
    st = load().bsvd_sgd_predict(ctx, nq, _ptr(u, np.int32, "u"),
                                 _ptr(i, np.int32, "i"),
                                 _ptr(yhat, np.float64, "yhat"))
    return _check(ctx, st)


def bsvd_sgd_get(ctx, m, n, k):
    P = np.zeros((m, k), np.float64)
    Q = np.zeros((n, k), np.float64)
    bu = np.zeros(m, np.float64)
    bi = np.zeros(n, np.float64)
    st = load().bsvd_sgd_get(ctx, P.ctypes.data, Q.ctypes.data,
                             bu.ctypes.data, bi.ctypes.data)
    _check(ctx, st)
    return P, Q, bu, bi


def bsvd_block_means_noalloc(m, n, u, i, x, p, q, counts, mu,
                             stream=None) -> int:
    """Block counts and means with no allocation (device arrays only).

    For callers that cannot allocate device memory during the call; the
    scratch lives in a fixed device array of the library (p * q <= 4096).
    Returns the status code (0 on success) instead of raising, since there
    is no context to hold an error message.
    """
    nnz = _len(u)
    if _len(i) != nnz or _len(x) != nnz:
        raise ValueError("u, i, x must have the same length")
    if _len(counts) < p * q or _len(mu) < p * q:
        raise ValueError("counts and mu need p * q entries")
    try:
        import torch
        cur = torch.cuda.current_device() if torch.cuda.is_available() else None
        for name, a in (("u", u), ("i", i), ("x", x), ("counts", counts),
                        ("mu", mu)):
            if (isinstance(a, torch.Tensor) and a.is_cuda
                    and a.device.index != cur):
                raise ValueError("%s is on cuda:%d, not the current device "
                                 "cuda:%s" % (name, a.device.index, cur))
    except ImportError:  # pragma: no cover
        pass
    if stream is not None and not isinstance(stream, int):
        stream = stream.cuda_stream
    return int(load().bsvd_block_means_noalloc(
        m, n, nnz, _ptr(u, np.int32, "u"), _ptr(i, np.int32, "i"),
        _ptr(x, np.float32, "x"), p, q, _ptr(counts, np.int64, "counts"),
        _ptr(mu, np.float32, "mu"), stream))


# ---- convenience wrapper ----------------------------------------------------

class Context:
    """One libbsvd context on the current CUDA device.

    ``stream``: a torch.cuda.Stream, a raw cudaStream_t integer, or None
    (the current torch stream when torch is imported, else the default
    stream).
    """

    def __init__(self, stream=None, **cfg_fields):
        cfg = bsvd_config_default()
        for k, v in cfg_fields.items():
            if not hasattr(cfg, k):
                raise TypeError("unknown config field %r" % k)
            setattr(cfg, k, v)
        if stream is None:
            try:
                import torch
                if torch.cuda.is_available():
                    stream = torch.cuda.current_stream()
            except ImportError:  # pragma: no cover
                pass
        if stream is not None and not isinstance(stream, int):
            stream = stream.cuda_stream
        cfg.stream = stream
        self.cfg = cfg
        self.handle = bsvd_create(cfg)
        self.nblocks = 0
        self.last_status = OK

    def close(self):
        if getattr(self, "handle", None):
            bsvd_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:  # pragma: no cover
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def partition(self, m, n, u, i, x, p, q, row_bounds=None, col_bounds=None,
                  row_perm=None, col_perm=None):
        bsvd_partition(self.handle, m, n, u, i, x, p, q, row_bounds,
                       col_bounds, row_perm, col_perm)
        self.nblocks = p * q

    def quantile_grid(self, m, n, u, i, p, q):
        """Keyword arguments for partition(): the activity-quantile grid of
        the ratings (u, i). The permutations live where u does (CUDA
        tensors for CUDA input, else numpy arrays)."""
        on_gpu = False
        try:
            import torch
            on_gpu = isinstance(u, torch.Tensor) and u.is_cuda
        except ImportError:  # pragma: no cover
            pass
        if on_gpu:
            rp = torch.empty(m, dtype=torch.int32, device=u.device)
            cp = torch.empty(n, dtype=torch.int32, device=u.device)
        else:
            rp = np.empty(m, np.int32)
            cp = np.empty(n, np.int32)
        rb, cb = bsvd_quantile_grid(self.handle, m, n, u, i, p, q, rp, cp)
        return dict(row_bounds=rb, col_bounds=cb, row_perm=rp, col_perm=cp)

    def partition_quantile(self, m, n, u, i, x, p, q):
        """quantile_grid() and partition() in one call (host ratings go up
        once); returns (row_bounds, col_bounds)."""
        rb, cb = bsvd_partition_quantile(self.handle, m, n, u, i, x, p, q)
        self.nblocks = p * q
        return rb, cb

    def partition_diag(self, row_bounds, col_bounds, u, i, x):
        bsvd_partition_diag(self.handle, row_bounds, col_bounds, u, i, x)
        self.nblocks = len(row_bounds) - 1

    def factor(self, k, warn=True):
        """k: one rank for every block, or a sequence of one per block."""
        if np.ndim(k) == 0:
            st = bsvd_factor(self.handle, int(k))
        else:
            st = bsvd_factor_ks(self.handle, k)
        self.last_status = st
        if st == ENOTCONV and warn:
            warnings.warn("bsvd_factor: " + bsvd_last_error(self.handle))
        return st

    def predict(self, u, i, out=None):
        if out is None:
            out = np.zeros(_len(u), np.float32)
        bsvd_predict(self.handle, u, i, out)
        return out

    def rmse(self, u, i, y):
        return bsvd_rmse(self.handle, u, i, y)

    def set_owned(self, owned=None):
        """Hold only the flagged blocks from the next partition on (multi-GPU
        sharding); None holds every block."""
        bsvd_set_owned(self.handle, owned)

    def sqerr(self, u, i, y):
        """(sum of squared errors, count) over the held blocks' queries."""
        return bsvd_sqerr(self.handle, u, i, y)

    def block_stats(self):
        return bsvd_block_stats(self.handle, self.nblocks)

    def get_block(self, b, want_factors=True, want_dense=False):
        return bsvd_get_block(self.handle, b, want_factors, want_dense)

    def reconstruct(self, b, add_mean=True, out=None):
        """Block b's rank-k reconstruction (mb x nb). `out`: an optional
        float32 device tensor of mb * nb entries to write into (returned);
        else a new host array."""
        info = bsvd_get_block(self.handle, b, want_factors=False)
        cells = info["mb"] * info["nb"]
        if out is None:
            out = np.zeros((info["mb"], info["nb"]), np.float32)
        else:
            have = int(out.numel()) if hasattr(out, "numel") else int(np.size(out))
            if have < cells:
                raise ValueError("out holds %d entries, the block has %d"
                                 % (have, cells))
        bsvd_reconstruct(self.handle, b, out, add_mean)
        return out

    def factor_report(self, full=False):
        return bsvd_factor_report(self.handle, self.nblocks, full)

    def phase_times(self) -> dict:
        return dict(zip(PHASES, bsvd_phase_times(self.handle).tolist()))

    def kernel_launches(self) -> int:
        return bsvd_kernel_launches(self.handle)

    def gram_path(self) -> int:
        return bsvd_gram_path(self.handle)

    def panel_launches(self) -> int:
        """Tensor-core panel-product launches in the last factor."""
        return bsvd_panel_launches(self.handle)

    def loop_form(self) -> int:
        """1: the last factor ran its eigen loop from the host; 2: as one
        CUDA graph decided on the device."""
        return bsvd_loop_form(self.handle)

    # ---- the paper's blocked SGD (Algorithms 1-2) ------------------------
    def sgd_prepare(self, u, i, x):
        """Epoch order of the training ratings on the last partition's grid
        (call partition first)."""
        bsvd_sgd_prepare(self.handle, u, i, x)
        self._sgd_shape = None

    def sgd_train(self, P0, Q0, **params):
        """Algorithm 1 from P0 (m x k), Q0 (n x k) float64; params override
        the Section 5 defaults (a_user, ..., delta, max_steps, precision:
        SGD_FP64 or SGD_FP32). Returns (training RMSE history, epochs
        run)."""
        prm = bsvd_sgd_params_default()
        prm.k = int(np.shape(P0)[1])
        for key, v in params.items():
            if not hasattr(prm, key):
                raise TypeError("unknown SGD parameter %r" % key)
            setattr(prm, key, v)
        self._sgd_shape = (int(np.shape(P0)[0]), int(np.shape(Q0)[0]), prm.k)
        return bsvd_sgd_train(self.handle, prm, P0, Q0)

    def sgd_predict(self, u, i, out=None):
        if out is None:
            out = np.zeros(_len(u), np.float64)
        bsvd_sgd_predict(self.handle, u, i, out)
        return out

    def sgd_get(self):
        """(P, Q, bu, bi) of the trained model, as host arrays."""
        m, n, k = self._sgd_shape
        return bsvd_sgd_get(self.handle, m, n, k)
