"""Python binding of the GB300 exact k-NN engine over an iSAX index (MESSI,
arXiv 2110.07519).

Argument marshalling only: every step of index construction and query
answering runs in the CUDA kernels of ``libmessi.so`` (C ABI in
``include/messi.h``).  PyTorch supplies device memory and streams; numpy
arrays (host memory) are accepted too and staged by the library.  Importing
this package fails loudly when the compiled library is missing -- there is no
CPU fallback.

Names mirror the C ABI: ``messi_build``, ``messi_query``, ... .
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libmessi.so")

MESSI_ED, MESSI_DTW = 0, 1
MESSI_BATCH_LB_REFINE, MESSI_BATCH_TC_SCREEN = 0, 1
STATUS_NAMES = {0: "OK", 1: "EINVAL", 2: "ENOMEM", 3: "ECUDA", 4: "ETIMEOUT", 5: "EBUSY", 6: "ETIES"}

if not os.path.exists(LIB_PATH):
    raise ImportError(
        f"{LIB_PATH} is missing: build it with `python -c 'import __graft_entry__ as g; g.build()'` "
        "(the CUDA library is required; there is no CPU fallback)")

_lib = ctypes.CDLL(LIB_PATH)
_P, _U32, _U64, _I = ctypes.c_void_p, ctypes.c_uint32, ctypes.c_uint64, ctypes.c_int


class MessiConfig(ctypes.Structure):
    _fields_ = [("leaf_capacity", ctypes.c_uint32), ("reserved", ctypes.c_uint32 * 7)]


class MessiStats(ctypes.Structure):
    _fields_ = [(n, ctypes.c_uint64) for n in (
        "queries", "lb_evaluated", "lb_survivors", "lbk_survivors", "seeded", "refined", "abandoned",
        "bsf_updates", "tie_rechecks", "kernel_launches", "scan_launches")] + [
        ("scan_ms", ctypes.c_double), ("query_ms_p50", ctypes.c_double), ("query_ms_p99", ctypes.c_double),
        ("leaves_live", ctypes.c_uint64), ("screened_queries", ctypes.c_uint64), ("row_bytes", ctypes.c_uint64),
        ("dtw_cells", ctypes.c_uint64), ("refine_ms", ctypes.c_double), ("refine_launches", ctypes.c_uint64)]

    def as_dict(self):
        return {n: getattr(self, n) for n, _ in self._fields_ if n != "reserved"}


class MessiIndexInfo(ctypes.Structure):
    _fields_ = [("n_series", ctypes.c_uint64), ("len", ctypes.c_uint32), ("segments", ctypes.c_uint32),
                ("cardinality", ctypes.c_uint32), ("leaf_capacity", ctypes.c_uint32),
                ("n_leaves", ctypes.c_uint64), ("max_leaf_size", ctypes.c_uint64),
                ("device_bytes", ctypes.c_uint64), ("build_ms", ctypes.c_double)]

    def as_dict(self):
        return {n: getattr(self, n) for n, _ in self._fields_}


class MessiTuning(ctypes.Structure):
    _fields_ = [("batch", ctypes.c_uint32), ("chunk_tiles", ctypes.c_uint32), ("ctas_per_sm", ctypes.c_uint32),
                ("mode", ctypes.c_uint32), ("ms_per_query", ctypes.c_double), ("reserved", ctypes.c_uint32 * 4)]

    def as_dict(self):
        return {n: getattr(self, n) for n, _ in self._fields_ if n != "reserved"}


class MessiServerConfig(ctypes.Structure):
    _fields_ = [("max_batch", ctypes.c_uint32), ("max_k", ctypes.c_uint32), ("streams", ctypes.c_uint32),
                ("max_queued", ctypes.c_uint32), ("mem_budget", ctypes.c_uint64),
                ("reserved", ctypes.c_uint64 * 4)]


class MessiServerStats(ctypes.Structure):
    _fields_ = [(n, ctypes.c_uint64) for n in ("submitted", "completed", "rejected", "batches", "inflight_peak")] + [
        ("p50_ms", ctypes.c_double), ("p99_ms", ctypes.c_double), ("mean_ms", ctypes.c_double),
        ("budget_waits", ctypes.c_uint64), ("reserved", ctypes.c_uint64 * 3)]

    def as_dict(self):
        return {n: getattr(self, n) for n, _ in self._fields_ if n != "reserved"}


_SIGS = {
    "messi_build": [_P, _U64, _U32, _U32, _U32, _P, _P, ctypes.POINTER(_P)],
    "messi_free": [_P],
    "messi_index_get_info": [_P, ctypes.POINTER(MessiIndexInfo)],
    "messi_windows": [_P, _U64, _U32, _U32, _I, _P, ctypes.POINTER(_U64), _P],
    "messi_query": [_P, _P, _U32, _U32, _I, _U32, _P, _P, _P],
    "messi_query_batched": [_P, _P, _U32, _U32, _I, _U32, _U32, _P, _P, _P],
    "messi_lower_bounds": [_P, _P, _I, _U32, _P, _P],
    "messi_lower_bounds_noalloc": [_P, _P, _I, _U32, _P, _P],
    "messi_query_stats": [_P, ctypes.POINTER(MessiStats)],
    "messi_set_profiling": [_P, _I],
    "messi_set_batch_mode": [_P, _I],
    "messi_autotune": [_P, _P, _U32, _U32, _P, ctypes.POINTER(MessiTuning)],
    "messi_set_tuning": [_P, ctypes.POINTER(MessiTuning)],
    "messi_debug_tc_gemm": [_P, _P, _U32, _U32, _U32, _U32, _P],
    "messi_check": [_P, _P],
    "messi_summarize": [_P, _U64, _U32, _U32, _U32, _P, _P],
    "messi_index_layout": [_P, _P, _P, _P],
    "messi_breakpoints": [_U32, _P],
    "messi_server_create": [_P, ctypes.POINTER(MessiServerConfig), ctypes.POINTER(_P)],
    "messi_server_submit": [_P, _P, _U32, _I, _U32, ctypes.POINTER(_U64)],
    "messi_server_poll": [_P, _U64, _P, _P, ctypes.POINTER(ctypes.c_double), _U64],
    "messi_server_get_stats": [_P, ctypes.POINTER(MessiServerStats)],
    "messi_server_pause": [_P, _I],
    "messi_server_destroy": [_P],
    "messi_debug_set_lock_fault": [_P, _U32, _I],
    "messi_last_error": [],
}
for _name, _args in _SIGS.items():
    _fn = getattr(_lib, _name)
    _fn.argtypes = _args
    _fn.restype = ctypes.c_char_p if _name == "messi_last_error" else (
        None if _name in ("messi_free", "messi_server_destroy") else _I)


class MessiError(RuntimeError):
    def __init__(self, status: int, where: str):
        msg = _lib.messi_last_error().decode(errors="replace")
        super().__init__(f"{where}: {STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


def _check(st: int, where: str):
    if st != 0:
        raise MessiError(st, where)


def exported_symbols() -> list[str]:
    return list(_SIGS)


# ------------------------------------------------------------- marshalling
def _is_torch(x) -> bool:
    return type(x).__module__.startswith("torch")


def _ptr(x):
    """(pointer, keepalive, is_cuda) of a torch tensor or numpy array."""
    if _is_torch(x):
        if not x.is_contiguous():
            raise ValueError("tensor must be contiguous")
        return ctypes.c_void_p(x.data_ptr()), x, bool(x.is_cuda)
    a = np.ascontiguousarray(x)
    return ctypes.c_void_p(a.ctypes.data), a, False


def _stream(stream, like=None):
    if stream is not None:
        return ctypes.c_void_p(int(stream))
    if like is not None and _is_torch(like) and like.is_cuda:
        import torch

        return ctypes.c_void_p(torch.cuda.current_stream(like.device).cuda_stream)
    return ctypes.c_void_p(0)


def _f32(x):
    if _is_torch(x):
        import torch

        return x if x.dtype == torch.float32 and x.is_contiguous() else x.to(torch.float32).contiguous()
    return np.ascontiguousarray(x, dtype=np.float32)


@dataclass
class Index:
    handle: ctypes.c_void_p
    n: int
    len: int
    segments: int
    cardinality: int
    _batch_mode: int = 1            # the library's default: MESSI_BATCH_TC_SCREEN

    def __del__(self):
        h = getattr(self, "handle", None)
        if h:
            _lib.messi_free(h)
            self.handle = None

    def free(self):
        self.__del__()


# ------------------------------------------------------------------- calls
def messi_build(series, segments: int = 16, cardinality: int = 256, leaf_capacity: int = 0,
                stream=None) -> Index:
    series = _f32(series)
    n, length = series.shape
    p, keep, _ = _ptr(series)
    cfg = MessiConfig()
    cfg.leaf_capacity = leaf_capacity
    out = ctypes.c_void_p()
    _check(_lib.messi_build(p, n, length, segments, cardinality, ctypes.byref(cfg),
                            _stream(stream, series), ctypes.byref(out)), "messi_build")
    return Index(out, n, length, segments, cardinality)


def messi_windows(series, n: int, stride: int = 1, znorm: bool = True, out=None, stream=None):
    """Every length-n window of the 1-D device tensor `series` at `stride`, as
    a [count, n] float32 device tensor (row i starts at i * stride),
    z-normalised per window when `znorm`."""
    import torch

    series = _f32(series)
    if not _is_torch(series) or not series.is_cuda or series.ndim != 1:
        raise ValueError("series must be a 1-D CUDA tensor")
    length = series.shape[0]
    if n < 1 or stride < 1 or length < n:
        raise ValueError("need 1 <= n <= len(series) and stride >= 1")
    count = (length - n) // stride + 1
    if out is None:
        out = torch.empty((count, n), dtype=torch.float32, device=series.device)
    elif tuple(out.shape) != (count, n) or out.dtype != torch.float32 or not out.is_contiguous():
        raise ValueError(f"out must be a contiguous float32 tensor of shape ({count}, {n})")
    got = ctypes.c_uint64(0)
    _check(_lib.messi_windows(ctypes.c_void_p(series.data_ptr()), length, n, stride, 1 if znorm else 0,
                              ctypes.c_void_p(out.data_ptr()), ctypes.byref(got), _stream(stream, series)),
           "messi_windows")
    return out


def messi_build_windows(series, n: int, stride: int = 1, znorm: bool = True, segments: int = 16,
                        cardinality: int = 256, leaf_capacity: int = 0, stream=None) -> Index:
    """Index every length-n window of one long device series (subsequence
    matching): ids of the answers are window numbers, start = id * stride.
    The window matrix is freed once the index holds its own copy."""
    w = messi_windows(series, n, stride, znorm, stream=stream)
    try:
        return messi_build(w, segments, cardinality, leaf_capacity, stream)
    finally:
        del w


def _outputs(nq, k, on_cuda, device=None):
    if on_cuda:
        import torch

        return (torch.empty((nq, k), dtype=torch.int64, device=device),
                torch.empty((nq, k), dtype=torch.float32, device=device))
    return np.empty((nq, k), dtype=np.int64), np.empty((nq, k), dtype=np.float32)


def messi_query(index: Index, queries, k: int = 1, dist: int = MESSI_ED, window: int = 0,
                ids=None, dists=None, stream=None):
    """Exact k-NN of every query row; returns (ids int64 [nq,k], dists f32 [nq,k])."""
    queries = _f32(queries)
    if queries.ndim == 1:
        queries = queries.reshape(1, -1)
    nq = queries.shape[0]
    qp, qkeep, qcuda = _ptr(queries)
    if ids is None or dists is None:
        ids, dists = _outputs(nq, k, qcuda, queries.device if qcuda else None)
    ip, ikeep, _ = _ptr(ids)
    dp, dkeep, _ = _ptr(dists)
    _check(_lib.messi_query(index.handle, qp, nq, k, dist, window, ip, dp, _stream(stream, queries)),
           "messi_query")
    return ids, dists


def messi_query_batched(index: Index, queries, k: int = 1, dist: int = MESSI_ED, window: int = 0,
                        batch: int = 0, ids=None, dists=None, stream=None):
    queries = _f32(queries)
    if queries.ndim == 1:
        queries = queries.reshape(1, -1)
    nq = queries.shape[0]
    qp, qkeep, qcuda = _ptr(queries)
    if ids is None or dists is None:
        ids, dists = _outputs(nq, k, qcuda, queries.device if qcuda else None)
    ip, ikeep, _ = _ptr(ids)
    dp, dkeep, _ = _ptr(dists)
    _check(_lib.messi_query_batched(index.handle, qp, nq, k, dist, window, batch, ip, dp,
                                    _stream(stream, queries)), "messi_query_batched")
    return ids, dists


def messi_lower_bounds(index: Index, query, dist: int = MESSI_ED, window: int = 0, out=None, stream=None):
    query = _f32(query).reshape(-1)
    qp, qkeep, qcuda = _ptr(query)
    if out is None:
        if qcuda:
            import torch

            out = torch.empty(index.n, dtype=torch.float32, device=query.device)
        else:
            out = np.empty(index.n, dtype=np.float32)
    op, okeep, _ = _ptr(out)
    _check(_lib.messi_lower_bounds(index.handle, qp, dist, window, op, _stream(stream, query)),
           "messi_lower_bounds")
    return out


def messi_lower_bounds_noalloc(index: Index, query, out, dist: int = MESSI_ED, window: int = 0, stream=None):
    """Lower bounds into a caller-provided device tensor ``out`` (n float32)
    without any device allocation by the library; ``query`` must be on the
    device too.  Calls sharing the library's fixed scratch must not overlap."""
    qp, qkeep, _ = _ptr(query)
    op, okeep, _ = _ptr(out)
    _check(_lib.messi_lower_bounds_noalloc(index.handle, qp, dist, window, op, _stream(stream, query)),
           "messi_lower_bounds_noalloc")
    return out


def messi_summarize(series, segments: int = 16, cardinality: int = 256, stream=None):
    """iSAX words of every row: uint8 [n, 16] (byte s = symbol of segment s)."""
    series = _f32(series)
    n, length = series.shape
    sp, skeep, scuda = _ptr(series)
    if scuda:
        import torch

        out = torch.empty((n, 16), dtype=torch.uint8, device=series.device)
    else:
        out = np.empty((n, 16), dtype=np.uint8)
    op, okeep, _ = _ptr(out)
    _check(_lib.messi_summarize(sp, n, length, segments, cardinality, op, _stream(stream, series)),
           "messi_summarize")
    return out


def messi_index_get_info(index: Index) -> dict:
    info = MessiIndexInfo()
    _check(_lib.messi_index_get_info(index.handle, ctypes.byref(info)), "messi_index_get_info")
    return info.as_dict()


def messi_index_layout(index: Index):
    """(order uint32 [n], leaf_off uint64 [L+1], leaf_depth uint8 [L]) on the host."""
    info = messi_index_get_info(index)
    L = info["n_leaves"]
    order = np.empty(index.n, dtype=np.uint32)
    off = np.empty(L + 1, dtype=np.uint64)
    depth = np.empty(L, dtype=np.uint8)
    _check(_lib.messi_index_layout(index.handle, order.ctypes.data, off.ctypes.data, depth.ctypes.data),
           "messi_index_layout")
    return order, off, depth


def messi_query_stats(index: Index) -> dict:
    st = MessiStats()
    _check(_lib.messi_query_stats(index.handle, ctypes.byref(st)), "messi_query_stats")
    return st.as_dict()


def messi_set_profiling(index: Index, level=2):
    """0 off; 1 events around the dominant kernel launches; 2 also per query
    (True means 2, False 0)."""
    level = 2 if level is True else 0 if level is False else int(level)
    _check(_lib.messi_set_profiling(index.handle, level), "messi_set_profiling")


def messi_set_batch_mode(index: Index, mode: int):
    _check(_lib.messi_set_batch_mode(index.handle, mode), "messi_set_batch_mode")
    index._batch_mode = mode


def messi_autotune(index: Index, queries, k: int = 1, stream=None) -> dict:
    """Time the batched shapes of the index's batch mode on `queries` (device
    rows) and keep the fastest; returns the choice."""
    queries = _f32(queries)
    qp, qkeep, qcuda = _ptr(queries)
    if not qcuda:
        raise MessiError(1, "messi_autotune: queries must be a device tensor")
    t = MessiTuning()
    _check(_lib.messi_autotune(index.handle, qp, queries.shape[0], k, _stream(stream), ctypes.byref(t)),
           "messi_autotune")
    return t.as_dict()


def messi_set_tuning(index: Index, batch: int, chunk_tiles: int = 32, ctas_per_sm: int = 2):
    t = MessiTuning(batch=batch, chunk_tiles=chunk_tiles, ctas_per_sm=ctas_per_sm)
    _check(_lib.messi_set_tuning(index.handle, ctypes.byref(t)), "messi_set_tuning")


def autotune_cached(index: Index, queries, k: int = 1, cache: str | None = None, stream=None) -> dict:
    """messi_autotune with a JSON cache keyed by collection shape, batch mode,
    k and device name: a cached choice is applied without timing."""
    import json

    info = messi_index_get_info(index)
    key = None
    if cache:
        try:
            import torch

            dev = torch.cuda.get_device_name()
        except Exception:
            dev = "cuda"
        key = f"{info['n_series']}x{info['len']}:mode{index._batch_mode}:k{k}:{dev}"
        try:
            with open(cache) as f:
                table = json.load(f)
        except (OSError, ValueError):
            table = {}
        if key in table:
            t = table[key]
            messi_set_tuning(index, t["batch"], t["chunk_tiles"], t["ctas_per_sm"])
            return t
    t = messi_autotune(index, queries, k, stream)
    if cache:
        table[key] = t
        with open(cache, "w") as f:
            json.dump(table, f, indent=1, sort_keys=True)
    return t


def messi_debug_tc_gemm(a_tile: np.ndarray, b_tile: np.ndarray, k: int, n: int, lbo: int, sbo: int) -> np.ndarray:
    """One 128 x n x k tensor-core tile, D = A B^T (operands as f16 bit patterns
    already in the tensor-core layout); returns D as float32 [128, n]."""
    a = np.ascontiguousarray(a_tile, dtype=np.uint16)
    b = np.ascontiguousarray(b_tile, dtype=np.uint16)
    d = np.empty((128, n), dtype=np.float32)
    _check(_lib.messi_debug_tc_gemm(a.ctypes.data, b.ctypes.data, k, n, lbo, sbo, d.ctypes.data),
           "messi_debug_tc_gemm")
    return d


def messi_debug_set_lock_fault(index: Index, spin_limit: int = 1 << 22, hold_lock: bool = False):
    """Test hook: tries of the k-array lock before a timeout, and whether every
    per-query call starts with that lock held (defaults restore normal use)."""
    _check(_lib.messi_debug_set_lock_fault(index.handle, spin_limit, 1 if hold_lock else 0),
           "messi_debug_set_lock_fault")


def messi_check(index: Index, stream=None):
    _check(_lib.messi_check(index.handle, _stream(stream)), "messi_check")


def messi_breakpoints(cardinality: int) -> np.ndarray:
    out = np.empty(cardinality - 1, dtype=np.float64)
    _check(_lib.messi_breakpoints(cardinality, out.ctypes.data), "messi_breakpoints")
    return out


def messi_free(index: Index):
    """Release the index's device memory now (also done when it is collected)."""
    index.free()


# ----------------------------------------------------------------- serving
class Server:
    def __init__(self, handle, index):
        self.handle = handle
        self.index = index          # the index must outlive the server

    def __del__(self):
        h = getattr(self, "handle", None)
        if h:
            _lib.messi_server_destroy(h)
            self.handle = None


def messi_server_create(index: Index, max_batch: int = 0, max_k: int = 0, streams: int = 0,
                        max_queued: int = 0, mem_budget: int = 0) -> Server:
    cfg = MessiServerConfig()
    cfg.max_batch, cfg.max_k, cfg.streams, cfg.max_queued, cfg.mem_budget = (max_batch, max_k, streams,
                                                                             max_queued, mem_budget)
    out = ctypes.c_void_p()
    _check(_lib.messi_server_create(index.handle, ctypes.byref(cfg), ctypes.byref(out)), "messi_server_create")
    return Server(out, index)


def messi_server_submit(server: Server, query, k: int = 1, dist: int = MESSI_ED, window: int = 0) -> int:
    q = np.ascontiguousarray(query, dtype=np.float32).reshape(-1)
    t = ctypes.c_uint64()
    _check(_lib.messi_server_submit(server.handle, q.ctypes.data, k, dist, window, ctypes.byref(t)),
           "messi_server_submit")
    return t.value


def messi_server_poll(server: Server, ticket: int, k: int, wait_us: int = 0):
    """(ids, dists, latency_ms) of a finished request, or None while it runs."""
    ids = np.empty(k, dtype=np.int64)
    d = np.empty(k, dtype=np.float32)
    lat = ctypes.c_double()
    st = _lib.messi_server_poll(server.handle, ticket, ids.ctypes.data, d.ctypes.data, ctypes.byref(lat), wait_us)
    if st == 5:
        return None
    _check(st, "messi_server_poll")
    return ids, d, lat.value


def messi_server_get_stats(server: Server) -> dict:
    out = MessiServerStats()
    _check(_lib.messi_server_get_stats(server.handle, ctypes.byref(out)), "messi_server_get_stats")
    return out.as_dict()


def messi_server_pause(server: Server, paused: bool = True):
    _check(_lib.messi_server_pause(server.handle, 1 if paused else 0), "messi_server_pause")


def messi_server_destroy(server: Server):
    server.__del__()


def messi_last_error() -> str:
    return _lib.messi_last_error().decode(errors="replace")
