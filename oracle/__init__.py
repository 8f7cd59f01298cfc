"""FP64 CPU oracle for the MESSI exact k-NN method (arXiv 2110.07519).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and
``bench.py``'s CPU-baseline / reference leg may import this package.  It
shares no code with the CUDA library in ``paper_2110_07519_gb300`` and never
imports it.

The numeric routines live in ``messi_oracle.c`` (plain C, FP64, built with
``-ffp-contract=off``); this module loads them with ctypes and adds:

* ``leaf_partition`` -- the leaf grouping of Sec. 2.2 / Sec. 3.2 (a node
  splits one iSAX bit at a time while it holds more than ``cap`` series),
  written as plain Python over the sorted keys;
* ``knn_stream`` -- the brute-force k-NN of Sec. 2.1 over a sequence of row
  blocks (the k best of a union are the k best of the per-block k best).

Parity status: every routine here is pinned by ``tests/test_oracle_pins.py``
(closed forms, textbook values, invariants, brute force); none is unpinned.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from typing import Iterable, Sequence

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "messi_oracle.c")
# MESSI_ORACLE_LIB names a prebuilt library to load instead (the planted-
# mistake tests compile mutated copies of the source and load them this way)
_LIB_PATH = os.environ.get("MESSI_ORACLE_LIB") or os.path.join(_HERE, "liboracle.so")
_lib = None

ED, DTW = 0, 1


def build(force: bool = False) -> str:
    """Compile ``messi_oracle.c`` into ``oracle/liboracle.so`` with gcc."""
    if os.environ.get("MESSI_ORACLE_LIB"):
        return _LIB_PATH
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < max(
        os.path.getmtime(_SRC), os.path.getmtime(os.path.join(_HERE, "messi_oracle.h"))
    ):
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-fopenmp", "-ffp-contract=off", "-fno-fast-math", "-fPIC",
               "-shared", "-Wall", "-o", tmp, _SRC, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    if _lib is not None:
        return _lib
    build()
    lib = ctypes.CDLL(_LIB_PATH)
    P = ctypes.c_void_p
    I, I64, D = ctypes.c_int, ctypes.c_int64, ctypes.c_double
    sig = {
        "orc_breakpoints": (None, [I, P]),
        "orc_paa": (None, [P, I, I, P]),
        "orc_sax": (None, [P, I, I, P, P]),
        "orc_summarize": (None, [P, I64, I, I, I, P, P]),
        "orc_isax_key": (None, [P, I, I, P]),
        "orc_ed2": (D, [P, P, I]),
        "orc_mindist_ed2": (D, [P, P, I, I, I, P]),
        "orc_envelope": (None, [P, I, I, P, P]),
        "orc_lb_keogh2": (D, [P, P, P, I]),
        "orc_mindist_dtw2": (D, [P, P, P, I, I, I, P]),
        "orc_dtw2": (D, [P, P, I, I]),
        "orc_lb_improved2": (D, [P, P, P, P, I, I]),
        "orc_knn": (None, [P, I64, I, P, I, I, I, I, I64, I, P, P]),
        "orc_max_threads": (I, []),
        "orc_windows": (I64, [P, I64, I, I, I, P]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def _f32(x) -> np.ndarray:
    return np.ascontiguousarray(x, dtype=np.float32)


def _f64(x) -> np.ndarray:
    return np.ascontiguousarray(x, dtype=np.float64)


def max_threads() -> int:
    return int(_load().orc_max_threads())


# ------------------------------------------------------------------ Sec. 2.2
def breakpoints(card: int) -> np.ndarray:
    """beta_1..beta_{c-1}: N(0,1) quantiles j/c (Sec. 2.2)."""
    out = np.empty(card - 1, dtype=np.float64)
    _load().orc_breakpoints(card, _ptr(out))
    return out


def paa(x, w: int) -> np.ndarray:
    """Segment means of one series (Sec. 2.2)."""
    x = _f32(x)
    out = np.empty(w, dtype=np.float64)
    _load().orc_paa(_ptr(x), x.shape[-1], w, _ptr(out))
    return out


def sax(p, card: int, beta=None) -> np.ndarray:
    """Symbols of a PAA vector: count of breakpoints <= value (Sec. 2.2)."""
    p = _f64(p)
    beta = breakpoints(card) if beta is None else _f64(beta)
    out = np.empty(p.shape[-1], dtype=np.uint8)
    _load().orc_sax(_ptr(p), p.shape[-1], card, _ptr(beta), _ptr(out))
    return out


def summarize(data, w: int, card: int) -> np.ndarray:
    """iSAX words (N x w symbols) of every row of ``data`` (Sec. 3.2, Alg. 3)."""
    data = _f32(data)
    N, n = data.shape
    beta = breakpoints(card)
    out = np.empty((N, w), dtype=np.uint8)
    _load().orc_summarize(_ptr(data), N, n, w, card, _ptr(beta), _ptr(out))
    return out


def isax_key(sym, card: int) -> int:
    """Interleaved 128-bit iSAX key as a Python int (MSB-first bit planes)."""
    sym = np.ascontiguousarray(sym, dtype=np.uint8)
    key = np.zeros(4, dtype=np.uint32)
    _load().orc_isax_key(_ptr(sym), sym.shape[-1], card, _ptr(key))
    return (int(key[0]) << 96) | (int(key[1]) << 64) | (int(key[2]) << 32) | int(key[3])


def isax_keys(words: np.ndarray, card: int) -> list[int]:
    return [isax_key(words[i], card) for i in range(words.shape[0])]


# ------------------------------------------------------------------ Sec. 2.1
def ed2(q, x) -> float:
    q, x = _f32(q), _f32(x)
    return float(_load().orc_ed2(_ptr(q), _ptr(x), q.shape[-1]))


# ------------------------------------------------------- Property 1, Sec. 4
def mindist_ed2(paa_q, sym, m: int, card: int, beta=None) -> float:
    paa_q = _f64(paa_q)
    sym = np.ascontiguousarray(sym, dtype=np.uint8)
    beta = breakpoints(card) if beta is None else _f64(beta)
    return float(_load().orc_mindist_ed2(_ptr(paa_q), _ptr(sym), sym.shape[-1], m, card, _ptr(beta)))


# ------------------------------------------------------------------ Sec. 3.4
def envelope(q, r: int):
    q = _f32(q)
    n = q.shape[-1]
    U = np.empty(n, dtype=np.float64)
    L = np.empty(n, dtype=np.float64)
    _load().orc_envelope(_ptr(q), n, r, _ptr(U), _ptr(L))
    return U, L


def lb_keogh2(U, L, x) -> float:
    U, L, x = _f64(U), _f64(L), _f32(x)
    return float(_load().orc_lb_keogh2(_ptr(U), _ptr(L), _ptr(x), x.shape[-1]))


def lb_improved2(q, x, r: int) -> float:
    """LB_Improved (squared): LB_Keogh of x against q's envelope plus q against
    the envelope of x clamped into q's envelope (window r)."""
    q, x = _f32(q), _f32(x)
    U, L = envelope(q, r)
    return float(_load().orc_lb_improved2(_ptr(q), _ptr(U), _ptr(L), _ptr(x), q.shape[-1], r))


def mindist_dtw2(paa_u, paa_l, sym, m: int, card: int, beta=None) -> float:
    paa_u, paa_l = _f64(paa_u), _f64(paa_l)
    sym = np.ascontiguousarray(sym, dtype=np.uint8)
    beta = breakpoints(card) if beta is None else _f64(beta)
    return float(_load().orc_mindist_dtw2(_ptr(paa_u), _ptr(paa_l), _ptr(sym), sym.shape[-1],
                                          m, card, _ptr(beta)))


def envelope_paa(q, r: int, w: int):
    """PAA (segment means, FP64) of the LB_Keogh envelope (Sec. 3.4)."""
    U, L = envelope(q, r)
    n = U.shape[0]
    m = n // w
    pu = np.array([sum(float(v) for v in U[s * m:(s + 1) * m]) / m for s in range(w)])
    pl = np.array([sum(float(v) for v in L[s * m:(s + 1) * m]) / m for s in range(w)])
    return pu, pl


def dtw2(q, x, r: int) -> float:
    q, x = _f32(q), _f32(x)
    return float(_load().orc_dtw2(_ptr(q), _ptr(x), q.shape[-1], r))


# ------------------------------------------------------------- k-NN, Sec. 5.4
def knn(data, queries, k: int, dist: int = ED, r: int = 0, id_base: int = 0,
        threads: int = 0):
    """Brute-force exact k-NN: (ids[nq,k] int64, d2[nq,k] FP64 squared)."""
    data = _f32(data)
    queries = _f32(queries)
    if queries.ndim == 1:
        queries = queries[None, :]
    N, n = data.shape
    nq = queries.shape[0]
    ids = np.empty((nq, k), dtype=np.int64)
    d2 = np.empty((nq, k), dtype=np.float64)
    _load().orc_knn(_ptr(data), N, n, _ptr(queries), nq, k, dist, r, id_base, threads,
                    _ptr(ids), _ptr(d2))
    return ids, d2


def windows(series, n: int, stride: int = 1, znorm: bool = True) -> np.ndarray:
    """Every length-n window of a 1-D series at `stride` ([count, n] float32),
    z-normalised per window by the FP64 steps of ``orc_windows``."""
    series = _f32(series).reshape(-1)
    count = (series.shape[0] - n) // stride + 1
    out = np.empty((count, n), dtype=np.float32)
    got = _load().orc_windows(_ptr(series), series.shape[0], n, stride, 1 if znorm else 0, _ptr(out))
    assert got == count
    return out


def merge_topk(parts: Sequence[tuple[np.ndarray, np.ndarray]], k: int):
    """k best by (d2, id) of the union of several per-block k-best lists."""
    ids = np.concatenate([p[0] for p in parts], axis=1)
    d2 = np.concatenate([p[1] for p in parts], axis=1)
    out_i = np.empty((ids.shape[0], k), dtype=np.int64)
    out_d = np.empty((ids.shape[0], k), dtype=np.float64)
    for q in range(ids.shape[0]):
        order = sorted(range(ids.shape[1]), key=lambda e: (d2[q, e], ids[q, e]))[:k]
        out_i[q] = ids[q, order]
        out_d[q] = d2[q, order]
    return out_i, out_d


def knn_stream(blocks: Iterable[tuple[int, np.ndarray]], queries, k: int, dist: int = ED,
               r: int = 0, threads: int = 0):
    """Brute-force k-NN over row blocks ``(first_id, rows)`` covering the data."""
    best = None
    for first_id, rows in blocks:
        part = knn(rows, queries, k, dist, r, id_base=first_id, threads=threads)
        best = part if best is None else merge_topk([best, part], k)
    return best


# ------------------------------------------------- leaf grouping, Sec. 3.2
def leaf_partition(words: np.ndarray, card: int, cap: int):
    """Leaf layout of the iSAX tree over ``words`` (N x w symbols).

    Returns ``(order, leaf_off, leaf_depth)``: ``order`` lists row ids sorted
    by (interleaved key, id); leaf ``i`` holds ``order[leaf_off[i]:leaf_off[i+1]]``
    and is the trie node whose key prefix has ``leaf_depth[i]`` bits.  The root
    has one child per value of the first bit of every segment (depth w); a
    node holding more than ``cap`` series is replaced by its two children on
    the next interleaved bit (Sec. 2.2: a split refines one segment by one
    bit), empty children are dropped, and a node whose prefix is already the
    whole key stays a leaf whatever its size.
    """
    N, w = words.shape
    b = int(card).bit_length() - 1
    total = w * b
    keys = isax_keys(words, card)
    order = sorted(range(N), key=lambda i: (keys[i], i))
    sk = [keys[i] for i in order]

    def bit(key, p):                      # p = 0 is the most significant of 128
        return (key >> (127 - p)) & 1

    def prefix(key, d):
        return key >> (128 - d)

    leaves: list[tuple[int, int]] = []    # (start, depth)
    # root children: runs of equal first-w-bit prefix
    start = 0
    roots = []
    for i in range(1, N + 1):
        if i == N or prefix(sk[i], w) != prefix(sk[start], w):
            roots.append((start, i))
            start = i
    stack = [(lo, hi, w) for (lo, hi) in reversed(roots)]
    while stack:
        lo, hi, d = stack.pop()
        if hi - lo <= cap or d >= total:
            leaves.append((lo, d))
            continue
        mid = lo
        while mid < hi and bit(sk[mid], d) == 0:
            mid += 1
        kids = [(lo, mid, d + 1), (mid, hi, d + 1)]
        for c in reversed(kids):
            if c[1] > c[0]:
                stack.append(c)
    leaves.sort()
    leaf_off = np.array([s for s, _ in leaves] + [N], dtype=np.int64)
    leaf_depth = np.array([d for _, d in leaves], dtype=np.int32)
    return np.array(order, dtype=np.int64), leaf_off, leaf_depth
