"""Oracle for queue-driven Bellman-Ford SSSP -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline / reference
legs of ``bench.py`` may import this package.  The library under
``paper_2608_21826_gb300`` never imports it and shares no code with it.

``sssp_oracle.c`` holds the plain sequential algorithms (FIFO label-correcting
Bellman-Ford, the same with the parent-graph search for negative cycles,
Dijkstra, Floyd-Warshall, the predecessor-tree invariant, and distances with
negative cycles resolved to minus infinity).  This
module compiles it with gcc on first use (or from ``build()``) and exposes thin
numpy wrappers.  ``broker_queue.py`` models the Broker Queue of Algorithm 1.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "sssp_oracle.c")
_OUT_DIR = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_OUT_DIR, "liboracle.so")
_lock = threading.Lock()
_lib = None

OK, NEG_CYCLE, RANGE = 0, 1, 4
INF32 = 2147483647


def build(force: bool = False) -> str:
    """Compile ``sssp_oracle.c`` into ``_build/liboracle.so`` (plain gcc -O2)."""
    os.makedirs(_OUT_DIR, exist_ok=True)
    stale = (not os.path.exists(_LIB_PATH)
             or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC))
    if force or stale:
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-shared", "-fPIC",
                               "-o", tmp, _SRC])
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _bind(lib):
    p32 = ctypes.POINTER(ctypes.c_int32)
    p64 = ctypes.POINTER(ctypes.c_int64)
    i32 = ctypes.c_int32
    lib.oracle_spfa.argtypes = [i32, p32, p32, p32, i32, p32, p32, p64]
    lib.oracle_spfa.restype = ctypes.c_int
    for name in ("oracle_dijkstra", "oracle_fw"):
        f = getattr(lib, name)
        f.argtypes = [i32, p32, p32, p32, i32, p32, p32]
        f.restype = ctypes.c_int
    lib.oracle_spfa_cycle_search.argtypes = [i32, p32, p32, p32, i32, p32, p32, p64, p32]
    lib.oracle_spfa_cycle_search.restype = ctypes.c_int
    lib.oracle_spfa_neg_inf.argtypes = [i32, p32, p32, p32, i32, p32, p32]
    lib.oracle_spfa_neg_inf.restype = ctypes.c_int
    lib.oracle_check_pred.argtypes = [i32, p32, p32, p32, i32, p32, p32]
    lib.oracle_check_pred.restype = ctypes.c_int
    lib.oracle_reached_edges.argtypes = [i32, p32, p32]
    lib.oracle_reached_edges.restype = ctypes.c_int64
    return lib


def _load():
    global _lib
    with _lock:
        if _lib is None:
            _lib = _bind(ctypes.CDLL(build()))
    return _lib


class Variant:
    """The same wrappers bound to another build of the oracle source (used by
    the mutation tests, which compile deliberately broken copies)."""

    def __init__(self, so_path: str):
        self._lib = _bind(ctypes.CDLL(so_path))

    def spfa(self, *a):
        return spfa(*a, _lib=self._lib)

    def dijkstra(self, *a):
        return dijkstra(*a, _lib=self._lib)

    def spfa_cycle_search(self, *a):
        return spfa_cycle_search(*a, _lib=self._lib)

    def spfa_neg_inf(self, *a):
        return spfa_neg_inf(*a, _lib=self._lib)

    def floyd_warshall(self, *a):
        return floyd_warshall(*a, _lib=self._lib)


def _i32(a) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(a, dtype=np.int32))


def _p(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_int32))


def _csr(row_ptr, col, w):
    row_ptr, col, w = _i32(row_ptr), _i32(col), _i32(w)
    V = len(row_ptr) - 1
    if V < 1 or len(col) != row_ptr[-1] or len(w) != len(col):
        raise ValueError("malformed CSR")
    return V, row_ptr, col, w


def spfa(row_ptr, col, w, src: int, _lib=None):
    """FIFO label-correcting Bellman-Ford.  Returns (status, dist, hops, scanned)."""
    V, row_ptr, col, w = _csr(row_ptr, col, w)
    dist = np.empty(V, np.int32)
    hops = np.empty(V, np.int32)
    scanned = ctypes.c_int64(0)
    st = (_lib or _load()).oracle_spfa(V, _p(row_ptr), _p(col), _p(w), int(src), _p(dist),
                             _p(hops), ctypes.byref(scanned))
    if st < 0:
        raise ValueError(f"oracle_spfa rejected its input ({st})")
    return st, dist, hops, scanned.value


def spfa_cycle_search(row_ptr, col, w, src: int, _lib=None):
    """FIFO label-correcting Bellman-Ford with the amortized parent-graph
    search for negative cycles (exact, and fast on large graphs with a
    negative cycle).  Returns (status, dist, hops, scanned, cycle_vertex):
    the labels and scan count equal spfa's when no negative cycle is
    reachable; cycle_vertex is a vertex on the cycle the search found, or -1."""
    V, row_ptr, col, w = _csr(row_ptr, col, w)
    dist = np.empty(V, np.int32)
    hops = np.empty(V, np.int32)
    scanned = ctypes.c_int64(0)
    cv = ctypes.c_int32(-1)
    st = (_lib or _load()).oracle_spfa_cycle_search(V, _p(row_ptr), _p(col), _p(w), int(src),
                                                    _p(dist), _p(hops), ctypes.byref(scanned),
                                                    ctypes.byref(cv))
    if st < 0:
        raise ValueError(f"oracle_spfa_cycle_search failed ({st})")
    return st, dist, hops, scanned.value, cv.value


NEG_INF_DIST = -2147483648      # dist of a vertex reachable from a negative cycle
NEG_INF_HOPS = -2


def spfa_neg_inf(row_ptr, col, w, src: int, _lib=None):
    """Distances with negative cycles resolved: vertices reachable from a
    reachable negative cycle get (INT32_MIN, -2), the others their
    lexicographic labels.  Returns (status, dist, hops)."""
    V, row_ptr, col, w = _csr(row_ptr, col, w)
    dist = np.empty(V, np.int32)
    hops = np.empty(V, np.int32)
    st = (_lib or _load()).oracle_spfa_neg_inf(V, _p(row_ptr), _p(col), _p(w), int(src),
                                               _p(dist), _p(hops))
    if st < 0:
        raise ValueError(f"oracle_spfa_neg_inf rejected its input ({st})")
    return st, dist, hops


def dijkstra(row_ptr, col, w, src: int, _lib=None):
    """Lexicographic Dijkstra (non-negative weights).  Returns (dist, hops)."""
    V, row_ptr, col, w = _csr(row_ptr, col, w)
    dist = np.empty(V, np.int32)
    hops = np.empty(V, np.int32)
    st = (_lib or _load()).oracle_dijkstra(V, _p(row_ptr), _p(col), _p(w), int(src),
                                 _p(dist), _p(hops))
    if st < 0:
        raise ValueError(f"oracle_dijkstra rejected its input ({st})")
    return dist, hops


def floyd_warshall(row_ptr, col, w, src: int, _lib=None):
    """Floyd-Warshall on (dist, hops) pairs, V <= 512.  Returns (status, dist, hops)."""
    V, row_ptr, col, w = _csr(row_ptr, col, w)
    dist = np.empty(V, np.int32)
    hops = np.empty(V, np.int32)
    st = (_lib or _load()).oracle_fw(V, _p(row_ptr), _p(col), _p(w), int(src), _p(dist),
                           _p(hops))
    if st < 0:
        raise ValueError(f"oracle_fw rejected its input ({st})")
    return st, dist, hops


def check_pred(row_ptr, col, w, src: int, dist, pred) -> bool:
    """Tight, acyclic predecessor tree rooted at src (see sssp_oracle.c)."""
    V, row_ptr, col, w = _csr(row_ptr, col, w)
    dist, pred = _i32(dist), _i32(pred)
    return bool(_load().oracle_check_pred(V, _p(row_ptr), _p(col), _p(w),
                                          int(src), _p(dist), _p(pred)))


def reached_edges(row_ptr, dist) -> int:
    """Directed edges whose tail is reachable (dist < INT32_MAX)."""
    row_ptr, dist = _i32(row_ptr), _i32(dist)
    return int(_load().oracle_reached_edges(len(row_ptr) - 1, _p(row_ptr), _p(dist)))
