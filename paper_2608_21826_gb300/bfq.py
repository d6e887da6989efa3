"""Thin ctypes binding of libbfq (the C ABI declared in include/bfq.h).

Each ``bfq_*`` function here marshals its arguments (numpy arrays, torch
tensors, raw pointers, streams) and calls the C entry point of the same name;
all computation runs in the library's CUDA kernels.  There is no fallback:
if the library cannot be built or loaded, ``lib()`` raises.  BFQ_LIBRARY may
name another build of the library to load instead of the in-tree one.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

from . import _build

OK, NEG_CYCLE, FULL, EMPTY, RANGE, PENDING = 0, 1, 2, 3, 4, 5
ERR_INVALID, ERR_OOM, ERR_TIMEOUT, ERR_CUDA, ERR_BUDGET = -1, -2, -3, -4, -5
QUEUE_BQ, QUEUE_BWD, QUEUE_BQ_WARP, QUEUE_BWD_WARP = 0, 1, 2, 3
QUEUE_FORM_AUTO, QUEUE_FORM_EXACT, QUEUE_FORM_SINGLE_SHOT = 0, 1, 2
INF32 = 2147483647


class BfqError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"bfq error {code}: {msg}")
        self.code = code


class Tune(ctypes.Structure):
    _fields_ = [("ctas_per_sm", ctypes.c_int32), ("threads_per_cta", ctypes.c_int32),
                ("queues_per_cta", ctypes.c_int32), ("batch_items", ctypes.c_int32),
                ("hub_degree", ctypes.c_int32), ("chunk_edges", ctypes.c_int32),
                ("spin_limit", ctypes.c_int64), ("time_limit_ms", ctypes.c_int64),
                ("l2_persist_pct", ctypes.c_int32), ("test_phantom_items", ctypes.c_int32),
                ("share_div", ctypes.c_int32), ("chunk_batch", ctypes.c_int32),
                ("neg_cycle_mode", ctypes.c_int32), ("cycle_walk_hops", ctypes.c_int32),
                ("relax_atomic", ctypes.c_int32), ("batch_budget_klabels", ctypes.c_int32),
                ("kernel_ctas", ctypes.c_int32), ("queue_form", ctypes.c_int32),
                ("small_path", ctypes.c_int32), ("small_threads", ctypes.c_int32)]


class Stats(ctypes.Structure):
    _fields_ = [("dequeued", ctypes.c_int64), ("relaxed", ctypes.c_int64),
                ("updated", ctypes.c_int64), ("enqueued", ctypes.c_int64),
                ("steals", ctypes.c_int64), ("hub_chunks", ctypes.c_int64),
                ("m_reached", ctypes.c_int64), ("reached", ctypes.c_int64),
                ("V", ctypes.c_int64), ("E", ctypes.c_int64),
                ("grid", ctypes.c_int32), ("block", ctypes.c_int32),
                ("queues", ctypes.c_int32), ("queue_capacity", ctypes.c_int32),
                ("kernel_ms", ctypes.c_double), ("idle_polls", ctypes.c_int64),
                ("reserved", ctypes.c_int64 * 4)]


class RoundsStats(ctypes.Structure):
    _fields_ = [("rounds", ctypes.c_int64), ("relaxed", ctypes.c_int64),
                ("updated", ctypes.c_int64), ("kernel_ms", ctypes.c_double),
                ("reserved", ctypes.c_int64 * 4)]


ROUNDS_ALL_EDGES = 1
NEG_CYCLE_STOP, NEG_CYCLE_MARK = 0, 1
RELAX_AUTO, RELAX_MIN, RELAX_CAS, RELAX_FILTERED = 0, 1, 2, 3
SMALL_PATH_AUTO, SMALL_PATH_ON, SMALL_PATH_OFF = 0, 1, 2
NEG_INF = -2147483648          # dist of a vertex reachable from a negative cycle (MARK)

_VP = ctypes.c_void_p
_I32 = ctypes.c_int32
_I64 = ctypes.c_int64
_SIGNATURES = {
    "bfq_last_error": ([], ctypes.c_char_p),
    "bfq_version": ([], _I32),
    "bfq_tune_default": ([ctypes.POINTER(Tune)], ctypes.c_int),
    "bfq_graph_create": ([ctypes.POINTER(_VP), _I32, _I64, _VP, _VP, _VP, ctypes.c_int,
                          ctypes.POINTER(Tune), _VP], ctypes.c_int),
    "bfq_graph_destroy": ([_VP], ctypes.c_int),
    "bfq_graph_device_bytes": ([_VP], _I64),
    "bfq_sssp": ([_VP, _I32, _VP, _VP, _VP, _VP], ctypes.c_int),
    "bfq_sssp_async": ([_VP, _I32, _VP, _VP, _VP, _VP, _VP], ctypes.c_int),
    "bfq_get_stats": ([_VP, ctypes.POINTER(Stats)], ctypes.c_int),
    "bfq_sssp_noalloc": ([_VP, _VP, _I32, _I64, _I32, _VP, _VP, _VP, _VP], ctypes.c_int),
    "bfq_sssp_rounds": ([_VP, _I32, _I32, _VP, _VP, _VP, ctypes.POINTER(RoundsStats), _VP],
                        ctypes.c_int),
    "bfq_graph_get_tune": ([_VP, ctypes.POINTER(Tune)], ctypes.c_int),
    "bfq_graph_set_tune": ([_VP, ctypes.POINTER(Tune)], ctypes.c_int),
    "bfq_autotune": ([_VP, _VP, _I32, ctypes.POINTER(Tune), _VP], ctypes.c_int),
    "bfq_batch_create": ([ctypes.POINTER(_VP), _VP, _I32, _I32, _I64, ctypes.POINTER(Tune)],
                         ctypes.c_int),
    "bfq_batch_destroy": ([_VP], ctypes.c_int),
    "bfq_batch_device_bytes": ([_VP], _I64),
    "bfq_sssp_batch": ([_VP, _I32, _VP, _VP, _VP, _VP, _VP, _VP], ctypes.c_int),
    "bfq_batch_get_stats": ([_VP, ctypes.POINTER(Stats)], ctypes.c_int),
    "bfq_batch_set_tune": ([_VP, ctypes.POINTER(Tune)], ctypes.c_int),
    "bfq_batch_autotune": ([_VP, _I32, _VP, _VP, _VP, _VP, ctypes.POINTER(Tune), _VP],
                           ctypes.c_int),
    "bfq_server_create": ([ctypes.POINTER(_VP), _VP, _I32, _I64, _I32, ctypes.POINTER(Tune)],
                          ctypes.c_int),
    "bfq_server_submit": ([_VP, _I32, _I32, _VP, _VP, ctypes.POINTER(_I64)], ctypes.c_int),
    "bfq_server_poll": ([_VP, _I64, ctypes.POINTER(_I32), ctypes.POINTER(_I64),
                         ctypes.POINTER(_I64)], ctypes.c_int),
    "bfq_server_wait": ([_VP, _I64, _I64, ctypes.POINTER(_I32)], ctypes.c_int),
    "bfq_server_stats": ([_VP, ctypes.POINTER(_I64), ctypes.POINTER(_I64),
                          ctypes.POINTER(_I64)], ctypes.c_int),
    "bfq_server_state": ([_VP, _VP, _I32], ctypes.c_int),
    "bfq_server_destroy": ([_VP], ctypes.c_int),
    "bfq_queue_create": ([ctypes.POINTER(_VP), _I64, _I32], ctypes.c_int),
    "bfq_queue_destroy": ([_VP], ctypes.c_int),
    "bfq_queue_reset": ([_VP, _VP], ctypes.c_int),
    "bfq_queue_enqueue": ([_VP, _VP, _I64, _VP, _I32, _I32, _VP], ctypes.c_int),
    "bfq_queue_dequeue": ([_VP, _VP, _I64, _VP, _I32, _I32, _VP], ctypes.c_int),
    "bfq_queue_mixed": ([_VP, _VP, _I64, _VP, _VP, _I64, _VP, _I32, _I32, _VP], ctypes.c_int),
    "bfq_queue_state": ([_VP, ctypes.POINTER(_I64), ctypes.POINTER(_I64),
                         ctypes.POINTER(_I64), _VP], ctypes.c_int),
    "bfq_atomic_bench": ([_I32, _I64, _I32, _I32, ctypes.POINTER(ctypes.c_double),
                          ctypes.POINTER(_I64), _VP], ctypes.c_int),
    "bfq_relax_bench": ([_I32, _I64, _I32, _I32, _I32, ctypes.POINTER(ctypes.c_double),
                         ctypes.POINTER(_I64), _VP], ctypes.c_int),
}

_lib = None
_lock = threading.Lock()


def lib() -> ctypes.CDLL:
    """Load libbfq.so, building it first if it is missing or stale."""
    global _lib
    with _lock:
        if _lib is None:
            path = os.environ.get("BFQ_LIBRARY") or _build.build()
            handle = ctypes.CDLL(path)
            for name, (args, res) in _SIGNATURES.items():
                f = getattr(handle, name)
                f.argtypes = args
                f.restype = res
            _lib = handle
    return _lib


def library_path() -> str:
    return _build.LIB


def last_error() -> str:
    return lib().bfq_last_error().decode()


def _check(rc: int) -> int:
    if rc < 0:
        raise BfqError(rc, last_error())
    return rc


def _ptr(x):
    """Raw address of a torch tensor, numpy array, int address or None."""
    if x is None:
        return None
    if hasattr(x, "data_ptr"):
        return _VP(x.data_ptr())
    if isinstance(x, np.ndarray):
        return _VP(x.ctypes.data)
    if isinstance(x, int):
        return _VP(x)
    raise TypeError(f"cannot take the address of {type(x)}")


def _stream(s):
    """cudaStream_t from a torch stream, an int handle, or the current torch
    stream when None."""
    if s is None:
        try:
            import torch
            if torch.cuda.is_available():
                return _VP(torch.cuda.current_stream().cuda_stream)
        except ImportError:
            pass
        return None
    if hasattr(s, "cuda_stream"):
        return _VP(s.cuda_stream)
    return _VP(int(s))


def _is_device(x) -> bool:
    return hasattr(x, "is_cuda") and bool(x.is_cuda)


def tune_default() -> Tune:
    t = Tune()
    _check(lib().bfq_tune_default(ctypes.byref(t)))
    return t


def make_tune(**kw) -> Tune:
    t = tune_default()
    for k, v in kw.items():
        setattr(t, k, v)
    return t


# ---- graphs -----------------------------------------------------------------

def bfq_graph_create(row_ptr, col, w, tune: Tune | None = None, stream=None):
    """CSR arrays as host numpy int32 arrays or CUDA int32 tensors."""
    on_dev = _is_device(row_ptr)
    if on_dev != _is_device(col) or on_dev != _is_device(w):
        raise ValueError("row_ptr, col and w must all be host or all be device arrays")
    if not on_dev:
        row_ptr = np.ascontiguousarray(row_ptr, dtype=np.int32)
        col = np.ascontiguousarray(col, dtype=np.int32)
        w = np.ascontiguousarray(w, dtype=np.int32)
    V = len(row_ptr) - 1
    E = len(col)
    h = _VP()
    _check(lib().bfq_graph_create(ctypes.byref(h), V, E, _ptr(row_ptr), _ptr(col), _ptr(w),
                                  int(on_dev), ctypes.byref(tune) if tune else None,
                                  _stream(stream)))
    return h


def bfq_graph_destroy(g) -> None:
    _check(lib().bfq_graph_destroy(g))


def bfq_graph_device_bytes(g) -> int:
    return int(lib().bfq_graph_device_bytes(g))


def bfq_sssp(g, src: int, dist, hops=None, pred=None, stream=None) -> int:
    """Synchronous single-source query; returns OK / NEG_CYCLE / RANGE."""
    return _check(lib().bfq_sssp(g, int(src), _ptr(dist), _ptr(hops), _ptr(pred),
                                 _stream(stream)))


def bfq_sssp_async(g, src: int, dist, hops=None, pred=None, status_dev=None, stream=None) -> int:
    return _check(lib().bfq_sssp_async(g, int(src), _ptr(dist), _ptr(hops), _ptr(pred),
                                       _ptr(status_dev), _stream(stream)))


def bfq_get_stats(g) -> dict:
    s = Stats()
    _check(lib().bfq_get_stats(g, ctypes.byref(s)))
    return {name: getattr(s, name) for name, _ in Stats._fields_ if name != "reserved"}


def bfq_sssp_rounds(g, src: int, dist, hops=None, pred=None, flags: int = 0,
                    stream=None) -> tuple[int, dict]:
    """Round-based query (change-counter rounds); returns (status, stats)."""
    st = RoundsStats()
    rc = _check(lib().bfq_sssp_rounds(g, int(src), int(flags), _ptr(dist), _ptr(hops),
                                      _ptr(pred), ctypes.byref(st), _stream(stream)))
    return rc, {name: getattr(st, name) for name, _ in RoundsStats._fields_ if name != "reserved"}


def bfq_graph_get_tune(g) -> Tune:
    t = Tune()
    _check(lib().bfq_graph_get_tune(g, ctypes.byref(t)))
    return t


def bfq_graph_set_tune(g, tune: Tune) -> None:
    _check(lib().bfq_graph_set_tune(g, ctypes.byref(tune)))


def bfq_sssp_noalloc(row_ptr, adj, V: int, E: int, src: int, dist, hops=None, status_dev=None,
                     stream=None) -> int:
    """Query without any allocation (fixed static scratch, V <= 524288); the
    status lands in status_dev (device int32).  Returns OK once enqueued."""
    return _check(lib().bfq_sssp_noalloc(_ptr(row_ptr), _ptr(adj), int(V), int(E), int(src),
                                         _ptr(dist), _ptr(hops), _ptr(status_dev),
                                         _stream(stream)))


def bfq_autotune(g, srcs, stream=None) -> Tune:
    """Pick the fastest run-time parameters for these sources; kept on g."""
    a = np.ascontiguousarray(srcs, dtype=np.int32)
    t = Tune()
    _check(lib().bfq_autotune(g, _ptr(a), len(a), ctypes.byref(t), _stream(stream)))
    return t


# ---- batched queries -------------------------------------------------------------

def _ptr_array(xs, n):
    arr = (_VP * max(1, n))()
    for i in range(n):
        x = xs[i] if xs is not None else None
        arr[i] = None if x is None else (x.data_ptr() if hasattr(x, "data_ptr") else int(x))
    return arr


def bfq_batch_create(graphs, max_queries: int, max_total_vertices: int = 0,
                     tune: Tune | None = None):
    hs = (_VP * len(graphs))(*[g.value if isinstance(g, _VP) else g for g in graphs])
    h = _VP()
    _check(lib().bfq_batch_create(ctypes.byref(h), hs, len(graphs), int(max_queries),
                                  int(max_total_vertices), ctypes.byref(tune) if tune else None))
    return h


def bfq_batch_destroy(b) -> None:
    _check(lib().bfq_batch_destroy(b))


def bfq_batch_device_bytes(b) -> int:
    return int(lib().bfq_batch_device_bytes(b))


def bfq_sssp_batch(b, graph_id, src, dist, hops=None, stream=None):
    """Run len(src) queries in one launch; dist/hops are lists of CUDA
    tensors.  Returns (rc, statuses)."""
    gid = np.ascontiguousarray(graph_id, dtype=np.int32)
    sr = np.ascontiguousarray(src, dtype=np.int32)
    n = len(sr)
    st = np.zeros(max(1, n), dtype=np.int32)
    rc = _check(lib().bfq_sssp_batch(b, n, _ptr(gid), _ptr(sr), _ptr_array(dist, n),
                                     _ptr_array(hops, n) if hops is not None else None,
                                     _ptr(st), _stream(stream)))
    return rc, st[:n]


def bfq_batch_get_stats(b) -> dict:
    s = Stats()
    _check(lib().bfq_batch_get_stats(b, ctypes.byref(s)))
    return {name: getattr(s, name) for name, _ in Stats._fields_ if name != "reserved"}


def bfq_batch_set_tune(b, tune: Tune) -> None:
    _check(lib().bfq_batch_set_tune(b, ctypes.byref(tune)))


def bfq_batch_autotune(b, graph_id, src, dist, hops=None, stream=None) -> Tune:
    gid = np.ascontiguousarray(graph_id, dtype=np.int32)
    sr = np.ascontiguousarray(src, dtype=np.int32)
    n = len(sr)
    t = Tune()
    _check(lib().bfq_batch_autotune(b, n, _ptr(gid), _ptr(sr), _ptr_array(dist, n),
                                    _ptr_array(hops, n) if hops is not None else None,
                                    ctypes.byref(t), _stream(stream)))
    return t


# ---- serving -----------------------------------------------------------------------

def bfq_server_create(graphs, hbm_budget_bytes: int, max_slots: int, tune: Tune | None = None):
    hs = (_VP * len(graphs))(*[g.value if isinstance(g, _VP) else g for g in graphs])
    h = _VP()
    _check(lib().bfq_server_create(ctypes.byref(h), hs, len(graphs), int(hbm_budget_bytes),
                                   int(max_slots), ctypes.byref(tune) if tune else None))
    return h


def bfq_server_submit(sv, graph_id: int, src: int, dist=None, hops=None) -> int:
    rid = _I64()
    _check(lib().bfq_server_submit(sv, int(graph_id), int(src), _ptr(dist), _ptr(hops),
                                   ctypes.byref(rid)))
    return rid.value


def bfq_server_poll(sv, req_id: int):
    """(rc, status, t_submit_ns, t_done_ns); rc is PENDING while not done."""
    st, t0, t1 = _I32(), _I64(), _I64()
    rc = _check(lib().bfq_server_poll(sv, int(req_id), ctypes.byref(st), ctypes.byref(t0),
                                      ctypes.byref(t1)))
    return rc, st.value, t0.value, t1.value


def bfq_server_wait(sv, req_id: int, timeout_ms: int = 60000) -> int:
    st = _I32()
    rc = _check(lib().bfq_server_wait(sv, int(req_id), int(timeout_ms), ctypes.byref(st)))
    if rc == PENDING:
        raise BfqError(ERR_TIMEOUT, f"request {req_id} still pending after {timeout_ms} ms")
    return st.value


def bfq_server_stats(sv):
    a, b, c = _I64(), _I64(), _I64()
    _check(lib().bfq_server_stats(sv, ctypes.byref(a), ctypes.byref(b), ctypes.byref(c)))
    return {"completed": a.value, "launches": b.value, "peak_active": c.value}


_STATE_KEYS = ("waiting", "admitted", "free_slots", "largest_free_labels", "launches",
               "completed", "kernel_running", "cuda_error", "bad_check", "bad_value")


def bfq_server_state(sv) -> dict:
    out = np.zeros(len(_STATE_KEYS), dtype=np.int64)
    _check(lib().bfq_server_state(sv, _ptr(out), len(out)))
    return dict(zip(_STATE_KEYS, (int(x) for x in out)))


def bfq_server_destroy(sv) -> None:
    _check(lib().bfq_server_destroy(sv))


# ---- standalone queue ----------------------------------------------------------

def bfq_queue_create(capacity: int, variant: int = QUEUE_BQ):
    h = _VP()
    _check(lib().bfq_queue_create(ctypes.byref(h), int(capacity), int(variant)))
    return h


def bfq_queue_destroy(q) -> None:
    _check(lib().bfq_queue_destroy(q))


def bfq_queue_reset(q, stream=None) -> None:
    _check(lib().bfq_queue_reset(q, _stream(stream)))


def bfq_queue_enqueue(q, items, pos_out=None, grid: int = 108, block: int = 256,
                      stream=None) -> None:
    _check(lib().bfq_queue_enqueue(q, _ptr(items), len(items), _ptr(pos_out), grid, block,
                                   _stream(stream)))


def bfq_queue_dequeue(q, out, pos_out=None, grid: int = 108, block: int = 256,
                      stream=None) -> None:
    _check(lib().bfq_queue_dequeue(q, _ptr(out), len(out), _ptr(pos_out), grid, block,
                                   _stream(stream)))


def bfq_queue_mixed(q, items, out, enq_pos=None, deq_pos=None, grid: int = 108,
                    block: int = 256, stream=None) -> None:
    _check(lib().bfq_queue_mixed(q, _ptr(items), len(items), _ptr(enq_pos), _ptr(out),
                                 len(out), _ptr(deq_pos), grid, block, _stream(stream)))


def bfq_queue_state(q, stream=None):
    """(status, head, tail, count); status ERR_TIMEOUT if a wait ran out."""
    h, t, c = _I64(), _I64(), _I64()
    rc = lib().bfq_queue_state(q, ctypes.byref(h), ctypes.byref(t), ctypes.byref(c),
                               _stream(stream))
    return rc, h.value, t.value, c.value


# ---- convenience object -----------------------------------------------------------

class Graph:
    """A resident graph: ``Graph(row_ptr, col, w).sssp(src)``."""

    def __init__(self, row_ptr, col, w, tune: Tune | None = None, stream=None):
        self.V = len(row_ptr) - 1
        self.E = len(col)
        self.handle = bfq_graph_create(row_ptr, col, w, tune, stream)

    def sssp(self, src: int, dist=None, hops=None, pred=None, stream=None):
        """Returns (status, dist, hops, pred) with CUDA int32 tensors."""
        import torch
        dev = torch.device("cuda", torch.cuda.current_device())
        if dist is None:
            dist = torch.empty(self.V, dtype=torch.int32, device=dev)
        st = bfq_sssp(self.handle, src, dist, hops, pred, stream)
        return st, dist, hops, pred

    def sssp_rounds(self, src: int, dist=None, hops=None, pred=None, flags: int = 0,
                    stream=None):
        """Round-based query; returns (status, dist, stats)."""
        import torch
        dev = torch.device("cuda", torch.cuda.current_device())
        if dist is None:
            dist = torch.empty(self.V, dtype=torch.int32, device=dev)
        st, stats = bfq_sssp_rounds(self.handle, src, dist, hops, pred, flags, stream)
        return st, dist, stats

    def stats(self) -> dict:
        return bfq_get_stats(self.handle)

    def device_bytes(self) -> int:
        return bfq_graph_device_bytes(self.handle)

    def close(self):
        if self.handle:
            bfq_graph_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def bfq_relax_bench(mode: int, n_edges: int, n_labels: int, grid: int, block: int,
                    stream=None):
    """Relaxation memory pattern alone (mode 0: atomicMin per edge, 1: load
    then atomicMin when lower); returns (ms, lowered)."""
    ms, low = ctypes.c_double(), _I64()
    _check(lib().bfq_relax_bench(int(mode), int(n_edges), int(n_labels), int(grid), int(block),
                                 ctypes.byref(ms), ctypes.byref(low), _stream(stream)))
    return ms.value, low.value


def bfq_atomic_bench(mode: int, n_ops: int, grid: int, block: int, stream=None):
    """L2 atomic throughput microbenchmark; returns (ms, total)."""
    ms, tot = ctypes.c_double(), _I64()
    _check(lib().bfq_atomic_bench(int(mode), int(n_ops), int(grid), int(block),
                                  ctypes.byref(ms), ctypes.byref(tot), _stream(stream)))
    return ms.value, tot.value
