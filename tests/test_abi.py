"""The C-ABI library builds, loads and exports every function include/*.h
declares; host-side argument checks work without a GPU."""
import ctypes
import glob
import os
import re
import subprocess

import pytest

from paper_2608_21826_gb300 import _build, bfq

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", " ", text, flags=re.S)
        text = re.sub(r"//[^\n]*", " ", text)
        for m in re.finditer(r"\b(bfq_\w+)\s*\(", text):
            names.add(m.group(1))
    return sorted(names)


def test_header_declares_entry_points():
    names = declared_functions()
    for n in ("bfq_graph_create", "bfq_sssp", "bfq_sssp_async", "bfq_queue_enqueue",
              "bfq_queue_dequeue", "bfq_queue_mixed", "bfq_last_error"):
        assert n in names


def test_library_exports_every_declared_symbol():
    path = _build.build()
    lib = ctypes.CDLL(path)
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing
    out = subprocess.run(["nm", "-D", "--defined-only", path], capture_output=True,
                         text=True).stdout
    exported = {ln.split()[-1] for ln in out.splitlines() if ln.strip()}
    assert set(declared_functions()) <= exported


def test_binding_covers_every_declared_symbol():
    for n in declared_functions():
        assert n in bfq._SIGNATURES, f"binding lacks {n}"


def test_host_side_checks_without_gpu():
    assert bfq.lib().bfq_version() >= 10000
    t = bfq.tune_default()
    assert t.threads_per_cta == 256 and t.batch_items == 32 and t.spin_limit > 0
    h = ctypes.c_void_p()
    rc = bfq.lib().bfq_queue_create(ctypes.byref(h), 0, bfq.QUEUE_BQ)
    assert rc == bfq.ERR_INVALID and "capacity" in bfq.last_error()
    rc = bfq.lib().bfq_queue_create(ctypes.byref(h), 16, 7)
    assert rc == bfq.ERR_INVALID
    rc = bfq.lib().bfq_graph_create(ctypes.byref(h), 0, 0, None, None, None, 0, None, None)
    assert rc == bfq.ERR_INVALID and "V" in bfq.last_error()
    bad = bfq.make_tune(batch_items=33)
    import numpy as np
    rp = np.array([0, 0], np.int32)
    rc = bfq.lib().bfq_graph_create(ctypes.byref(h), 1, 0, rp.ctypes.data, None, None, 0,
                                    ctypes.byref(bad), None)
    assert rc == bfq.ERR_INVALID and "batch_items" in bfq.last_error()
    with pytest.raises(bfq.BfqError):
        bfq.bfq_sssp(None, 0, None)


def test_tune_struct_layout_matches_the_header():
    """bfq_tune_default clears exactly sizeof(bfq_tune) bytes: a sentinel
    after the Python struct stays intact, and the fields land where the
    binding expects them (defaults of the last fields)."""
    n = ctypes.sizeof(bfq.Tune)
    buf = (ctypes.c_ubyte * (n + 64))(*([0xAB] * (n + 64)))
    assert bfq.lib().bfq_tune_default(ctypes.cast(buf, ctypes.POINTER(bfq.Tune))) == bfq.OK
    assert all(b == 0xAB for b in bytes(buf)[n:])
    t = bfq.Tune.from_buffer_copy(bytes(buf)[:n])
    assert t.cycle_walk_hops == 64 and t.relax_atomic == bfq.RELAX_AUTO
    assert t.neg_cycle_mode == bfq.NEG_CYCLE_STOP and t.batch_budget_klabels == 0
    assert t.share_div == 2 and t.chunk_batch == 4 and t.l2_persist_pct == 0
    assert t.kernel_ctas == 0


@pytest.mark.parametrize("field,value", [("relax_atomic", 4), ("relax_atomic", -1), ("neg_cycle_mode", 2), ("small_path", 3), ("small_threads", 256),
                                         ("cycle_walk_hops", 1), ("l2_persist_pct", 101),
                                         ("kernel_ctas", 2), ("kernel_ctas", 5)])
def test_bad_tunes_rejected_before_any_device_work(field, value):
    import numpy as np
    h = ctypes.c_void_p()
    rp = np.array([0, 0], np.int32)
    bad = bfq.make_tune(**{field: value})
    rc = bfq.lib().bfq_graph_create(ctypes.byref(h), 1, 0, rp.ctypes.data, None, None, 0,
                                    ctypes.byref(bad), None)
    assert rc == bfq.ERR_INVALID
