"""The allocation-free query entry point (bfq_sssp_noalloc), for callers that
cannot allocate device memory when they issue a query (inside stream capture,
fixed start-up budgets, foreign memory arenas).  Call after call it must give
exactly what the oracle gives and what the regular entry point (bfq_sssp on a
graph handle) gives, although every call reuses the same static scratch
array.

This file is collected last on purpose."""
import numpy as np
import pytest

import oracle
from paper_2608_21826_gb300 import bfq, synth
from tests import gpu_util

pytestmark = pytest.mark.gpu


def _noalloc(g, src, want_hops=True, stream=None, adj_override=None):
    import torch
    rp = torch.from_numpy(np.ascontiguousarray(g.row_ptr)).cuda()
    adj_np = np.stack([g.col, g.w], axis=1).reshape(-1).astype(np.int32)
    if adj_override is not None:
        adj_np = adj_override
    adj = torch.from_numpy(np.ascontiguousarray(adj_np)).cuda()
    dist = torch.full((g.V,), -5, dtype=torch.int32, device="cuda")
    hops = torch.full((g.V,), -5, dtype=torch.int32, device="cuda") if want_hops else None
    status = torch.full((1,), -99, dtype=torch.int32, device="cuda")
    torch.cuda.synchronize()
    assert bfq.bfq_sssp_noalloc(rp, adj, g.V, g.E, src, dist, hops, status,
                                stream=stream) == bfq.OK
    torch.cuda.synchronize()
    return (int(status.item()), dist.cpu().numpy(),
            hops.cpu().numpy() if hops is not None else None)


def test_matches_oracle_and_regular_entry_point_on_consecutive_calls():
    # different graphs back to back: a call must not see the previous call's
    # leftovers in the shared scratch array
    cases = [(synth.workload_rmat(14), None), (synth.grid_graph(100, 120, seed=9), 0),
             (synth.workload_rmat(14), None), (synth.workload_grid4k(), 0)]
    for g, src in cases:
        s = int(g.sources[0]) if src is None else src
        ost, od, oh, _ = oracle.spfa(g.row_ptr, g.col, g.w, s)
        st_ref, d_ref, h_ref, _ = gpu_util.sssp(g, s)
        st, d, h = _noalloc(g, s)
        assert st == st_ref == ost == bfq.OK
        assert np.array_equal(d, od) and np.array_equal(h, oh)
        assert np.array_equal(d, d_ref) and np.array_equal(h, h_ref)


def test_negative_cycle_status_then_clean():
    g = synth.plant_negative_cycle(synth.grid_graph(40, 40, seed=2), 5, seed=1)
    st, _, _ = _noalloc(g, 0)
    assert st == bfq.NEG_CYCLE == oracle.spfa(g.row_ptr, g.col, g.w, 0)[0]
    g2 = synth.grid_graph(40, 40, seed=3)
    st, d, h = _noalloc(g2, 0)
    ost, od, oh, _ = oracle.spfa(g2.row_ptr, g2.col, g2.w, 0)
    assert st == ost == bfq.OK and np.array_equal(d, od) and np.array_equal(h, oh)


def test_without_hops_on_a_side_stream():
    import torch
    g = synth.workload_rmat(13)
    s = int(g.sources[0])
    side = torch.cuda.Stream()
    st, d, h = _noalloc(g, s, want_hops=False, stream=side)
    ost, od, _, _ = oracle.spfa(g.row_ptr, g.col, g.w, s)
    assert h is None and st == ost == bfq.OK and np.array_equal(d, od)


def test_bad_column_reported_in_status():
    """A column out of range passes the host checks (the CSR lives on the
    device); the device-side check reports it in status_dev, and the next
    call is clean."""
    g = synth.grid_graph(20, 20, seed=4)
    adj = np.stack([g.col, g.w], axis=1).reshape(-1).astype(np.int32)
    adj[2 * 7] = g.V + 3
    st, _, _ = _noalloc(g, 0, adj_override=adj)
    assert st == bfq.ERR_INVALID
    st, d, h = _noalloc(g, 0)
    ost, od, oh, _ = oracle.spfa(g.row_ptr, g.col, g.w, 0)
    assert st == ost == bfq.OK and np.array_equal(d, od) and np.array_equal(h, oh)


def test_rejects_graphs_beyond_the_limit():
    import torch
    V = (1 << 19) + 1
    rp = torch.zeros(V + 1, dtype=torch.int32, device="cuda")
    adj = torch.zeros(2, dtype=torch.int32, device="cuda")
    dist = torch.empty(V, dtype=torch.int32, device="cuda")
    status = torch.zeros(1, dtype=torch.int32, device="cuda")
    with pytest.raises(bfq.BfqError) as e:
        bfq.bfq_sssp_noalloc(rp, adj, V, 0, 0, dist, None, status)
    assert e.value.code == bfq.ERR_INVALID and "524288" in str(e.value)
