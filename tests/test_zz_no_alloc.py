"""The allocation-free query entry point (bfq_sssp_noalloc), for callers that
cannot allocate device memory when they issue a query (inside stream capture,
fixed start-up budgets, foreign memory arenas).  It must give exactly what
the regular entry point (bfq_sssp on a graph handle) gives, call after call,
although every call reuses the same static scratch array.

This file is collected last on purpose."""
import numpy as np
import pytest

from paper_2608_21826_gb300 import bfq, synth
from tests import gpu_util

pytestmark = pytest.mark.gpu


def _noalloc(g, src):
    import torch
    rp = torch.from_numpy(np.ascontiguousarray(g.row_ptr)).cuda()
    adj = torch.from_numpy(np.ascontiguousarray(
        np.stack([g.col, g.w], axis=1).reshape(-1).astype(np.int32))).cuda()
    dist = torch.full((g.V,), -5, dtype=torch.int32, device="cuda")
    hops = torch.full((g.V,), -5, dtype=torch.int32, device="cuda")
    status = torch.full((1,), -99, dtype=torch.int32, device="cuda")
    assert bfq.bfq_sssp_noalloc(rp, adj, g.V, g.E, src, dist, hops, status) == bfq.OK
    torch.cuda.synchronize()
    return int(status.item()), dist.cpu().numpy(), hops.cpu().numpy()


def test_matches_regular_entry_point_on_consecutive_calls():
    # two different graphs back to back: the second call must not see the
    # first call's leftovers in the shared scratch array
    cases = [(synth.workload_rmat(14), None), (synth.grid_graph(100, 120, seed=9), 0),
             (synth.workload_rmat(14), None)]
    for g, src in cases:
        s = int(g.sources[0]) if src is None else src
        st_ref, d_ref, h_ref, _ = gpu_util.sssp(g, s)
        st, d, h = _noalloc(g, s)
        assert st == st_ref == bfq.OK
        assert np.array_equal(d, d_ref) and np.array_equal(h, h_ref)


def test_negative_cycle_status_then_clean():
    g = synth.plant_negative_cycle(synth.grid_graph(40, 40, seed=2), 5, seed=1)
    st, _, _ = _noalloc(g, 0)
    assert st == bfq.NEG_CYCLE == gpu_util.sssp(g, 0)[0]
    g2 = synth.grid_graph(40, 40, seed=3)
    st, d, h = _noalloc(g2, 0)
    st_ref, d_ref, h_ref, _ = gpu_util.sssp(g2, 0)
    assert st == st_ref == bfq.OK and np.array_equal(d, d_ref) and np.array_equal(h, h_ref)


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
