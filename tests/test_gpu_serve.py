"""Serving (continuous batching on a resident kernel): every request's result
equals its solo run and the oracle, whatever else runs beside it; admission
by memory budget; requests that arrive while others run overlap with them."""
import time

import numpy as np
import pytest

import oracle
from paper_2608_21826_gb300 import bfq, synth
from tests import gpu_util, helpers

pytestmark = pytest.mark.gpu


def _setup(n_graphs=8, seed=21, vmax=20000):
    graphs, queries = synth.workload_batched(n_graphs=n_graphs, vmin=300, vmax=vmax, seed=seed)
    handles = [gpu_util.create(g) for g in graphs]
    return graphs, queries, handles


def _solo(handles, graphs, gi, s):
    return gpu_util.run(handles[gi], graphs[gi].V, int(s))


def test_results_match_solo_and_oracle():
    import torch
    graphs, queries, handles = _setup()
    sv = bfq.bfq_server_create(handles, 1 << 30, 64)
    try:
        bufs = []
        for gi, s in queries:
            d = torch.full((graphs[gi].V,), -3, dtype=torch.int32, device="cuda")
            bufs.append((gi, s, d, torch.full_like(d, -3)))
        torch.cuda.synchronize()        # buffers ready before the server writes them
        outs = [(bfq.bfq_server_submit(sv, int(gi), int(s), d, h), gi, s, d, h)
                for gi, s, d, h in bufs]
        for rid, gi, s, d, h in outs:
            st = bfq.bfq_server_wait(sv, rid, 60000)
            sst, sd, sh, _ = _solo(handles, graphs, gi, s)
            assert st == sst
            g = graphs[gi]
            ost, od, oh, _ = oracle.spfa(g.row_ptr, g.col, g.w, int(s))
            assert st == ost
            if st == bfq.OK:
                assert np.array_equal(d.cpu().numpy(), sd) and np.array_equal(d.cpu().numpy(), od)
                assert np.array_equal(h.cpu().numpy(), sh) and np.array_equal(h.cpu().numpy(), oh)
        stats = bfq.bfq_server_stats(sv)
        assert stats["completed"] == len(queries)
        assert stats["peak_active"] > 1
    finally:
        bfq.bfq_server_destroy(sv)
        for h in handles:
            bfq.bfq_graph_destroy(h)


def test_budget_admission_and_rejection():
    import torch
    g_small = synth.grid_graph(40, 40, seed=3)
    g_big = synth.workload_rmat(16)
    handles = [gpu_util.create(g_small), gpu_util.create(g_big)]
    # room for the big graph's labels once (plus page rounding), not twice
    budget = 32 * (((g_big.V + 4095) // 4096) * 4096 + 4096)
    sv = bfq.bfq_server_create(handles, budget, 8)
    try:
        outs = []
        for k in range(6):
            gi = k % 2
            g = [g_small, g_big][gi]
            s = int(g.sources[k % len(g.sources)])
            d = torch.empty(g.V, dtype=torch.int32, device="cuda")
            torch.cuda.synchronize()
            outs.append((bfq.bfq_server_submit(sv, gi, s, d), gi, s, d))
        for rid, gi, s, d in outs:
            assert bfq.bfq_server_wait(sv, rid, 60000) == bfq.OK
            sst, sd, _, _ = gpu_util.run(handles[gi], [g_small, g_big][gi].V, s)
            assert np.array_equal(d.cpu().numpy(), sd)
        g_huge = synth.workload_rmat(17)
        h3 = gpu_util.create(g_huge)
        sv2 = bfq.bfq_server_create([h3], budget, 4)
        with pytest.raises(bfq.BfqError) as e:
            bfq.bfq_server_submit(sv2, 0, int(g_huge.sources[0]))
        assert e.value.code == bfq.ERR_BUDGET
        bfq.bfq_server_destroy(sv2)
        bfq.bfq_graph_destroy(h3)
    finally:
        bfq.bfq_server_destroy(sv)
        for h in handles:
            bfq.bfq_graph_destroy(h)


def test_arrivals_during_running_queries_and_idle_gaps():
    """Requests trickle in (some while others run, some after the kernel went
    idle and left); all finish with exact results."""
    import torch
    graphs, queries, handles = _setup(n_graphs=6, seed=31, vmax=60000)
    sv = bfq.bfq_server_create(handles, 1 << 30, 16)
    try:
        outs = []
        rng = np.random.default_rng(0)
        for k, (gi, s) in enumerate(queries[:40]):
            d = torch.empty(graphs[gi].V, dtype=torch.int32, device="cuda")
            torch.cuda.synchronize()
            outs.append((bfq.bfq_server_submit(sv, int(gi), int(s), d), gi, s, d))
            time.sleep(float(rng.exponential(0.0005)) if k != 20 else 0.05)
        for rid, gi, s, d in outs:
            st = bfq.bfq_server_wait(sv, rid, 60000)
            sst, sd, _, _ = _solo(handles, graphs, gi, s)
            assert st == sst
            if st == bfq.OK:
                assert np.array_equal(d.cpu().numpy(), sd)
        assert bfq.bfq_server_stats(sv)["launches"] >= 1
    finally:
        bfq.bfq_server_destroy(sv)
        for h in handles:
            bfq.bfq_graph_destroy(h)


def test_large_requests_run_alone_between_small_ones():
    """Requests over half of the label budget (here 32K labels, so graphs of
    16K+ vertices) run alone through the single-query kernel while the
    resident kernel is stopped and later resumed; small requests submitted
    around them still complete, and every result equals the solo run."""
    import torch
    graphs, queries, handles = _setup(n_graphs=6, seed=33, vmax=5000)
    big = [synth.grid_graph(160, 160, seed=9), synth.workload_rmat(15)]
    bh = [gpu_util.create(g) for g in big]
    all_g = list(graphs) + big
    all_h = list(handles) + bh
    sv = bfq.bfq_server_create(all_h, 1 << 30, 64, bfq.make_tune(batch_budget_klabels=32))
    try:
        reqs = []
        k = 0
        for gi, s in queries:
            reqs.append((int(gi), int(s)))
            if k % 5 == 0:                                 # a large one every few
                bi = len(graphs) + (k // 5) % 2
                reqs.append((bi, int(all_g[bi].sources[k % len(all_g[bi].sources)])))
            k += 1
        bufs = [torch.full((all_g[gi].V,), -3, dtype=torch.int32, device="cuda")
                for gi, _ in reqs]
        torch.cuda.synchronize()
        ids = [bfq.bfq_server_submit(sv, gi, s, bufs[i]) for i, (gi, s) in enumerate(reqs)]
        sts = [bfq.bfq_server_wait(sv, rid, 60000) for rid in ids]
        assert bfq.bfq_server_stats(sv)["completed"] == len(reqs)
    finally:
        bfq.bfq_server_destroy(sv)
    try:
        for (gi, s), st, d in zip(reqs, sts, bufs):
            sst, sd, _, _ = gpu_util.run(all_h[gi], all_g[gi].V, s)
            assert st == sst, (gi, s)
            if st == bfq.OK:
                assert np.array_equal(d.cpu().numpy(), sd), (gi, s)
        for bi in (len(graphs), len(graphs) + 1):
            g = all_g[bi]
            s = int(g.sources[0])
            ost, od, _, _ = oracle.spfa(g.row_ptr, g.col, g.w, s)
            sst, sd, _, _ = gpu_util.run(all_h[bi], g.V, s)
            assert sst == ost and np.array_equal(sd, od)
    finally:
        for h in all_h:
            bfq.bfq_graph_destroy(h)


def test_full_serving_mix_matches_oracle():
    """The serving workload at full size: the 64-graph batched mix plus an
    R-MAT scale-23 graph (8.4M vertices, 131M edges) resident in one server.
    240 requests over the mix and 4 on R-MAT 23 arrive in Poisson-like
    trickles, so many are admitted while others run and the large ones run
    alone between batches.  Every result (status, dist, hops) equals the
    oracle's, element by element."""
    import torch
    graphs, _ = helpers.batched_workload()
    g23 = synth.workload_rmat(23)
    all_g = list(graphs) + [g23]
    rng = np.random.default_rng(2024)
    reqs = []
    for k in range(240):
        gi = int(rng.integers(0, len(graphs)))
        reqs.append((gi, int(rng.choice(graphs[gi].sources))))
        if k % 60 == 30:
            reqs.append((len(graphs), int(g23.sources[(k // 60) % len(g23.sources)])))
    expect = helpers.oracle_many([(all_g[gi], s) for gi, s in reqs])
    handles = [gpu_util.create(g) for g in all_g]
    sv = bfq.bfq_server_create(handles, 32 * 400_000_000, 512)
    try:
        bufs = [(torch.full((all_g[gi].V,), -3, dtype=torch.int32, device="cuda"),
                 torch.full((all_g[gi].V,), -3, dtype=torch.int32, device="cuda"))
                for gi, _ in reqs]
        torch.cuda.synchronize()
        ids = []
        for k, (gi, s) in enumerate(reqs):
            ids.append(bfq.bfq_server_submit(sv, gi, s, bufs[k][0], bufs[k][1]))
            if k % 16 == 15:
                time.sleep(float(rng.exponential(0.002)))
        sts = [bfq.bfq_server_wait(sv, rid, 120000) for rid in ids]
        assert bfq.bfq_server_stats(sv)["completed"] == len(reqs)
        assert bfq.bfq_server_stats(sv)["peak_active"] > 1
        n_cyc = 0
        for k, ((gi, s), st) in enumerate(zip(reqs, sts)):
            ost, od, oh = expect[k]
            assert st == ost, (k, gi, s, st, ost)
            n_cyc += st == bfq.NEG_CYCLE
            if st == bfq.OK:
                assert np.array_equal(bufs[k][0].cpu().numpy(), od), (k, gi, s)
                assert np.array_equal(bufs[k][1].cpu().numpy(), oh), (k, gi, s)
        assert n_cyc > 0
    finally:
        bfq.bfq_server_destroy(sv)
        for h in handles:
            bfq.bfq_graph_destroy(h)
