"""Batched queries (many sources over many graphs in one launch): every
query's dist/hops/status equals the oracle's and its own solo run's; planted
negative cycles stop only their own queries; launch-level errors and the
autotuner."""
import numpy as np
import pytest

import oracle
from paper_2608_21826_gb300 import bfq, synth
from tests import gpu_util, helpers

pytestmark = pytest.mark.gpu


class Mix:
    def __init__(self, n_graphs=10, vmin=200, vmax=6000, seed=5, max_queries=None, tune=None):
        import torch
        self.graphs, self.queries = synth.workload_batched(n_graphs=n_graphs, vmin=vmin,
                                                           vmax=vmax, seed=seed)
        self.handles = [gpu_util.create(g) for g in self.graphs]
        nq = len(self.queries)
        self.b = bfq.bfq_batch_create(self.handles, max_queries or nq,
                                      sum(self.graphs[g].V for g, _ in self.queries), tune)
        self.dist = [torch.full((self.graphs[g].V,), -5, dtype=torch.int32, device="cuda")
                     for g, _ in self.queries]
        self.hops = [torch.full_like(d, -5) for d in self.dist]

    def run(self, sel=None):
        sel = np.arange(len(self.queries)) if sel is None else np.asarray(sel, dtype=np.int64)
        q = self.queries[sel]
        rc, st = bfq.bfq_sssp_batch(self.b, q[:, 0], q[:, 1], [self.dist[i] for i in sel],
                                    [self.hops[i] for i in sel])
        return rc, st, sel

    def close(self):
        bfq.bfq_batch_destroy(self.b)
        for h in self.handles:
            bfq.bfq_graph_destroy(h)


def _check_query(mix, i, st):
    gi, s = mix.queries[i]
    g = mix.graphs[gi]
    ost, od, oh, _ = oracle.spfa(g.row_ptr, g.col, g.w, int(s))
    assert st == ost, (i, st, ost)
    if ost == oracle.OK:
        assert np.array_equal(mix.dist[i].cpu().numpy(), od), f"query {i}: dist"
        assert np.array_equal(mix.hops[i].cpu().numpy(), oh), f"query {i}: hops"


def test_small_mix_matches_oracle_and_solo():
    mix = Mix()
    try:
        rc, st, sel = mix.run()
        assert rc == bfq.OK
        n_cyc = 0
        for i in sel:
            _check_query(mix, i, st[i])
            n_cyc += st[i] == bfq.NEG_CYCLE
        assert n_cyc == sum(len(g.sources) for g in mix.graphs if g.cycle is not None) > 0
        # isolation: each query alone gives the same result as in the mix
        for i in sel[::7]:
            gi, s = mix.queries[i]
            sst, sd, sh, _ = gpu_util.run(mix.handles[gi], mix.graphs[gi].V, int(s))
            assert sst == st[i]
            if sst == bfq.OK:
                assert np.array_equal(sd, mix.dist[i].cpu().numpy())
                assert np.array_equal(sh, mix.hops[i].cpu().numpy())
    finally:
        mix.close()


def test_varying_query_sets_on_one_handle():
    mix = Mix(n_graphs=6, seed=8)
    try:
        rng = np.random.default_rng(0)
        n = len(mix.queries)
        for sel in (np.arange(n), [0], rng.choice(n, size=n // 2, replace=False),
                    np.arange(n)[::-1], []):
            rc, st, sel = mix.run(sel)
            assert rc == bfq.OK
            for k, i in enumerate(sel):
                _check_query(mix, i, st[k])
    finally:
        mix.close()


def test_rejects_oversized_batches():
    mix = Mix(n_graphs=4, seed=9, max_queries=8)
    try:
        with pytest.raises(bfq.BfqError) as e:
            mix.run(np.arange(min(9, len(mix.queries))) if len(mix.queries) >= 9 else None)
        assert e.value.code == bfq.ERR_INVALID
        rc, st, sel = mix.run(np.arange(4))
        assert rc == bfq.OK
    finally:
        mix.close()


def test_timeout_then_clean_batch():
    import torch
    g = synth.workload_rmat(12)
    h = gpu_util.create(g)
    try:
        t = bfq.make_tune(time_limit_ms=30, test_phantom_items=1)
        b = bfq.bfq_batch_create([h], 4, 4 * g.V, t)
        d = [torch.empty(g.V, dtype=torch.int32, device="cuda") for _ in range(4)]
        with pytest.raises(bfq.BfqError) as e:
            bfq.bfq_sssp_batch(b, [0] * 4, g.sources, d)
        assert e.value.code == bfq.ERR_TIMEOUT
        bfq.bfq_batch_destroy(b)
        b = bfq.bfq_batch_create([h], 4, 4 * g.V)
        rc, st = bfq.bfq_sssp_batch(b, [0] * 4, g.sources, d)
        assert rc == bfq.OK
        for k, s in enumerate(g.sources):
            ost, od, _, _ = oracle.spfa(g.row_ptr, g.col, g.w, int(s))
            assert st[k] == ost and np.array_equal(d[k].cpu().numpy(), od)
        bfq.bfq_batch_destroy(b)
    finally:
        bfq.bfq_graph_destroy(h)


def test_autotune_keeps_results_exact():
    mix = Mix(n_graphs=6, seed=12)
    try:
        q = mix.queries
        t = bfq.bfq_batch_autotune(mix.b, q[:, 0], q[:, 1], mix.dist, mix.hops)
        assert t.share_div in (1, 2, 4, 8) and t.chunk_batch in (2, 4, 8)
        rc, st, sel = mix.run()
        for i in sel:
            _check_query(mix, i, st[i])
    finally:
        mix.close()


def test_single_graph_autotune():
    g = synth.workload_rmat(14)
    h = gpu_util.create(g)
    try:
        t = bfq.bfq_autotune(h, g.sources)
        assert t.share_div in (1, 2, 4, 8) and t.kernel_ctas in (0, 3, 4)
        for s in g.sources:
            st, d, hh, _ = gpu_util.run(h, g.V, int(s))
            ost, od, oh, _ = oracle.spfa(g.row_ptr, g.col, g.w, int(s))
            assert st == ost and np.array_equal(d, od) and np.array_equal(hh, oh)
    finally:
        bfq.bfq_graph_destroy(h)


def test_full_batched_workload():
    """64 graphs (V log-uniform in [1e3, 1e6]), 512 queries, 6 graphs with a
    planted negative cycle: every query's status, dist and hops equal the
    oracle's (FIFO Bellman-Ford with the parent-graph cycle search, exact
    and fast on the cycle graphs), element by element; the oracle's cycle
    statuses also fall exactly on the planted graphs' queries; and each
    result equals the query's solo run."""
    import torch
    graphs, queries = helpers.batched_workload()
    expect = helpers.oracle_many([(graphs[gi], s) for gi, s in queries])
    handles = [gpu_util.create(g) for g in graphs]
    total = int(sum(graphs[g].V for g, _ in queries))
    b = bfq.bfq_batch_create(handles, len(queries), total)
    try:
        dist = [torch.full((graphs[g].V,), -5, dtype=torch.int32, device="cuda")
                for g, _ in queries]
        hops = [torch.full_like(d, -5) for d in dist]
        rc, st = bfq.bfq_sssp_batch(b, queries[:, 0], queries[:, 1], dist, hops)
        assert rc == bfq.OK
        ost = np.array([e[0] for e in expect])
        assert np.array_equal(st, ost), np.nonzero(st != ost)[0][:10]
        cyc = np.array([graphs[g].cycle is not None for g, _ in queries])
        assert np.array_equal(ost == oracle.NEG_CYCLE, cyc)
        assert sum(g.cycle is not None for g in graphs) == 6
        for i, (gi, s) in enumerate(queries):
            if ost[i] != oracle.OK:
                continue
            assert np.array_equal(dist[i].cpu().numpy(), expect[i][1]), f"query {i}: dist"
            assert np.array_equal(hops[i].cpu().numpy(), expect[i][2]), f"query {i}: hops"
        # isolation: the same query alone gives the same result
        for i in range(0, len(queries), 9):
            gi, s = queries[i]
            sst, sd, sh, _ = gpu_util.run(handles[gi], graphs[gi].V, int(s))
            assert sst == st[i]
            if sst == bfq.OK:
                assert np.array_equal(sd, expect[i][1]) and np.array_equal(sh, expect[i][2])
    finally:
        bfq.bfq_batch_destroy(b)
        for h in handles:
            bfq.bfq_graph_destroy(h)


@pytest.mark.parametrize("budget", [-1, 4, 16, 0])
def test_label_budget_staggers_starts_exactly(budget):
    """Queries start in order while the running ones' labels fit the budget
    (4 = 4096 labels: one or two graphs' queries at a time; 0 = half of L2;
    -1 = all at once); the results do not depend on it, including the
    planted-cycle queries.  Graphs stay small so the oracle ends quickly
    on the cycle graph."""
    mix = Mix(n_graphs=12, vmin=500, vmax=6000, seed=8,
              tune=bfq.make_tune(batch_budget_klabels=budget))
    try:
        rc, st, sel = mix.run()
        assert rc == bfq.OK
        for i in sel:
            _check_query(mix, i, st[i])
        # a second run on the same handle, in reverse order
        rc, st2, sel2 = mix.run(sel[::-1])
        for k, i in enumerate(sel2):
            assert st2[k] == st[i]
    finally:
        mix.close()


def test_label_budget_is_validated():
    g = synth.grid_graph(8, 8, seed=1)
    h = gpu_util.create(g)
    try:
        with pytest.raises(bfq.BfqError):
            bfq.bfq_batch_create([h], 4, 4 * g.V, bfq.make_tune(batch_budget_klabels=-2))
    finally:
        bfq.bfq_graph_destroy(h)
