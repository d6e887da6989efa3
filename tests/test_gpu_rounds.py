"""Parity of the round-based path (bfq_sssp_rounds: change-counter rounds of
Algorithm 3) with the oracle, in both edge-selection modes, plus the round
count bound that the change counter implies."""
import numpy as np
import pytest

import oracle
from paper_2608_21826_gb300 import bfq, synth
from tests import gpu_util, helpers

pytestmark = pytest.mark.gpu
INF = helpers.INF
MODES = [0, bfq.ROUNDS_ALL_EDGES]
MODE_IDS = ["changed-tails", "all-edges"]


def _run(h, V, src, flags, want_pred=False):
    import torch
    dist = torch.full((V,), -7, dtype=torch.int32, device="cuda")
    hops = torch.full((V,), -7, dtype=torch.int32, device="cuda")
    pred = torch.full((V,), -7, dtype=torch.int32, device="cuda") if want_pred else None
    st, stats = bfq.bfq_sssp_rounds(h, src, dist, hops, pred, flags)
    return (st, dist.cpu().numpy(), hops.cpu().numpy(),
            pred.cpu().numpy() if pred is not None else None, stats)


def _compare(g, src, res, check_pred=False):
    st, d, h, p, stats = res
    ost, od, oh, _ = oracle.spfa(g.row_ptr, g.col, g.w, src)
    assert st == ost, (st, ost)
    assert 1 <= stats["rounds"] <= g.V
    if ost == oracle.OK:
        bad = np.nonzero(d != od)[0]
        assert bad.size == 0, f"{bad.size} dist mismatches, first {bad[:5]}: {d[bad[:5]]} vs {od[bad[:5]]}"
        assert np.array_equal(h, oh), "hops mismatch"
        # after round k every label is at most the best walk of k + 1 edges,
        # so the last change happens by round max(hops) and the next round
        # finds none
        assert stats["rounds"] <= int(oh[oh >= 0].max()) + 1
        reached = int(np.sum(od != INF))
        assert stats["updated"] >= reached - 1
        if check_pred:
            assert oracle.check_pred(g.row_ptr, g.col, g.w, src, d, p)
    return ost


def _one(g, src, flags, want_pred=False, tune=None):
    h = gpu_util.create(g, tune)
    try:
        return _run(h, g.V, src, flags, want_pred)
    finally:
        bfq.bfq_graph_destroy(h)


@pytest.mark.parametrize("flags", MODES, ids=MODE_IDS)
@pytest.mark.parametrize("path", helpers.golden_files(), ids=lambda p: p.split("/")[-1])
def test_golden(path, flags):
    g, exp = helpers.load_golden(path)
    st, d, h, p, _ = _one(g, 0, flags, want_pred=True)
    assert st == exp["status"]
    if "dist" in exp:
        assert d.tolist() == exp["dist"] and h.tolist() == exp["hops"]
        assert oracle.check_pred(g.row_ptr, g.col, g.w, 0, d, p)


@pytest.mark.parametrize("flags", MODES, ids=MODE_IDS)
@pytest.mark.parametrize("seed", range(20))
def test_random_with_cycles(seed, flags):
    rng = np.random.default_rng(seed)
    V = int(rng.integers(1, 3000))
    E = int(rng.integers(0, 6 * V + 1))
    g = synth.random_graph(V, E, seed=500 + seed, wlo=-3, whi=40)
    _compare(g, 0, _one(g, 0, flags))


@pytest.mark.parametrize("flags", MODES, ids=MODE_IDS)
@pytest.mark.parametrize("seed", range(6))
def test_random_potential(seed, flags):
    rng = np.random.default_rng(100 + seed)
    V = int(rng.integers(2000, 40000))
    g = synth.random_potential_graph(V, 6 * V, seed=seed)
    assert _compare(g, 0, _one(g, 0, flags, want_pred=True), check_pred=True) == oracle.OK


@pytest.mark.parametrize("flags", MODES, ids=MODE_IDS)
def test_grid_and_road(flags):
    for g in (synth.workload_grid4k(), synth.road_graph(256, seed=7)):
        h = gpu_util.create(g)
        try:
            for s in g.sources[:3]:
                _compare(g, int(s), _run(h, g.V, int(s), flags, want_pred=True), check_pred=True)
        finally:
            bfq.bfq_graph_destroy(h)


@pytest.mark.parametrize("scale", [12, 16])
def test_rmat_twins(scale):
    g = synth.workload_rmat(scale)
    h = gpu_util.create(g)
    try:
        for s in g.sources[:4]:
            for flags in MODES:
                _compare(g, int(s), _run(h, g.V, int(s), flags, want_pred=True), check_pred=True)
    finally:
        bfq.bfq_graph_destroy(h)


def test_rmat22_full_against_dijkstra():
    g = synth.workload_rmat(22)
    h = gpu_util.create(g)
    try:
        for s in g.sources[:2]:
            st, d, hh, _, stats = _run(h, g.V, int(s), 0)
            db, hb = oracle.dijkstra(g.row_ptr, g.col, g.base_w, int(s))
            ed, eh = helpers.shifted_expectation(db, hb, g.potential, int(s))
            assert st == bfq.OK
            assert np.array_equal(d, ed) and np.array_equal(hh, eh)
            assert stats["rounds"] <= int(eh[eh >= 0].max()) + 1
    finally:
        bfq.bfq_graph_destroy(h)


def test_long_path_takes_v_rounds():
    """A path needs one round per edge plus the round that finds no change:
    exactly V rounds, the most a run without a negative cycle can take."""
    V = 3000
    w = np.random.default_rng(2).integers(-5, 9, size=V - 1).astype(np.int32)
    g = synth.path_graph(V, w)
    st, d, h, _, stats = _one(g, 0, 0)
    assert st == bfq.OK and stats["rounds"] == V
    assert np.array_equal(d, np.r_[0, np.cumsum(w)]) and np.array_equal(h, np.arange(V))


def test_star():
    V = 200_000
    w = np.random.default_rng(1).integers(-1000, 1000, size=V - 1).astype(np.int32)
    g = synth.star_graph(V, w)
    for flags in MODES:
        st, d, h, p, stats = _one(g, 0, flags, want_pred=True)
        assert st == bfq.OK and d[0] == 0 and np.array_equal(d[1:], w)
        assert np.all(h[1:] == 1) and np.all(p[1:] == 0)
        assert stats["rounds"] == 2 and stats["updated"] == V - 1


def test_single_vertex_and_no_edges():
    g = synth.Graph("one", np.array([0, 0], np.int32), np.zeros(0, np.int32),
                    np.zeros(0, np.int32), np.array([0], np.int32))
    st, d, h, p, stats = _one(g, 0, 0, want_pred=True)
    assert st == bfq.OK and d.tolist() == [0] and h.tolist() == [0] and p.tolist() == [-1]
    assert stats["rounds"] == 1 and stats["relaxed"] == 0
    rp = np.zeros(1001, np.int32)
    g = synth.Graph("empty", rp, np.zeros(0, np.int32), np.zeros(0, np.int32),
                    np.array([0], np.int32))
    st, d, h, _, _ = _one(g, 500, bfq.ROUNDS_ALL_EDGES)
    assert st == bfq.OK and d[500] == 0 and np.sum(d == INF) == 999


def test_self_loop_negative_on_single_vertex():
    g = synth.Graph("loop", np.array([0, 1], np.int32), np.zeros(1, np.int32),
                    np.array([-1], np.int32), np.array([0], np.int32))
    for flags in MODES:
        st, _, _, _, stats = _one(g, 0, flags)
        assert st == bfq.NEG_CYCLE and stats["rounds"] == 1


@pytest.mark.parametrize("flags", MODES, ids=MODE_IDS)
def test_planted_cycles(flags):
    base = synth.grid_graph(64, 64, seed=5)
    for seed, cw in [(2, -1), (3, -1), (4, -5)]:
        g = synth.plant_negative_cycle(base, 5, seed=seed, base_weight=cw)
        assert _compare(g, 0, _one(g, 0, flags)) == oracle.NEG_CYCLE


def test_rounds_and_queue_share_a_handle():
    """Round-based and queue-driven queries on one handle, with a cycle run in
    between: every query exact."""
    base = synth.grid_graph(60, 60, seed=5)
    V = base.V
    u = base.tails().astype(np.int64)
    v = base.col.astype(np.int64)
    rp, col, order = synth.csr_from_edges(2 * V, np.r_[u, u + V], np.r_[v, v + V],
                                          return_order=True)
    two = synth.Graph("two", rp, col, np.r_[base.w, base.w][order].astype(np.int32),
                      np.array([V], np.int32))
    g = synth.plant_negative_cycle(two, 5, seed=3, reachable_from=[V])
    h = gpu_util.create(g)
    try:
        for src in (0, V, 17, V + 3, 5):
            for fn in ("rounds", "queue"):
                if fn == "rounds":
                    res = _run(h, g.V, src, 0)
                    ost = _compare(g, src, res)
                else:
                    st, d, hh, _ = gpu_util.run(h, g.V, src)
                    ost, od, oh, _ = oracle.spfa(g.row_ptr, g.col, g.w, src)
                    assert st == ost
                    if ost == oracle.OK:
                        assert np.array_equal(d, od) and np.array_equal(hh, oh)
                assert ost == (oracle.NEG_CYCLE if src >= V else oracle.OK)
    finally:
        bfq.bfq_graph_destroy(h)


def test_time_limit_ends_run_and_context_stays_usable():
    """A 40000-vertex path needs 40000 rounds; a 1 ms limit ends the run at a
    grid barrier with BFQ_ERR_TIMEOUT, and the device serves exact queries
    afterwards."""
    V = 40_000
    g = synth.path_graph(V, np.ones(V - 1, np.int32))
    h = gpu_util.create(g, bfq.make_tune(time_limit_ms=1))
    try:
        with pytest.raises(bfq.BfqError) as e:
            _run(h, g.V, 0, 0)
        assert e.value.code == bfq.ERR_TIMEOUT
    finally:
        bfq.bfq_graph_destroy(h)
    small = synth.workload_rmat(12)
    _compare(small, int(small.sources[0]), _one(small, int(small.sources[0]), 0))


def test_bad_arguments():
    g = synth.grid_graph(8, 8, seed=1)
    h = gpu_util.create(g)
    try:
        import torch
        d = torch.empty(g.V, dtype=torch.int32, device="cuda")
        for bad in (dict(src=g.V), dict(src=-1), dict(flags=2)):
            with pytest.raises(bfq.BfqError) as e:
                bfq.bfq_sssp_rounds(h, bad.get("src", 0), d, flags=bad.get("flags", 0))
            assert e.value.code == bfq.ERR_INVALID
        with pytest.raises(bfq.BfqError):
            bfq.bfq_sssp_rounds(h, 0, None)
        before = bfq.bfq_graph_device_bytes(h)
        st, _ = bfq.bfq_sssp_rounds(h, 0, d)
        assert st == bfq.OK and bfq.bfq_graph_device_bytes(h) > before
    finally:
        bfq.bfq_graph_destroy(h)


# ---- run-time tuning of a handle, L2 persisting window -----------------------

def test_set_tune_and_l2_window():
    g = synth.workload_rmat(16)
    h = gpu_util.create(g)
    try:
        t = bfq.bfq_graph_get_tune(h)
        assert t.l2_persist_pct == 0 and t.share_div >= 0
        ref = [gpu_util.run(h, g.V, int(s)) for s in g.sources[:2]]
        for pct, share in [(25, 1), (75, 4), (100, 0), (0, 2)]:
            t.l2_persist_pct = pct
            t.share_div = share
            bfq.bfq_graph_set_tune(h, t)
            got = bfq.bfq_graph_get_tune(h)
            assert got.l2_persist_pct == pct
            for s, r in zip(g.sources[:2], ref):
                res = gpu_util.run(h, g.V, int(s))
                assert res[0] == r[0] and np.array_equal(res[1], r[1])
                assert np.array_equal(res[2], r[2])
        for field, value in [("hub_degree", 4096), ("queues_per_cta", 3),
                             ("ctas_per_sm", 1), ("threads_per_cta", 128)]:
            bad = bfq.bfq_graph_get_tune(h)
            setattr(bad, field, value)
            with pytest.raises(bfq.BfqError) as e:
                bfq.bfq_graph_set_tune(h, bad)
            assert e.value.code == bfq.ERR_INVALID
        bad = bfq.bfq_graph_get_tune(h)
        bad.l2_persist_pct = 101
        with pytest.raises(bfq.BfqError):
            bfq.bfq_graph_set_tune(h, bad)
        _cmp = oracle.spfa(g.row_ptr, g.col, g.w, int(g.sources[0]))
        assert ref[0][0] == _cmp[0] and np.array_equal(ref[0][1], _cmp[1])
    finally:
        bfq.bfq_graph_destroy(h)
