"""Parity of the CUDA SSSP path (through the C ABI) with the oracle: dist,
hops and status bit-exact, predecessor trees checked by invariant."""
import numpy as np
import pytest

import oracle
from paper_2608_21826_gb300 import bfq, synth
from tests import gpu_util, helpers

pytestmark = pytest.mark.gpu
INF = helpers.INF


def _compare(g, src, res, check_pred=False):
    st, d, h, p = res
    ost, od, oh, _ = oracle.spfa(g.row_ptr, g.col, g.w, src)
    assert st == ost, (st, ost)
    if ost == oracle.OK:
        bad = np.nonzero(d != od)[0]
        assert bad.size == 0, f"{bad.size} dist mismatches, first {bad[:5]}: {d[bad[:5]]} vs {od[bad[:5]]}"
        assert np.array_equal(h, oh), "hops mismatch"
        if check_pred:
            assert oracle.check_pred(g.row_ptr, g.col, g.w, src, d, p)
    return ost


# the persistent kernel explicitly (small graphs run on the single-CTA path by
# default, which tests/test_gpu_small.py covers)
PERSISTENT = bfq.make_tune(small_path=bfq.SMALL_PATH_OFF)


@pytest.mark.parametrize("tune", [None, PERSISTENT], ids=["auto", "persistent"])
@pytest.mark.parametrize("path", helpers.golden_files(), ids=lambda p: p.split("/")[-1])
def test_golden(path, tune):
    g, exp = helpers.load_golden(path)
    st, d, h, p = gpu_util.sssp(g, 0, tune=tune, want_pred=True)
    assert st == exp["status"]
    if "dist" in exp:
        assert d.tolist() == exp["dist"] and h.tolist() == exp["hops"]
        assert oracle.check_pred(g.row_ptr, g.col, g.w, 0, d, p)


@pytest.mark.parametrize("tune", [None, PERSISTENT], ids=["auto", "persistent"])
@pytest.mark.parametrize("seed", range(30))
def test_random_with_cycles(seed, tune):
    rng = np.random.default_rng(seed)
    V = int(rng.integers(1, 3000))
    E = int(rng.integers(0, 6 * V + 1))
    g = synth.random_graph(V, E, seed=500 + seed, wlo=-3, whi=40)
    _compare(g, 0, gpu_util.sssp(g, 0, tune=tune))


@pytest.mark.parametrize("seed", range(10))
def test_random_potential(seed):
    rng = np.random.default_rng(100 + seed)
    V = int(rng.integers(2000, 40000))
    g = synth.random_potential_graph(V, 6 * V, seed=seed)
    assert _compare(g, 0, gpu_util.sssp(g, 0, want_pred=True), check_pred=True) == oracle.OK


def test_tie_heavy():
    g = synth.random_potential_graph(30000, 200000, seed=3, wmax=1, pmax=3)
    _compare(g, 0, gpu_util.sssp(g, 0, want_pred=True), check_pred=True)


@pytest.mark.parametrize("tune", [None, PERSISTENT], ids=["auto", "persistent"])
def test_grid4k_full(tune):
    g = synth.workload_grid4k()
    h = gpu_util.create(g, tune)
    try:
        res = gpu_util.run(h, g.V, 0, want_pred=True)
        _compare(g, 0, res, check_pred=True)
        stats = bfq.bfq_get_stats(h)
        assert stats["m_reached"] == oracle.reached_edges(g.row_ptr, res[1]) == g.E
        assert stats["reached"] == g.V
        assert stats["relaxed"] >= g.E and stats["dequeued"] >= g.V
    finally:
        bfq.bfq_graph_destroy(h)


def test_road_twin_all_sources():
    g = synth.road_graph(256, seed=7)
    h = gpu_util.create(g)
    try:
        for s in g.sources:
            _compare(g, int(s), gpu_util.run(h, g.V, int(s), want_pred=True), check_pred=True)
    finally:
        bfq.bfq_graph_destroy(h)


def test_road1m_full_all_sources():
    g = synth.workload_road1m()
    h = gpu_util.create(g)
    try:
        for s in g.sources:
            _compare(g, int(s), gpu_util.run(h, g.V, int(s)))
    finally:
        bfq.bfq_graph_destroy(h)


@pytest.mark.parametrize("scale", [12, 16])
def test_rmat_twins(scale):
    g = synth.workload_rmat(scale)
    h = gpu_util.create(g)
    try:
        for s in g.sources:
            _compare(g, int(s), gpu_util.run(h, g.V, int(s), want_pred=True), check_pred=True)
        assert bfq.bfq_get_stats(h)["hub_chunks"] > 0 or np.diff(g.row_ptr).max() <= 512
    finally:
        bfq.bfq_graph_destroy(h)


def test_rmat22_full_all_sources():
    g = synth.workload_rmat(22)
    h = gpu_util.create(g)
    try:
        for s in g.sources:
            st, d, hh, _ = gpu_util.run(h, g.V, int(s))
            # exact against Dijkstra through the potential transform (fast),
            # and against the label-correcting oracle for the first source
            db, hb = oracle.dijkstra(g.row_ptr, g.col, g.base_w, int(s))
            ed, eh = helpers.shifted_expectation(db, hb, g.potential, int(s))
            assert st == bfq.OK
            assert np.array_equal(d, ed) and np.array_equal(hh, eh)
        _compare(g, int(g.sources[0]), gpu_util.run(h, g.V, int(g.sources[0])))
    finally:
        bfq.bfq_graph_destroy(h)


@pytest.mark.parametrize("tune", [
    dict(hub_degree=32, chunk_edges=32),
    dict(batch_items=1),
    dict(queues_per_cta=4),
    dict(ctas_per_sm=1),
    dict(hub_degree=64, chunk_edges=32, batch_items=4, queues_per_cta=2),
    dict(relax_atomic=1),
    dict(relax_atomic=2),
    dict(relax_atomic=2, hub_degree=32, chunk_edges=32, batch_items=4),
    dict(kernel_ctas=3),
    dict(kernel_ctas=4),
    dict(kernel_ctas=3, relax_atomic=2, hub_degree=32, chunk_edges=32, batch_items=4),
    dict(kernel_ctas=3, ctas_per_sm=2, queues_per_cta=2),
    dict(queue_form=2),
    dict(queue_form=2, kernel_ctas=3),
    dict(queue_form=2, hub_degree=32, chunk_edges=32, batch_items=4, queues_per_cta=4),
    dict(queue_form=2, relax_atomic=2, ctas_per_sm=1),
    dict(relax_atomic=3),
    dict(relax_atomic=3, kernel_ctas=3, hub_degree=32, chunk_edges=32, batch_items=4),
    dict(relax_atomic=3, queue_form=2, queues_per_cta=4),
], ids=lambda d: ",".join(f"{k}={v}" for k, v in d.items()))
def test_tunes(tune):
    g = synth.workload_rmat(14)
    t = bfq.make_tune(**tune)
    h = gpu_util.create(g, t)
    try:
        for s in g.sources[:2]:
            _compare(g, int(s), gpu_util.run(h, g.V, int(s), want_pred=True), check_pred=True)
    finally:
        bfq.bfq_graph_destroy(h)


def test_star_hub_chunks():
    V = 200_000
    w = np.random.default_rng(1).integers(-1000, 1000, size=V - 1).astype(np.int32)
    g = synth.star_graph(V, w)
    st, d, h, p = gpu_util.sssp(g, 0, want_pred=True)
    assert st == bfq.OK and d[0] == 0 and np.array_equal(d[1:], w)
    assert np.all(h[1:] == 1) and np.all(p[1:] == 0)


def test_long_path():
    V = 20_000
    w = np.random.default_rng(2).integers(-5, 9, size=V - 1).astype(np.int32)
    g = synth.path_graph(V, w)
    st, d, h, _ = gpu_util.sssp(g, 0)
    assert st == bfq.OK
    assert np.array_equal(d, np.r_[0, np.cumsum(w)]) and np.array_equal(h, np.arange(V))


@pytest.mark.parametrize("tune", [None, PERSISTENT], ids=["auto", "persistent"])
def test_single_vertex_and_no_edges(tune):
    g = synth.Graph("one", np.array([0, 0], np.int32), np.zeros(0, np.int32),
                    np.zeros(0, np.int32), np.array([0], np.int32))
    st, d, h, p = gpu_util.sssp(g, 0, tune=tune, want_pred=True)
    assert st == bfq.OK and d.tolist() == [0] and h.tolist() == [0] and p.tolist() == [-1]
    rp = np.zeros(1001, np.int32)
    g = synth.Graph("empty", rp, np.zeros(0, np.int32), np.zeros(0, np.int32),
                    np.array([0], np.int32))
    st, d, h, _ = gpu_util.sssp(g, 500, tune=tune)
    assert st == bfq.OK and d[500] == 0 and np.sum(d == INF) == 999


def test_device_resident_input():
    g = synth.rmat_graph(13, 8, seed=4)
    _compare(g, int(g.sources[0]), gpu_util.sssp(g, int(g.sources[0]), on_device=True))


def test_cycle_then_clean_on_one_handle():
    """A run that stops on a negative cycle leaves the queues dirty; the next
    run on the same handle must reset them and still be exact."""
    base = synth.grid_graph(60, 60, seed=5)
    V = base.V
    u = base.tails().astype(np.int64)
    v = base.col.astype(np.int64)
    rp, col, order = synth.csr_from_edges(2 * V, np.r_[u, u + V], np.r_[v, v + V],
                                          return_order=True)
    two = synth.Graph("two", rp, col, np.r_[base.w, base.w][order].astype(np.int32),
                      np.array([V], np.int32), base_w=np.r_[base.base_w, base.base_w][order],
                      potential=np.r_[base.potential, base.potential])
    g = synth.plant_negative_cycle(two, 5, seed=3, reachable_from=[V])   # in copy 2
    assert np.all(g.cycle >= V)
    h = gpu_util.create(g, PERSISTENT)
    try:
        for src in (V, 0, V + 17, 5, 0):
            res = gpu_util.run(h, g.V, src)
            ost = _compare(g, src, res)
            assert ost == (oracle.NEG_CYCLE if src >= V else oracle.OK)
    finally:
        bfq.bfq_graph_destroy(h)


def _two_copies_cycle_in_second(side=60):
    base = synth.grid_graph(side, side, seed=5)
    V = base.V
    u = base.tails().astype(np.int64)
    v = base.col.astype(np.int64)
    rp, col, order = synth.csr_from_edges(2 * V, np.r_[u, u + V], np.r_[v, v + V],
                                          return_order=True)
    two = synth.Graph("two", rp, col, np.r_[base.w, base.w][order].astype(np.int32),
                      np.array([V], np.int32))
    return synth.plant_negative_cycle(two, 5, seed=3, reachable_from=[V]), V


def test_register_forms_switch_on_one_handle():
    """The two register forms run different grids over a prefix of the same
    sub-queues.  Runs that stop on a negative cycle leave queues dirty in one
    form; the next run, in either form, must reset every sub-queue and be
    exact; the stats report the grid of the form that ran."""
    g, V = _two_copies_cycle_in_second()
    h = gpu_util.create(g, PERSISTENT)
    try:
        grids = {}
        seq = [(4, V), (3, 0), (3, V + 11), (4, 0), (4, 7), (3, V), (3, 5), (4, V + 3), (4, 9)]
        for form, src in seq:
            t = bfq.bfq_graph_get_tune(h)
            t.kernel_ctas = form
            bfq.bfq_graph_set_tune(h, t)
            ost = _compare(g, src, gpu_util.run(h, g.V, src, want_pred=True), check_pred=True)
            assert ost == (oracle.NEG_CYCLE if src >= V else oracle.OK)
            st = bfq.bfq_get_stats(h)
            grids.setdefault(form, set()).add((st["grid"], st["queues"]))
        assert len(grids[3]) == 1 and len(grids[4]) == 1
        (g3, q3), = grids[3]
        (g4, q4), = grids[4]
        assert g3 <= g4 and q3 <= q4 and g3 * q4 == g4 * q3
    finally:
        bfq.bfq_graph_destroy(h)


@pytest.mark.parametrize("form", [0, 3, 4])
def test_register_forms_road_and_hubs(form):
    t = bfq.make_tune(kernel_ctas=form)
    for g in (synth.grid_graph(256, 256, seed=8), synth.workload_rmat(13)):
        h = gpu_util.create(g, t)
        try:
            for s in g.sources[:2]:
                _compare(g, int(s), gpu_util.run(h, g.V, int(s), want_pred=True),
                         check_pred=True)
        finally:
            bfq.bfq_graph_destroy(h)


def test_many_runs_reuse_state():
    g = synth.workload_rmat(15)
    h = gpu_util.create(g)
    try:
        rng = np.random.default_rng(0)
        cand = np.nonzero(np.diff(g.row_ptr) > 0)[0]
        for s in rng.choice(cand, size=12, replace=False):
            _compare(g, int(s), gpu_util.run(h, g.V, int(s)))
    finally:
        bfq.bfq_graph_destroy(h)


def test_bad_arguments():
    g = synth.grid_graph(8, 8, seed=1)
    h = gpu_util.create(g)
    try:
        import torch
        d = torch.empty(g.V, dtype=torch.int32, device="cuda")
        with pytest.raises(bfq.BfqError) as e:
            bfq.bfq_sssp(h, g.V, d)
        assert e.value.code == bfq.ERR_INVALID
        with pytest.raises(bfq.BfqError):
            bfq.bfq_sssp(h, 0, None)
        bad_col = g.col.copy()
        bad_col[3] = g.V
        with pytest.raises(bfq.BfqError):
            bfq.bfq_graph_create(g.row_ptr, bad_col, g.w)
        st, dd, _, _ = gpu_util.run(h, g.V, 0)          # handle still usable
        assert st == bfq.OK
    finally:
        bfq.bfq_graph_destroy(h)


def test_timeout_leaves_context_usable():
    """An in-flight count that nothing can retire (test hook) keeps the
    persistent kernel idle until its time limit; the run must end with
    BFQ_ERR_TIMEOUT, and the device must serve exact queries afterwards."""
    g = synth.workload_rmat(12)
    t = bfq.make_tune(time_limit_ms=30, test_phantom_items=1)
    h = gpu_util.create(g, t)
    try:
        with pytest.raises(bfq.BfqError) as e:
            gpu_util.run(h, g.V, int(g.sources[0]))
        assert e.value.code == bfq.ERR_TIMEOUT
    finally:
        bfq.bfq_graph_destroy(h)
    _compare(g, int(g.sources[0]), gpu_util.sssp(g, int(g.sources[0])))


def _path_into_cycle(n_path, cyc_w, seed=0):
    """0 -> 1 -> ... -> n_path-1 (weights U[-3,5]) then a 5-cycle on the last
    five path vertices closed with total weight cyc_w."""
    rng = np.random.default_rng(seed)
    w = rng.integers(-3, 6, size=n_path - 1).astype(np.int64)
    u = list(range(n_path - 1))
    v = list(range(1, n_path))
    ww = list(w)
    c = list(range(n_path - 5, n_path))
    # the cycle c0 -> c1 -> ... -> c4 -> c0 reuses the path edges c0..c4 and
    # adds the closing edge c4 -> c0
    inner = int(sum(w[n_path - 5:n_path - 1]))
    u.append(c[4])
    v.append(c[0])
    ww.append(cyc_w - inner)
    rp, col, order = synth.csr_from_edges(n_path, np.array(u), np.array(v), return_order=True)
    return synth.Graph("pathcycle", rp, col, np.array(ww, np.int32)[order], np.array([0], np.int32))


@pytest.mark.parametrize("tune", [None, PERSISTENT], ids=["auto", "persistent"])
@pytest.mark.parametrize("cyc_w", [-1, 0, 3])
def test_cycle_accelerator_sound_and_fast(cyc_w, tune):
    """A deep path feeding a 5-cycle: the hop counts pass the walk threshold,
    so the recorded-edge walk runs; it must report only a negative cycle (the
    zero and positive ones are not), and quickly."""
    g = _path_into_cycle(3000, cyc_w)
    h = gpu_util.create(g, tune)
    try:
        res = gpu_util.run(h, g.V, 0)
        ost = _compare(g, 0, res)
        assert ost == (oracle.NEG_CYCLE if cyc_w < 0 else oracle.OK)
    finally:
        bfq.bfq_graph_destroy(h)


def test_planted_cycle_detected_fast_on_large_graph():
    """A 5-edge negative cycle in a 1M-vertex grid: hops >= V alone would need
    ~V/5 laps of the cycle; the recorded-edge walk proves it far sooner."""
    base = synth.grid_graph(1024, 1024, seed=13)
    g = synth.plant_negative_cycle(base, 5, seed=2)
    h = gpu_util.create(g)
    try:
        st, _, _, _ = gpu_util.run(h, g.V, 0, want_hops=False)
        assert st == bfq.NEG_CYCLE
        assert bfq.bfq_get_stats(h)["kernel_ms"] < 200.0
    finally:
        bfq.bfq_graph_destroy(h)


@pytest.mark.parametrize("relax", [1, 2, 3])
@pytest.mark.parametrize("walk", [2, 8, 64, 1 << 30])
def test_cycle_walk_threshold_changes_speed_only(walk, relax):
    """Every first-walk threshold gives the same answers: exact labels on a
    clean deep graph, BFQ_NEG_CYCLE with a planted cycle (at 2^30 only the
    hops >= V test is left)."""
    t = bfq.make_tune(cycle_walk_hops=walk, relax_atomic=relax,
                      small_path=bfq.SMALL_PATH_OFF)
    clean = synth.road_graph(128, seed=3)
    _compare(clean, 0, gpu_util.sssp(clean, 0, tune=t))
    g = synth.plant_negative_cycle(synth.grid_graph(48, 48, seed=4), 5, seed=6)
    assert _compare(g, 0, gpu_util.sssp(g, 0, tune=t)) == oracle.NEG_CYCLE


def test_cycle_walk_threshold_validated():
    g = synth.grid_graph(8, 8, seed=1)
    for bad in (1, -3, (1 << 30) + 1):
        with pytest.raises(bfq.BfqError):
            gpu_util.create(g, bfq.make_tune(cycle_walk_hops=bad))


@pytest.mark.parametrize("form", [1, 2])
def test_queue_forms_full_size_and_cycles(form):
    """The exact-count (1) and single-shot (2) worklist reservations give
    the oracle's results on the road-like grid, R-MAT 16 and a planted
    cycle, and a switch between them on one handle meets no stale queue
    state."""
    road = synth.workload_road1m()
    rm = synth.workload_rmat(16)
    cyc = synth.plant_negative_cycle(synth.grid_graph(50, 50, seed=3), 5, seed=2)
    for g, srcs in ((road, road.sources[:2]), (rm, rm.sources[:2]), (cyc, [0])):
        h = gpu_util.create(g, bfq.make_tune(queue_form=form, small_path=bfq.SMALL_PATH_OFF))
        try:
            for s in srcs:
                _compare(g, int(s), gpu_util.run(h, g.V, int(s)))
            t = bfq.bfq_graph_get_tune(h)
            t.queue_form = 3 - form
            bfq.bfq_graph_set_tune(h, t)
            _compare(g, int(srcs[0]), gpu_util.run(h, g.V, int(srcs[0])))
        finally:
            bfq.bfq_graph_destroy(h)


@pytest.mark.parametrize("form", [bfq.RELAX_MIN, bfq.RELAX_CAS, bfq.RELAX_FILTERED])
def test_relax_forms_full_size_and_cycles(form):
    """Each relaxation form (atomicMin, compare-and-swap, load-filtered
    atomicMin) gives the oracle's results on R-MAT 22, the road-like grid
    and a planted cycle, and a switch to the next form on one handle meets
    no stale state."""
    rm = synth.workload_rmat(22)
    road = synth.workload_road1m()
    cyc = synth.plant_negative_cycle(synth.grid_graph(50, 50, seed=3), 5, seed=2)
    nxt = {bfq.RELAX_MIN: bfq.RELAX_CAS, bfq.RELAX_CAS: bfq.RELAX_FILTERED,
           bfq.RELAX_FILTERED: bfq.RELAX_MIN}[form]
    for g, srcs in ((rm, rm.sources[:1]), (road, road.sources[:2]), (cyc, [0])):
        h = gpu_util.create(g, bfq.make_tune(relax_atomic=form, small_path=bfq.SMALL_PATH_OFF))
        try:
            for s in srcs:
                _compare(g, int(s), gpu_util.run(h, g.V, int(s)))
            t = bfq.bfq_graph_get_tune(h)
            t.relax_atomic = nxt
            bfq.bfq_graph_set_tune(h, t)
            _compare(g, int(srcs[0]), gpu_util.run(h, g.V, int(srcs[0])))
        finally:
            bfq.bfq_graph_destroy(h)


@pytest.mark.parametrize("seed", range(12))
def test_single_shot_random_and_edge_cases(seed):
    """The single-shot sub-queues (whose warps publish a batch's children in
    the same round trips as their next dequeue) on random graphs with and
    without cycles, a hub star, a long path and the golden fixtures."""
    rng = np.random.default_rng(300 + seed)
    t = bfq.make_tune(queue_form=2, small_path=bfq.SMALL_PATH_OFF)
    V = int(rng.integers(1, 4000))
    g = (synth.random_graph(V, int(rng.integers(0, 4 * V + 1)), seed=seed, wlo=-3, whi=40)
         if seed % 2 else synth.random_potential_graph(max(2, V), 5 * max(2, V), seed=seed))
    _compare(g, 0, gpu_util.sssp(g, 0, tune=t, want_pred=True), check_pred=True)
    if seed == 0:
        w = np.random.default_rng(1).integers(-1000, 1000, size=60_000 - 1).astype(np.int32)
        star = synth.star_graph(60_000, w)
        st, d, h, p = gpu_util.sssp(star, 0, tune=t, want_pred=True)
        assert st == bfq.OK and np.array_equal(d[1:], w) and np.all(p[1:] == 0)
        pw = np.random.default_rng(2).integers(-5, 9, size=5_000 - 1).astype(np.int32)
        path = synth.path_graph(5_000, pw)
        st, d, h, _ = gpu_util.sssp(path, 0, tune=t)
        assert st == bfq.OK and np.array_equal(d, np.r_[0, np.cumsum(pw)])
        for fx in helpers.golden_files():
            gg, exp = helpers.load_golden(fx)
            st, d, h, _ = gpu_util.sssp(gg, 0, tune=t)
            assert st == exp["status"], fx
            if "dist" in exp:
                assert d.tolist() == exp["dist"] and h.tolist() == exp["hops"], fx
