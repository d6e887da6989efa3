"""Pins for the oracle: each test ties oracle/sssp_oracle.c to something other
than itself -- hand-derived fixtures, brute force, Floyd-Warshall, Dijkstra
through the potential transform, closed forms, invariants, and scipy."""
import numpy as np
import pytest

import oracle
from paper_2608_21826_gb300 import synth
from tests import helpers

INF = helpers.INF


@pytest.mark.parametrize("path", helpers.golden_files(), ids=lambda p: p.split("/")[-1])
def test_golden_fixtures(path):
    g, exp = helpers.load_golden(path)
    st, dist, hops, _ = oracle.spfa(g.row_ptr, g.col, g.w, int(g.sources[0]))
    assert st == exp["status"]
    if "dist" in exp:
        assert dist.tolist() == exp["dist"]
        assert hops.tolist() == exp["hops"]


@pytest.mark.parametrize("seed", range(60))
def test_brute_force_tiny(seed):
    rng = np.random.default_rng(seed)
    V = int(rng.integers(1, 8))
    E = int(rng.integers(0, 3 * V + 1))
    g = synth.random_graph(V, E, seed=1000 + seed, wlo=-4, whi=9)
    neg, bd, bh = helpers.brute_force(g, 0)
    st, d, h, _ = oracle.spfa(g.row_ptr, g.col, g.w, 0)
    assert st == (oracle.NEG_CYCLE if neg else oracle.OK)
    if not neg:
        assert np.array_equal(d, bd) and np.array_equal(h, bh)


@pytest.mark.parametrize("seed", range(80))
def test_floyd_warshall_small(seed):
    rng = np.random.default_rng(10_000 + seed)
    V = int(rng.integers(2, 48))
    E = int(rng.integers(V, 5 * V))
    if seed % 2:
        g = synth.random_graph(V, E, seed=seed, wlo=-3, whi=30)     # cycles likely
    else:
        g = synth.random_potential_graph(V, E, seed=seed)        # no cycles
    st_fw, dfw, hfw = oracle.floyd_warshall(g.row_ptr, g.col, g.w, 0)
    st, d, h, _ = oracle.spfa(g.row_ptr, g.col, g.w, 0)
    assert st == st_fw
    if st == oracle.OK:
        assert np.array_equal(d, dfw) and np.array_equal(h, hfw)


def _check_potential_pin(g, s):
    st, d, h, _ = oracle.spfa(g.row_ptr, g.col, g.w, s)
    assert st == oracle.OK
    db, hb = oracle.dijkstra(g.row_ptr, g.col, g.base_w, s)
    ed, eh = helpers.shifted_expectation(db, hb, g.potential, s)
    assert np.array_equal(d, ed)
    assert np.array_equal(h, eh)
    return d, h


def test_potential_transform_grid4k():
    g = synth.workload_grid4k()
    assert (g.V, g.E) == (4096, 16128)
    assert g.w.min() < 0
    _check_potential_pin(g, int(g.sources[0]))


@pytest.mark.parametrize("seed", range(6))
def test_potential_transform_random(seed):
    g = synth.random_potential_graph(3000, 12000, seed=seed)
    _check_potential_pin(g, 0)


@pytest.mark.parametrize("seed", range(6))
def test_potential_transform_tie_heavy(seed):
    """Base weights in {0, 1}: many equal-weight paths with different edge
    counts, so the fewest-edges rule decides most labels."""
    g = synth.random_potential_graph(2000, 12000, seed=900 + seed, wmax=1, pmax=3)
    _check_potential_pin(g, 0)


@pytest.mark.slow
def test_potential_transform_road1m_one_source():
    g = synth.workload_road1m()
    _check_potential_pin(g, int(g.sources[0]))


@pytest.mark.parametrize("seed", range(4))
def test_invariants_random(seed):
    """d[v] <= d[u] + w on every edge out of a reached vertex; every reached
    v != s has a tight in-edge, and hops[v] is 1 + the least hops[u] over its
    tight in-edges."""
    g = synth.random_potential_graph(2000, 9000, seed=50 + seed)
    st, d, h, _ = oracle.spfa(g.row_ptr, g.col, g.w, 0)
    assert st == oracle.OK
    u = g.tails().astype(np.int64)
    v = g.col.astype(np.int64)
    w = g.w.astype(np.int64)
    d64 = d.astype(np.int64)
    reached = d64[u] != INF
    assert np.all(d64[v][reached] <= d64[u][reached] + w[reached])
    tight = reached & (d64[u] + w == d64[v])
    best_h = np.full(g.V, np.iinfo(np.int64).max)
    np.minimum.at(best_h, v[tight], h[u[tight]].astype(np.int64) + 1)
    for x in range(g.V):
        if x == 0 or d[x] == INF:
            continue
        assert best_h[x] == h[x]


def test_path_closed_form():
    rng = np.random.default_rng(3)
    w = rng.integers(-50, 50, size=199).astype(np.int32)
    g = synth.path_graph(200, w)
    st, d, h, _ = oracle.spfa(g.row_ptr, g.col, g.w, 0)
    assert st == oracle.OK
    assert np.array_equal(d, np.concatenate([[0], np.cumsum(w)]))
    assert np.array_equal(h, np.arange(200))


def test_star_closed_form():
    w = np.arange(-20, 19, dtype=np.int32)
    g = synth.star_graph(40, w)
    st, d, h, _ = oracle.spfa(g.row_ptr, g.col, g.w, 0)
    assert st == oracle.OK
    assert np.array_equal(d[1:], w) and d[0] == 0
    assert np.array_equal(h, np.r_[0, np.ones(39, np.int32)])


def test_single_vertex_and_isolated_source():
    g = synth.Graph("one", np.array([0, 0], np.int32), np.zeros(0, np.int32),
                    np.zeros(0, np.int32), np.array([0], np.int32))
    st, d, h, _ = oracle.spfa(g.row_ptr, g.col, g.w, 0)
    assert st == oracle.OK and d.tolist() == [0] and h.tolist() == [0]
    g = synth.random_graph(50, 200, seed=9)
    # make vertex 0 have no out-edges
    deg = np.diff(g.row_ptr)
    keep = np.repeat(np.arange(50), deg) != 0
    row_ptr = np.r_[0, np.cumsum(np.where(np.arange(50) == 0, 0, deg))].astype(np.int32)
    st, d, h, _ = oracle.spfa(row_ptr, g.col[keep], g.w[keep], 0)
    assert st == oracle.OK
    assert d[0] == 0 and np.all(d[1:] == INF) and np.all(h[1:] == -1)


def test_zero_reduced_weights():
    """w = p(u) - p(v): every s->v path weighs p(s) - p(v), so dist is that and
    hops is the unweighted BFS level."""
    g = synth.grid_graph(20, 23, seed=4, wmax=1, pmax=1000)
    g.w = synth.potential_shift(g.row_ptr, g.col, np.zeros(g.E, np.int32), g.potential)
    st, d, h, _ = oracle.spfa(g.row_ptr, g.col, g.w, 7)
    p = g.potential.astype(np.int64)
    assert st == oracle.OK
    assert np.array_equal(d, p[7] - p)
    assert np.array_equal(h, helpers.bfs_levels(g, 7))


@pytest.mark.parametrize("seed", range(5))
def test_planted_cycle_reachable_and_not(seed):
    base = synth.grid_graph(30, 30, seed=seed, wmax=100, pmax=50, src=0)
    g = synth.plant_negative_cycle(base, 5, seed=seed)
    st, _, _, _ = oracle.spfa(g.row_ptr, g.col, g.w, 0)
    assert st == oracle.NEG_CYCLE
    # the same cycle planted where 0 cannot reach it: two disjoint copies of
    # the grid, source in the first, cycle in the second
    V = base.V
    u = base.tails().astype(np.int64)
    v = base.col.astype(np.int64)
    u2 = np.concatenate([u, u + V])
    v2 = np.concatenate([v, v + V])
    rp, col, order = synth.csr_from_edges(2 * V, u2, v2, return_order=True)
    w2 = np.concatenate([base.w, base.w])[order]
    two = synth.Graph("two", rp, col, w2.astype(np.int32), np.array([0], np.int32),
                      base_w=np.concatenate([base.base_w, base.base_w])[order],
                      potential=np.concatenate([base.potential, base.potential]))
    cyc = synth.plant_negative_cycle(two, 5, seed=seed, reachable_from=[])
    assert np.all(cyc.cycle >= V)
    st, d, h, _ = oracle.spfa(cyc.row_ptr, cyc.col, cyc.w, 0)
    assert st == oracle.OK
    st0, d0, h0, _ = oracle.spfa(base.row_ptr, base.col, base.w, 0)
    assert np.array_equal(d[:V], d0) and np.array_equal(h[:V], h0)
    assert np.all(d[V:] == INF)


@pytest.mark.parametrize("seed", range(10))
def test_scipy_cross_check(seed):
    sp = pytest.importorskip("scipy.sparse")
    cg = pytest.importorskip("scipy.sparse.csgraph")
    g = synth.random_potential_graph(400, 2500, seed=77 + seed)
    m = sp.csr_matrix((g.w.astype(np.float64), g.col, g.row_ptr), shape=(g.V, g.V))
    ref = cg.bellman_ford(m, directed=True, indices=0)
    st, d, _, _ = oracle.spfa(g.row_ptr, g.col, g.w, 0)
    assert st == oracle.OK
    ref_i = np.where(np.isinf(ref), INF, ref).astype(np.int64)
    assert np.array_equal(d.astype(np.int64), ref_i)


def test_pred_invariant_checker_accepts_and_rejects():
    g = synth.random_potential_graph(300, 1500, seed=5)
    st, d, h, _ = oracle.spfa(g.row_ptr, g.col, g.w, 0)
    # build one valid tree: for each reached v pick a tight in-edge with
    # hops[u] + 1 == hops[v]
    u = g.tails()
    pred = np.full(g.V, -1, np.int32)
    for e in range(g.E):
        a, b = int(u[e]), int(g.col[e])
        if b != 0 and d[a] != INF and int(d[a]) + int(g.w[e]) == int(d[b]) and h[a] + 1 == h[b]:
            pred[b] = a
    assert oracle.check_pred(g.row_ptr, g.col, g.w, 0, d, pred)
    bad = pred.copy()
    x = int(np.nonzero(bad > 0)[0][0])
    bad[x] = x                              # self-pointer: not an edge, a cycle
    assert not oracle.check_pred(g.row_ptr, g.col, g.w, 0, d, bad)


def test_reached_edges_counts_tails():
    g = synth.random_graph(100, 300, seed=2, wlo=1, whi=5)
    st, d, _, _ = oracle.spfa(g.row_ptr, g.col, g.w, 0)
    reach = synth.reachable(g.row_ptr, g.col, 0)
    assert oracle.reached_edges(g.row_ptr, d) == int(np.diff(g.row_ptr)[reach].sum())


# ---- spfa_cycle_search: the same FIFO Bellman-Ford with the parent-graph
# search for negative cycles (used where spfa's hops >= V test is too slow)

@pytest.mark.parametrize("seed", range(60))
def test_cycle_search_brute_force_tiny(seed):
    rng = np.random.default_rng(seed)
    V = int(rng.integers(1, 8))
    g = synth.random_graph(V, int(rng.integers(0, 3 * V + 1)), seed=1000 + seed, wlo=-4, whi=9)
    neg, bd, bh = helpers.brute_force(g, 0)
    st, d, h, _, cv = oracle.spfa_cycle_search(g.row_ptr, g.col, g.w, 0)
    assert st == (oracle.NEG_CYCLE if neg else oracle.OK)
    if not neg:
        assert np.array_equal(d, bd) and np.array_equal(h, bh) and cv == -1


@pytest.mark.parametrize("seed", range(40))
def test_cycle_search_agrees_with_spfa(seed):
    """Same status as spfa; without a cycle the same labels and the same scan
    count (the search changes nothing then)."""
    rng = np.random.default_rng(20_000 + seed)
    V = int(rng.integers(2, 300))
    E = int(rng.integers(V, 5 * V))
    if seed % 2:
        g = synth.random_graph(V, E, seed=seed, wlo=-3, whi=30)
    else:
        g = synth.random_potential_graph(V, E, seed=seed)
    st, d, h, n = oracle.spfa(g.row_ptr, g.col, g.w, 0)
    st2, d2, h2, n2, cv = oracle.spfa_cycle_search(g.row_ptr, g.col, g.w, 0)
    assert st == st2
    if st == oracle.OK:
        assert np.array_equal(d, d2) and np.array_equal(h, h2) and n == n2 and cv == -1


@pytest.mark.parametrize("seed", range(4))
def test_cycle_search_planted_cycles(seed):
    """A planted 5-cycle reachable from the source is found early, and the
    vertex reported lies on it; planted where the source cannot reach it, the
    status is OK with the labels of the graph without it."""
    base = synth.grid_graph(60, 60, seed=seed, wmax=100, pmax=50, src=0)
    g = synth.plant_negative_cycle(base, 5, seed=seed)
    st, _, _, n, cv = oracle.spfa_cycle_search(g.row_ptr, g.col, g.w, 0)
    assert st == oracle.NEG_CYCLE
    assert cv in set(int(x) for x in g.cycle)
    assert n <= 20 * g.E                # spfa's hops test needs about V/5 laps
    # the same kind of cycle in a second, unreachable copy of the grid
    V = base.V
    u = base.tails().astype(np.int64)
    v = base.col.astype(np.int64)
    rp, col, order = synth.csr_from_edges(2 * V, np.r_[u, u + V], np.r_[v, v + V],
                                          return_order=True)
    two = synth.Graph("two", rp, col, np.r_[base.w, base.w][order].astype(np.int32),
                      np.array([0], np.int32),
                      base_w=np.r_[base.base_w, base.base_w][order],
                      potential=np.r_[base.potential, base.potential])
    far = synth.plant_negative_cycle(two, 5, seed=seed, reachable_from=[])
    assert np.all(far.cycle >= V)
    st, d, h, _, cv = oracle.spfa_cycle_search(far.row_ptr, far.col, far.w, 0)
    st0, d0, h0, _ = oracle.spfa(far.row_ptr, far.col, far.w, 0)
    assert st == st0 == oracle.OK and cv == -1
    assert np.array_equal(d, d0) and np.array_equal(h, h0)


def test_cycle_search_cycle_through_source_and_golden():
    for path in helpers.golden_files():
        g, exp = helpers.load_golden(path)
        st, d, h, _, _ = oracle.spfa_cycle_search(g.row_ptr, g.col, g.w, int(g.sources[0]))
        assert st == exp["status"], path
        if "dist" in exp:
            assert d.tolist() == exp["dist"] and h.tolist() == exp["hops"], path
