"""Pins of the oracle's negative-cycle resolution (oracle_spfa_neg_inf):
hand-derived fixtures, enumeration on tiny graphs, agreement with the plain
oracle when no negative cycle is reachable, structural invariants, and
planted mistakes that the pins must catch."""
import numpy as np
import pytest

import oracle
from paper_2608_21826_gb300 import synth
from tests import helpers
from tests.test_oracle_mutations import SRC, _compile

NEG_INF = helpers.NEG_INF
INF = helpers.INF


def _golden(o):
    for path in helpers.golden_neg_inf_files():
        g, exp = helpers.load_golden(path)
        st, d, h = o.spfa_neg_inf(g.row_ptr, g.col, g.w, 0)
        if st != exp["status"]:
            return f"{path}: status {st}"
        if d.tolist() != exp["dist"] or h.tolist() != exp["hops"]:
            return f"{path}: labels {d.tolist()} {h.tolist()}"
    return None


def _tiny(o, n=60):
    for seed in range(n):
        rng = np.random.default_rng(seed)
        V = int(rng.integers(1, 8))
        wlo, whi = (-4, 9) if seed % 2 == 0 else (-8, 6)
        g = synth.random_graph(V, int(rng.integers(0, 3 * V + 1)), seed=2000 + seed,
                               wlo=wlo, whi=whi)
        src = int(rng.integers(0, V))
        neg, bd, bh = helpers.brute_force_neg_inf(g, src)
        st, d, h = o.spfa_neg_inf(g.row_ptr, g.col, g.w, src)
        if st != (oracle.NEG_CYCLE if neg else oracle.OK):
            return f"tiny {seed}: status"
        if not (np.array_equal(d, bd) and np.array_equal(h, bh)):
            return f"tiny {seed}: labels {d} vs {bd}"
    return None


def _path(o, V=60):
    w = np.random.default_rng(3).integers(-50, 50, size=V - 1).astype(np.int32)
    g = synth.path_graph(V, w)
    st, d, h = o.spfa_neg_inf(g.row_ptr, g.col, g.w, 0)
    if st != oracle.OK or not np.array_equal(d, np.r_[0, np.cumsum(w)]):
        return "path closed form"
    return None


def _battery(o):
    for fn in (_golden, _tiny, _path):
        r = fn(o)
        if r:
            return r
    return None


def test_golden_fixtures():
    assert helpers.golden_neg_inf_files()
    assert _golden(oracle) is None


def test_enumeration_on_tiny_graphs():
    assert _tiny(oracle, n=200) is None


def test_path_closed_form():
    assert _path(oracle) is None


@pytest.mark.parametrize("seed", range(4))
def test_equals_plain_oracle_without_negative_cycles(seed):
    g = synth.random_potential_graph(3000, 15000, seed=seed)
    st, d, h, _ = oracle.spfa(g.row_ptr, g.col, g.w, 0)
    st2, d2, h2 = oracle.spfa_neg_inf(g.row_ptr, g.col, g.w, 0)
    assert st == st2 == oracle.OK
    assert np.array_equal(d, d2) and np.array_equal(h, h2)


@pytest.mark.parametrize("seed", range(6))
def test_invariants_with_planted_cycles(seed):
    """-inf is closed under successors and holds only reachable vertices; the
    finite labels satisfy every edge between finite vertices; the planted
    cycle is -inf."""
    base = synth.grid_graph(24, 24, seed=seed)
    g = synth.plant_negative_cycle(base, 4, seed=seed)
    st, d, h = oracle.spfa_neg_inf(g.row_ptr, g.col, g.w, 0)
    assert st == oracle.NEG_CYCLE
    ninf = d == NEG_INF
    assert np.all(ninf[g.cycle])
    assert np.all(h[ninf] == -2)
    lev = helpers.bfs_levels(g, 0)
    assert np.all(lev[ninf] >= 0)
    tails = g.tails()
    assert not np.any(ninf[tails] & ~ninf[g.col])            # closed under successors
    fin = (d != INF) & ~ninf
    m = fin[tails] & fin[g.col]
    assert np.all(d[tails[m]].astype(np.int64) + g.w[m] >= d[g.col[m]])


def test_unreachable_cycle_changes_nothing():
    base = synth.grid_graph(20, 20, seed=1)
    V = base.V
    u = base.tails().astype(np.int64)
    v = base.col.astype(np.int64)
    rp, col, order = synth.csr_from_edges(2 * V, np.r_[u, u + V], np.r_[v, v + V],
                                          return_order=True)
    two = synth.Graph("two", rp, col, np.r_[base.w, base.w][order].astype(np.int32),
                      np.array([V], np.int32))
    g = synth.plant_negative_cycle(two, 5, seed=3, reachable_from=[V])
    st, d, h, _ = oracle.spfa(g.row_ptr, g.col, g.w, 0)
    st2, d2, h2 = oracle.spfa_neg_inf(g.row_ptr, g.col, g.w, 0)
    assert st == st2 == oracle.OK and np.array_equal(d, d2) and np.array_equal(h, h2)
    st3, d3, _ = oracle.spfa_neg_inf(g.row_ptr, g.col, g.w, V)
    assert st3 == oracle.NEG_CYCLE
    assert np.all(d3[:V] == INF) and np.any(d3[V:] == NEG_INF)


MUTATIONS = {
    "no_propagation": ("const int32_t u = stack[--top];",
                       "const int32_t u = stack[--top]; continue;"),
    "one_round_short": ("round <= (int64_t)V - 1", "round <= (int64_t)V - 2"),
    "cycle_status_dropped": ("if (status >= 0 && any) status = ORC_NEG_CYCLE;", ""),
    "sign_of_weight": ("const int64_t nd = d[u] + (int64_t)w[e];",
                       "const int64_t nd = d[u] - (int64_t)w[e];"),
    "strict_test_loosened": ("if (d[u] + (int64_t)w[e] < d[v] && !ninf[v])",
                             "if (d[u] + (int64_t)w[e] <= d[v] && !ninf[v])"),
    "hops_marker": ("hops[v] = -2;", "hops[v] = -1;"),
}


def test_unmutated_copy_passes(tmp_path):
    assert _battery(_compile(tmp_path, open(SRC).read(), "clean_neg_inf")) is None


@pytest.mark.parametrize("name", sorted(MUTATIONS))
def test_mutation_is_caught(tmp_path, name):
    text = open(SRC).read()
    head, body = text.split("int oracle_spfa_neg_inf(", 1)
    old, new = MUTATIONS[name]
    assert old in body, f"mutation anchor missing: {name}"
    body = body.replace(old, new, 1)
    o = _compile(tmp_path, head + "int oracle_spfa_neg_inf(" + body, name)
    assert _battery(o) is not None, f"pins did not catch mutation {name}"
