"""Plant plausible mistakes in a copy of the oracle's label-correcting routine
(on the CPU) and check that the pins catch every one of them.

Dropping the explicit ">= INT32_MAX" discard is not listed: unreached labels
start at (INT32_MAX, -1), so such a candidate never compares smaller and the
mutant is equivalent to the original."""
import os
import subprocess

import numpy as np
import pytest

import oracle
from paper_2608_21826_gb300 import synth
from tests import helpers

SRC = os.path.join(os.path.dirname(oracle.__file__), "sssp_oracle.c")

MUTATIONS = {
    "dropped_weight": ("int64_t nd = du + (int64_t)w[e];", "int64_t nd = du;"),
    "wrong_sign": ("int64_t nd = du + (int64_t)w[e];", "int64_t nd = du - (int64_t)w[e];"),
    "hops_not_counted": ("int64_t nh = hu + 1;", "int64_t nh = hu;"),
    "no_tie_break": ("if (!lex_less(nd, nh, d[v], h[v])) continue;",
                     "if (!(nd < d[v])) continue;"),
    "transposed_compare": ("if (!lex_less(nd, nh, d[v], h[v])) continue;",
                           "if (!lex_less(d[v], h[v], nd, nh)) continue;"),
    "cycle_bound_off_by_one": ("if (nh >= V) { status = ORC_NEG_CYCLE; break; }",
                               "if (nh >= V - 1) { status = ORC_NEG_CYCLE; break; }"),
    "queue_flag_never_cleared": ("    inq[u] = 0;\n", "\n"),
    "weight_wrong_index": ("int64_t nd = du + (int64_t)w[e];",
                           "int64_t nd = du + (int64_t)w[row_ptr[u]];"),
    "source_label_wrong": ("  d[src] = 0;\n  h[src] = 0;\n  /* at most", "  d[src] = 0;\n  h[src] = 1;\n  /* at most"),
}


def _battery(o):
    """A compact run of the pins; returns the first failure or None."""
    for path in helpers.golden_files():
        g, exp = helpers.load_golden(path)
        st, d, h, _ = o.spfa(g.row_ptr, g.col, g.w, 0)
        if st != exp["status"]:
            return f"golden {path}: status"
        if "dist" in exp and (d.tolist() != exp["dist"] or h.tolist() != exp["hops"]):
            return f"golden {path}: labels"
    for seed in range(25):
        rng = np.random.default_rng(seed)
        V = int(rng.integers(1, 8))
        g = synth.random_graph(V, int(rng.integers(0, 3 * V + 1)), seed=1000 + seed,
                               wlo=-4, whi=9)
        neg, bd, bh = helpers.brute_force(g, 0)
        st, d, h, _ = o.spfa(g.row_ptr, g.col, g.w, 0)
        if st != (oracle.NEG_CYCLE if neg else oracle.OK):
            return f"brute force {seed}: status"
        if not neg and not (np.array_equal(d, bd) and np.array_equal(h, bh)):
            return f"brute force {seed}: labels"
    g = synth.workload_grid4k()
    st, d, h, _ = o.spfa(g.row_ptr, g.col, g.w, 0)
    db, hb = oracle.dijkstra(g.row_ptr, g.col, g.base_w, 0)
    ed, eh = helpers.shifted_expectation(db, hb, g.potential, 0)
    if st != oracle.OK or not np.array_equal(d, ed) or not np.array_equal(h, eh):
        return "potential transform"
    for seed in range(3):
        g = synth.random_potential_graph(500, 3000, seed=seed, wmax=1, pmax=3)
        st, d, h, _ = o.spfa(g.row_ptr, g.col, g.w, 0)
        db, hb = oracle.dijkstra(g.row_ptr, g.col, g.base_w, 0)
        ed, eh = helpers.shifted_expectation(db, hb, g.potential, 0)
        if st != oracle.OK or not np.array_equal(d, ed) or not np.array_equal(h, eh):
            return "potential transform, tie-heavy"
    w = np.random.default_rng(3).integers(-50, 50, size=199).astype(np.int32)
    g = synth.path_graph(200, w)
    st, d, h, _ = o.spfa(g.row_ptr, g.col, g.w, 0)
    if st != oracle.OK or not np.array_equal(d, np.r_[0, np.cumsum(w)]):
        return "path closed form"
    return None


def _compile(tmp_path, text, name):
    c = tmp_path / f"{name}.c"
    c.write_text(text)
    so = tmp_path / f"{name}.so"
    subprocess.check_call(["gcc", "-O1", "-std=c11", "-shared", "-fPIC", "-o", str(so), str(c)])
    return oracle.Variant(str(so))


def test_unmutated_copy_passes(tmp_path):
    assert _battery(_compile(tmp_path, open(SRC).read(), "clean")) is None


@pytest.mark.parametrize("name", sorted(MUTATIONS))
def test_mutation_is_caught(tmp_path, name):
    text = open(SRC).read()
    head, body = text.split("int oracle_spfa(", 1)
    old, new = MUTATIONS[name]
    assert old in body, f"mutation anchor missing: {name}"
    body = body.replace(old, new, 1)
    o = _compile(tmp_path, head + "int oracle_spfa(" + body, name)
    assert _battery(o) is not None, f"pins did not catch mutation {name}"


# ---- the parent-graph search of oracle_spfa_cycle_search -------------------

CYCLE_SEARCH_MUTATIONS = {
    # without parents the search never closes a cycle: only the slow hops test
    "parent_not_recorded": ("      p[v] = u;\n", "\n"),
    # a walk that stops on any earlier walk's vertex reports false cycles
    "walk_id_ignored": ("if (x >= 0 && mark[x] == *walk) return x;",
                        "if (x >= 0) return x;"),
    "weight_wrong_sign": ("      pw[v] = w[e];\n", "      pw[v] = -w[e];\n"),
    "search_never_run": ("if (++since_search >= V) {", "if (++since_search >= 4 * (int64_t)V * V) {"),
    "dropped_weight": ("      int64_t nd = du + (int64_t)w[e];\n      int64_t nh = hu + 1;\n"
                       "      if (nd >= ORC_INF32) continue;\n      if (!lex_less",
                       "      int64_t nd = du;\n      int64_t nh = hu + 1;\n"
                       "      if (nd >= ORC_INF32) continue;\n      if (!lex_less"),
}


def _battery_cycle(o):
    """Pins of the cycle search, compact; returns the first failure or None."""
    try:
        for seed in range(25):
            rng = np.random.default_rng(seed)
            V = int(rng.integers(1, 8))
            g = synth.random_graph(V, int(rng.integers(0, 3 * V + 1)), seed=1000 + seed,
                                   wlo=-4, whi=9)
            neg, bd, bh = helpers.brute_force(g, 0)
            st, d, h, _, _ = o.spfa_cycle_search(g.row_ptr, g.col, g.w, 0)
            if st != (oracle.NEG_CYCLE if neg else oracle.OK):
                return f"brute force {seed}: status"
            if not neg and not (np.array_equal(d, bd) and np.array_equal(h, bh)):
                return f"brute force {seed}: labels"
        for seed in range(3):
            g = synth.random_potential_graph(300, 1500, seed=seed)
            st, d, h, _ = oracle.spfa(g.row_ptr, g.col, g.w, 0)
            st2, d2, h2, _, _ = o.spfa_cycle_search(g.row_ptr, g.col, g.w, 0)
            if st2 != st or not (np.array_equal(d, d2) and np.array_equal(h, h2)):
                return "agreement with spfa"
        g = synth.plant_negative_cycle(synth.grid_graph(30, 30, seed=2, src=0), 5, seed=2)
        st, _, _, n, cv = o.spfa_cycle_search(g.row_ptr, g.col, g.w, 0)
        if st != oracle.NEG_CYCLE or n > 20 * g.E or cv not in set(int(x) for x in g.cycle):
            return "planted cycle found early"
    except ValueError as e:                 # the routine's own sign check fired
        return f"internal check: {e}"
    return None


def test_unmutated_cycle_search_passes(tmp_path):
    assert _battery_cycle(_compile(tmp_path, open(SRC).read(), "clean_cs")) is None


@pytest.mark.parametrize("name", sorted(CYCLE_SEARCH_MUTATIONS))
def test_cycle_search_mutation_is_caught(tmp_path, name):
    text = open(SRC).read()
    head, body = text.split("int oracle_spfa_cycle_search(", 1)
    old, new = CYCLE_SEARCH_MUTATIONS[name]
    if old not in body:                      # anchors inside the helper above it
        assert old in head, f"mutation anchor missing: {name}"
        head = head.replace(old, new, 1)
    else:
        body = body.replace(old, new, 1)
    o = _compile(tmp_path, head + "int oracle_spfa_cycle_search(" + body, name)
    assert _battery_cycle(o) is not None, f"pins did not catch mutation {name}"
