"""Generator checks: determinism, CSR well-formedness, workload shapes,
potential-shifted weights free of negative cycles, planted cycles."""
import numpy as np
import pytest

import oracle
from paper_2608_21826_gb300 import synth


def _well_formed(g):
    assert g.row_ptr.dtype == np.int32 and g.col.dtype == np.int32 and g.w.dtype == np.int32
    assert g.row_ptr[0] == 0 and np.all(np.diff(g.row_ptr) >= 0) and g.row_ptr[-1] == g.E
    assert g.col.min(initial=0) >= 0 and g.col.max(initial=0) < g.V
    u = g.tails().astype(np.int64)
    assert not np.any(u == g.col)                                   # no self-loops
    key = u * g.V + g.col
    assert np.all(np.diff(key) > 0)                                 # sorted, no repeats


def test_deterministic():
    a = synth.workload_grid4k()
    b = synth.workload_grid4k()
    assert np.array_equal(a.w, b.w) and np.array_equal(a.col, b.col)
    r1 = synth.rmat_graph(12, 8, seed=5)
    r2 = synth.rmat_graph(12, 8, seed=5)
    assert np.array_equal(r1.row_ptr, r2.row_ptr) and np.array_equal(r1.w, r2.w)
    assert np.array_equal(r1.sources, r2.sources)


def test_grid4k_shape():
    g = synth.workload_grid4k()
    _well_formed(g)
    assert (g.V, g.E) == (4096, 16128)
    assert g.base_w.min() >= 1 and g.base_w.max() <= 100
    assert g.potential.min() >= 0 and g.potential.max() <= 50
    assert g.w.min() < 0 and list(g.sources) == [0]


def test_road_small_twin_shape():
    g = synth.road_graph(64, seed=3)
    _well_formed(g)
    und = 2 * 64 * 63
    kept = int(round(0.9 * und))
    short = int(round(0.01 * 64 * 64))
    assert 2 * (kept + short) - 4 * short <= g.E <= 2 * (kept + short)
    assert len(g.sources) == 8


def test_rmat_small_twin():
    g = synth.rmat_graph(14, 16, seed=9)
    _well_formed(g)
    assert g.V == 2**14 and g.E <= 16 * 2**14
    deg = np.diff(g.row_ptr)
    assert deg.max() > 20 * deg.mean()                               # skewed degrees
    assert np.all(deg[g.sources] > 0) and len(g.sources) == 4


def test_pair_table_probabilities():
    t = synth._pair_table((0.57, 0.19, 0.19, 0.05))
    ub, vb = t >> 2, t & 3
    # first-level marginals: u bit set with prob c+d, v bit set with prob b+d
    assert abs((ub >> 1).mean() - 0.24) < 1e-3
    assert abs((vb >> 1).mean() - 0.24) < 1e-3
    both = ((ub >> 1) & (vb >> 1)).mean()
    assert abs(both - 0.05) < 1e-3


@pytest.mark.parametrize("seed", range(3))
def test_potentials_leave_no_negative_cycle(seed):
    g = synth.rmat_graph(11, 8, seed=seed)
    for s in g.sources:
        st, _, _, _ = oracle.spfa(g.row_ptr, g.col, g.w, int(s))
        assert st == oracle.OK


def test_planted_cycle_is_negative_and_reachable():
    g = synth.plant_negative_cycle(synth.grid_graph(20, 20, seed=2), 5, seed=3)
    cyc = g.cycle
    total = 0
    for a, b in zip(cyc, np.roll(cyc, -1)):
        lo, hi = g.row_ptr[a], g.row_ptr[a + 1]
        e = lo + int(np.nonzero(g.col[lo:hi] == b)[0][0])
        total += int(g.w[e])
    assert total == -5
    reach = synth.reachable(g.row_ptr, g.col, 0)
    assert np.all(reach[cyc])


def test_batched_mix_small():
    graphs, q = synth.workload_batched(n_graphs=10, vmin=200, vmax=3000, seed=5)
    assert len(graphs) == 10
    assert sum(g.cycle is not None for g in graphs) == 1
    for g in graphs:
        _well_formed(g)
    assert q.shape[1] == 2 and q[:, 0].max() == 9
    for gi, s in q:
        g = graphs[gi]
        st, _, _, _ = oracle.spfa(g.row_ptr, g.col, g.w, int(s))
        assert st == (oracle.NEG_CYCLE if g.cycle is not None else oracle.OK)
