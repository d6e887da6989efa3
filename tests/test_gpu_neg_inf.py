"""Parity of negative-cycle resolution (neg_cycle_mode = MARK) on the
queue-driven path with the oracle's minus-infinity distances: status, dist and
hops bit-exact; predecessors checked on the finite vertices."""
import numpy as np
import pytest

import oracle
from paper_2608_21826_gb300 import bfq, synth
from tests import gpu_util, helpers

pytestmark = pytest.mark.gpu
INF = helpers.INF
NEG_INF = helpers.NEG_INF
MARK = bfq.make_tune(neg_cycle_mode=bfq.NEG_CYCLE_MARK)


def _check_pred_finite(g, src, d, h, p):
    """pred[v] is a tight edge one hop closer for every finite v != src, and
    -1 on the source, unreachable and minus-infinity vertices."""
    tails = g.tails()
    fin = (d != INF) & (d != NEG_INF)
    assert p[src] == -1 or not fin[src]
    assert np.all(p[~fin] == -1)
    v = np.nonzero(fin)[0]
    v = v[v != src]
    u = p[v]
    assert np.all(u >= 0) and np.all(fin[u])
    assert np.all(h[u] + 1 == h[v])
    # (u, v) must be an edge with d[u] + w == d[v]
    key = tails.astype(np.int64) * g.V + g.col
    order = np.argsort(key, kind="stable")
    ks = key[order]
    want = u.astype(np.int64) * g.V + v
    pos = np.searchsorted(ks, want)
    ok = np.zeros(len(v), bool)
    for i in range(len(v)):      # parallel edges: any tight one counts
        j = pos[i]
        while j < len(ks) and ks[j] == want[i]:
            e = order[j]
            if int(d[u[i]]) + int(g.w[e]) == int(d[v[i]]):
                ok[i] = True
                break
            j += 1
    assert ok.all()


def _compare(g, src, res, check_pred=False):
    st, d, h, p = res
    ost, od, oh = oracle.spfa_neg_inf(g.row_ptr, g.col, g.w, src)
    assert st == ost, (st, ost)
    if ost in (oracle.OK, oracle.NEG_CYCLE):
        bad = np.nonzero(d != od)[0]
        assert bad.size == 0, f"{bad.size} dist mismatches, first {bad[:5]}: {d[bad[:5]]} vs {od[bad[:5]]}"
        assert np.array_equal(h, oh), "hops mismatch"
        if check_pred:
            _check_pred_finite(g, src, d, h, p)
    return ost


def _one(g, src, want_pred=True):
    return gpu_util.sssp(g, src, tune=MARK, want_pred=want_pred)


@pytest.mark.parametrize("path", helpers.golden_neg_inf_files(), ids=lambda p: p.split("/")[-1])
def test_golden(path):
    g, exp = helpers.load_golden(path)
    st, d, h, p = _one(g, 0)
    assert st == exp["status"]
    assert d.tolist() == exp["dist"] and h.tolist() == exp["hops"]
    _check_pred_finite(g, 0, d, h, p)


@pytest.mark.parametrize("seed", range(30))
def test_random_with_cycles(seed):
    rng = np.random.default_rng(seed)
    V = int(rng.integers(1, 3000))
    E = int(rng.integers(0, 6 * V + 1))
    g = synth.random_graph(V, E, seed=700 + seed, wlo=-3, whi=40)
    src = int(rng.integers(0, V))
    _compare(g, src, _one(g, src), check_pred=True)


@pytest.mark.parametrize("seed", range(6))
def test_random_with_cycles_cas_relaxation(seed):
    rng = np.random.default_rng(50 + seed)
    V = int(rng.integers(100, 3000))
    g = synth.random_graph(V, 5 * V, seed=900 + seed, wlo=-3, whi=40)
    t = bfq.make_tune(neg_cycle_mode=bfq.NEG_CYCLE_MARK, relax_atomic=bfq.RELAX_CAS)
    _compare(g, 0, gpu_util.sssp(g, 0, tune=t, want_pred=True), check_pred=True)


@pytest.mark.parametrize("seed", range(6))
def test_random_with_cycles_filtered_relaxation(seed):
    rng = np.random.default_rng(60 + seed)
    V = int(rng.integers(100, 3000))
    g = synth.random_graph(V, 9 * V, seed=920 + seed, wlo=-3, whi=40)
    t = bfq.make_tune(neg_cycle_mode=bfq.NEG_CYCLE_MARK, relax_atomic=bfq.RELAX_FILTERED)
    _compare(g, 0, gpu_util.sssp(g, 0, tune=t, want_pred=True), check_pred=True)


@pytest.mark.parametrize("seed", range(6))
def test_random_with_cycles_single_shot_queues(seed):
    """Minus-infinity marking with single-shot sub-queues (children published
    in the same round trips as the next dequeue)."""
    rng = np.random.default_rng(80 + seed)
    V = int(rng.integers(100, 3000))
    g = synth.random_graph(V, 5 * V, seed=950 + seed, wlo=-3, whi=40)
    t = bfq.make_tune(neg_cycle_mode=bfq.NEG_CYCLE_MARK, queue_form=bfq.QUEUE_FORM_SINGLE_SHOT)
    _compare(g, 0, gpu_util.sssp(g, 0, tune=t, want_pred=True), check_pred=True)


@pytest.mark.parametrize("seed", range(4))
def test_planted_cycles_grid(seed):
    base = synth.grid_graph(64, 64, seed=seed)
    g = synth.plant_negative_cycle(base, 3 + seed, seed=seed)
    assert _compare(g, 0, _one(g, 0), check_pred=True) == oracle.NEG_CYCLE


def test_planted_cycle_rmat_with_hubs():
    base = synth.workload_rmat(13)
    g = synth.plant_negative_cycle(base, 6, seed=11)
    s = int(g.sources[0])
    ost = _compare(g, s, _one(g, s), check_pred=True)
    assert ost == oracle.NEG_CYCLE


def test_two_copies_cycle_in_one():
    """The cycle sits in the second copy: from the first copy everything is
    finite, from the second the cycle's reach is minus infinity."""
    base = synth.grid_graph(40, 40, seed=5)
    V = base.V
    u = base.tails().astype(np.int64)
    v = base.col.astype(np.int64)
    rp, col, order = synth.csr_from_edges(2 * V, np.r_[u, u + V], np.r_[v, v + V],
                                          return_order=True)
    two = synth.Graph("two", rp, col, np.r_[base.w, base.w][order].astype(np.int32),
                      np.array([V], np.int32))
    g = synth.plant_negative_cycle(two, 5, seed=3, reachable_from=[V])
    h = gpu_util.create(g, MARK)
    try:
        for src in (0, V, 17, V + 3):
            ost = _compare(g, src, gpu_util.run(h, g.V, src, want_pred=True), check_pred=True)
            assert ost == (oracle.NEG_CYCLE if src >= V else oracle.OK)
    finally:
        bfq.bfq_graph_destroy(h)


def test_hub_on_a_negative_self_loop():
    """The source is a hub (its edges go through chunk sub-queues) with a
    negative self-loop: every vertex it reaches is minus infinity."""
    V = 20_000
    w = np.random.default_rng(1).integers(-1000, 1000, size=V - 1).astype(np.int32)
    star = synth.star_graph(V, w)
    rp = star.row_ptr.copy()
    rp[1:] += 1
    col = np.r_[0, star.col].astype(np.int32)
    ww = np.r_[-1, w].astype(np.int32)
    g = synth.Graph("star_loop", rp, col, ww, np.array([0], np.int32))
    st, d, h, p = _one(g, 0)
    assert st == bfq.NEG_CYCLE
    assert np.all(d == NEG_INF) and np.all(h == -2) and np.all(p == -1)
    _compare(g, 0, (st, d, h, p))


def test_range_is_reported_in_both_modes():
    w = np.array([-2 ** 30, -2 ** 30, -2 ** 30, 5], np.int32)
    g = synth.path_graph(5, w)
    for tune in (None, MARK):
        st, _, _, _ = gpu_util.sssp(g, 0, tune=tune)
        assert st == bfq.RANGE


def test_modes_switch_on_one_handle():
    base = synth.grid_graph(48, 48, seed=2)
    g = synth.plant_negative_cycle(base, 4, seed=9)
    h = gpu_util.create(g)
    try:
        t = bfq.bfq_graph_get_tune(h)
        for mode in (0, 1, 0, 1):
            t.neg_cycle_mode = mode
            bfq.bfq_graph_set_tune(h, t)
            st, d, hh, p = gpu_util.run(h, g.V, 0, want_pred=True)
            assert st == bfq.NEG_CYCLE
            if mode == 1:
                _compare(g, 0, (st, d, hh, p), check_pred=True)
            else:
                assert np.all(p == -1)
        bad = bfq.bfq_graph_get_tune(h)
        bad.neg_cycle_mode = 2
        with pytest.raises(bfq.BfqError):
            bfq.bfq_graph_set_tune(h, bad)
        # a clean graph on the same settings: plain labels
        t.neg_cycle_mode = 1
        bfq.bfq_graph_set_tune(h, t)
    finally:
        bfq.bfq_graph_destroy(h)
    clean = synth.workload_rmat(12)
    s = int(clean.sources[0])
    assert _compare(clean, s, _one(clean, s), check_pred=True) == oracle.OK
