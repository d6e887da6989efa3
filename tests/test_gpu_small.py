"""Single-CTA path of bfq_sssp (small_path): the labels, recorded edges and
vertex queue in one CTA's shared memory.  Every result is compared with the
oracle element by element, as for the persistent kernel."""
import numpy as np
import pytest

import oracle
from paper_2608_21826_gb300 import bfq, synth

from tests import gpu_util, helpers

pytestmark = pytest.mark.gpu

ON = bfq.make_tune(small_path=bfq.SMALL_PATH_ON)
OFF = bfq.make_tune(small_path=bfq.SMALL_PATH_OFF)


def _compare(g, src, res, check_pred=False):
    st, d, h, p = res
    ost, od, oh, _ = oracle.spfa(g.row_ptr, g.col, g.w, src)
    assert st == ost, (st, ost)
    if ost == oracle.OK:
        bad = np.nonzero(d != od)[0]
        assert bad.size == 0, f"{bad.size} dist mismatches, first {bad[:5]}"
        assert np.array_equal(h, oh), "hops mismatch"
        if check_pred:
            assert oracle.check_pred(g.row_ptr, g.col, g.w, src, d, p)
    return ost


def _on_small_path(h):
    s = bfq.bfq_get_stats(h)
    return s["grid"] == 1 and s["block"] in (512, 1024)


def _run_small(g, src, tune=ON, want_pred=True):
    h = gpu_util.create(g, tune)
    try:
        res = gpu_util.run(h, g.V, src, want_pred)
        assert _on_small_path(h)
        return res
    finally:
        bfq.bfq_graph_destroy(h)


@pytest.mark.parametrize("path", helpers.golden_files(), ids=lambda p: p.split("/")[-1])
def test_golden(path):
    g, exp = helpers.load_golden(path)
    st, d, h, p = _run_small(g, 0)
    assert st == exp["status"]
    if "dist" in exp:
        assert d.tolist() == exp["dist"] and h.tolist() == exp["hops"]
        assert oracle.check_pred(g.row_ptr, g.col, g.w, 0, d, p)


ON512 = bfq.make_tune(small_path=bfq.SMALL_PATH_ON, small_threads=512)


@pytest.mark.parametrize("tune", [ON, ON512], ids=["1024", "512"])
@pytest.mark.parametrize("seed", range(24))
def test_random_with_cycles(seed, tune):
    rng = np.random.default_rng(700 + seed)
    V = int(rng.integers(1, 8000))
    E = int(rng.integers(0, 12 * V + 1))
    g = synth.random_graph(V, E, seed=1700 + seed, wlo=-3, whi=40)
    _compare(g, 0, _run_small(g, 0, tune), check_pred=True)


@pytest.mark.parametrize("seed", range(8))
def test_random_potential(seed):
    rng = np.random.default_rng(900 + seed)
    V = int(rng.integers(2, 8000))
    g = synth.random_potential_graph(V, int(rng.integers(V, 10 * V)), seed=seed)
    _compare(g, 0, _run_small(g, 0), check_pred=True)


@pytest.mark.parametrize("tune", [None, ON512], ids=["auto", "512"])
def test_grid4k_all_sources_and_auto(tune):
    """The 64x64 grid (the default path for it) from every source of the
    workload, against the oracle."""
    g = synth.workload_grid4k()
    h = gpu_util.create(g, tune)
    try:
        for s in g.sources:
            _compare(g, int(s), gpu_util.run(h, g.V, int(s), want_pred=True), check_pred=True)
            assert _on_small_path(h)
    finally:
        bfq.bfq_graph_destroy(h)


@pytest.mark.parametrize("tune", [ON, ON512], ids=["1024", "512"])
def test_planted_cycle_found_fast(tune):
    g = synth.plant_negative_cycle(synth.grid_graph(60, 60, seed=3), 5, seed=4)
    h = gpu_util.create(g, tune)
    try:
        st, _, _, _ = gpu_util.run(h, g.V, 0)
        assert st == bfq.NEG_CYCLE
        assert _on_small_path(h)
        assert bfq.bfq_get_stats(h)["kernel_ms"] < 50.0
    finally:
        bfq.bfq_graph_destroy(h)


def test_hub_path_and_degenerate_graphs():
    w = np.random.default_rng(1).integers(-1000, 1000, size=7999).astype(np.int32)
    st, d, h, p = _run_small(synth.star_graph(8000, w), 0)
    assert st == bfq.OK and np.array_equal(d[1:], w) and np.all(p[1:] == 0)
    pw = np.random.default_rng(2).integers(-5, 9, size=7999).astype(np.int32)
    st, d, h, _ = _run_small(synth.path_graph(8000, pw), 0)
    assert st == bfq.OK and np.array_equal(d, np.r_[0, np.cumsum(pw)])
    assert np.array_equal(h, np.arange(8000))
    one = synth.Graph("one", np.array([0, 0], np.int32), np.zeros(0, np.int32),
                      np.zeros(0, np.int32), np.array([0], np.int32))
    st, d, h, p = _run_small(one, 0)
    assert st == bfq.OK and d.tolist() == [0] and h.tolist() == [0] and p.tolist() == [-1]
    iso = synth.random_graph(500, 0, seed=3)
    st, d, h, _ = _run_small(iso, 7)
    assert st == bfq.OK and d[7] == 0 and np.all(np.delete(d, 7) == 2 ** 31 - 1)


def test_range_reported():
    w = np.array([-2 ** 30, -2 ** 30, -2 ** 30, 5], np.int32)
    st, _, _, _ = _run_small(synth.path_graph(5, w), 0, want_pred=False)
    assert st == bfq.RANGE


def test_paths_alternate_on_one_handle():
    """Small and persistent runs share a handle: a cycle run on either path
    leaves nothing stale for the other."""
    clean = synth.random_potential_graph(3000, 20000, seed=5)
    cyc = synth.plant_negative_cycle(synth.grid_graph(40, 40, seed=6), 5, seed=7)
    for g in (clean, cyc):
        h = gpu_util.create(g, ON)
        try:
            t = bfq.bfq_graph_get_tune(h)
            for mode in (bfq.SMALL_PATH_ON, bfq.SMALL_PATH_OFF, bfq.SMALL_PATH_ON,
                         bfq.SMALL_PATH_OFF):
                t.small_path = mode
                bfq.bfq_graph_set_tune(h, t)
                _compare(g, 0, gpu_util.run(h, g.V, 0, want_pred=True), check_pred=True)
                assert _on_small_path(h) == (mode == bfq.SMALL_PATH_ON)
        finally:
            bfq.bfq_graph_destroy(h)


def test_dirty_queues_cleared_across_paths():
    """A persistent run that stops on a negative cycle leaves its sub-queues
    dirty; a clean single-CTA run in between must not hide that from the
    next persistent run (two grid copies, the cycle in the second)."""
    base = synth.grid_graph(40, 40, seed=5)
    V = base.V
    u = base.tails().astype(np.int64)
    v = base.col.astype(np.int64)
    rp, col, order = synth.csr_from_edges(2 * V, np.r_[u, u + V], np.r_[v, v + V],
                                          return_order=True)
    two = synth.Graph("two", rp, col, np.r_[base.w, base.w][order].astype(np.int32),
                      np.array([V], np.int32))
    g = synth.plant_negative_cycle(two, 5, seed=3, reachable_from=[V])
    h = gpu_util.create(g, OFF)
    try:
        t = bfq.bfq_graph_get_tune(h)
        seq = [(bfq.SMALL_PATH_OFF, V), (bfq.SMALL_PATH_ON, 0), (bfq.SMALL_PATH_OFF, 3),
               (bfq.SMALL_PATH_ON, V + 9), (bfq.SMALL_PATH_OFF, 11), (bfq.SMALL_PATH_OFF, V),
               (bfq.SMALL_PATH_ON, 5), (bfq.SMALL_PATH_ON, 6), (bfq.SMALL_PATH_OFF, 0)]
        for mode, src in seq:
            t.small_path = mode
            bfq.bfq_graph_set_tune(h, t)
            ost = _compare(g, src, gpu_util.run(h, g.V, src, want_pred=True), check_pred=True)
            assert ost == (oracle.NEG_CYCLE if src >= V else oracle.OK)
            assert _on_small_path(h) == (mode == bfq.SMALL_PATH_ON)
    finally:
        bfq.bfq_graph_destroy(h)


def test_falls_back_when_it_does_not_fit_or_marks():
    big = synth.random_potential_graph(40_000, 120_000, seed=8)
    h = gpu_util.create(big, ON)
    try:
        _compare(big, 0, gpu_util.run(h, big.V, 0))
        assert not _on_small_path(h)
    finally:
        bfq.bfq_graph_destroy(h)
    g = synth.plant_negative_cycle(synth.grid_graph(30, 30, seed=2), 4, seed=3)
    t = bfq.make_tune(small_path=bfq.SMALL_PATH_ON, neg_cycle_mode=bfq.NEG_CYCLE_MARK)
    h = gpu_util.create(g, t)
    try:
        st, d, _, _ = gpu_util.run(h, g.V, 0)
        assert st == bfq.NEG_CYCLE and not _on_small_path(h)
        ost, od, _ = oracle.spfa_neg_inf(g.row_ptr, g.col, g.w, 0)
        assert np.array_equal(d, od)
    finally:
        bfq.bfq_graph_destroy(h)


def test_timeout_leaves_context_usable():
    g = synth.grid_graph(20, 20, seed=1)
    h = gpu_util.create(g, bfq.make_tune(small_path=bfq.SMALL_PATH_ON, time_limit_ms=30,
                                         test_phantom_items=1))
    try:
        with pytest.raises(bfq.BfqError) as e:
            gpu_util.run(h, g.V, 0)
        assert e.value.code == bfq.ERR_TIMEOUT
        t = bfq.bfq_graph_get_tune(h)
        t.test_phantom_items = 0
        bfq.bfq_graph_set_tune(h, t)
        _compare(g, 0, gpu_util.run(h, g.V, 0, want_pred=True), check_pred=True)
    finally:
        bfq.bfq_graph_destroy(h)


def test_autotune_tries_both_paths():
    g = synth.workload_grid4k()
    h = gpu_util.create(g)
    try:
        t = bfq.bfq_autotune(h, [int(s) for s in g.sources[:2]])
        assert t.small_path in (bfq.SMALL_PATH_AUTO, bfq.SMALL_PATH_ON, bfq.SMALL_PATH_OFF)
        _compare(g, int(g.sources[0]), gpu_util.run(h, g.V, int(g.sources[0])))
    finally:
        bfq.bfq_graph_destroy(h)


def test_async_queries_back_to_back_on_one_stream():
    """Queries enqueued with bfq_sssp_async one after another on a stream
    (each into its own buffers, statuses on the device), on both block
    sizes: every result matches the oracle."""
    import torch
    g = synth.grid_graph(50, 50, seed=9)
    srcs = [0, 17, 1234, 2499, 600, 901]
    for tune in (ON, ON512):
        h = gpu_util.create(g, tune)
        try:
            s = torch.cuda.Stream()
            dist = [torch.full((g.V,), -7, dtype=torch.int32, device="cuda") for _ in srcs]
            hops = [torch.full((g.V,), -7, dtype=torch.int32, device="cuda") for _ in srcs]
            st = torch.full((len(srcs),), -99, dtype=torch.int32, device="cuda")
            for i, src in enumerate(srcs):
                bfq.bfq_sssp_async(h, src, dist[i], hops[i], None, st[i:i + 1], s)
            s.synchronize()
            assert _on_small_path(h)
            for i, src in enumerate(srcs):
                _compare(g, src, (int(st[i]), dist[i].cpu().numpy(), hops[i].cpu().numpy(), None))
        finally:
            bfq.bfq_graph_destroy(h)
