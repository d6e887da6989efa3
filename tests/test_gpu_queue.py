"""The standalone Broker Queue kernels (per-thread BQ and BWD of Algorithm 1,
and the warp-aggregated form) checked against the queue model's properties:
gap-free tickets, FIFO by position, conservation, exact FULL/EMPTY counts."""
import numpy as np
import pytest

from oracle import broker_queue as bq
from paper_2608_21826_gb300 import bfq

pytestmark = pytest.mark.gpu
VARIANTS = [bfq.QUEUE_BQ, bfq.QUEUE_BWD, bfq.QUEUE_BQ_WARP, bfq.QUEUE_BWD_WARP]
VNAMES = {bfq.QUEUE_BQ: "bq", bfq.QUEUE_BWD: "bwd", bfq.QUEUE_BQ_WARP: "bq_warp",
          bfq.QUEUE_BWD_WARP: "bwd_warp"}
WARP = (bfq.QUEUE_BQ_WARP, bfq.QUEUE_BWD_WARP)


def _t(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def _empty(n, dtype):
    import torch
    return torch.full((n,), -9, dtype=dtype, device="cuda")


@pytest.mark.parametrize("variant", VARIANTS, ids=VNAMES.get)
@pytest.mark.parametrize("shape", [(64, 32), (108, 256), (216, 512), (7, 96)])
def test_enqdeq(variant, shape):
    import torch
    grid, block = shape
    n = 100_003
    items = np.random.default_rng(1).permutation(n).astype(np.int32) + 10
    q = bfq.bfq_queue_create(n, variant)
    try:
        epos = _empty(n, torch.int64)
        bfq.bfq_queue_enqueue(q, _t(items), epos, grid, block)
        out, dpos = _empty(n, torch.int32), _empty(n, torch.int64)
        bfq.bfq_queue_dequeue(q, out, dpos, grid, block)
        st, head, tail, count = bfq.bfq_queue_state(q)
        assert st == bfq.OK and head == tail == n and count == 0
        epos, dpos, out = epos.cpu().numpy(), dpos.cpu().numpy(), out.cpu().numpy()
        assert np.all(epos >= 0) and np.all(dpos >= 0)
        err = bq.check_fifo_positions(items, epos, out, dpos)
        assert err is None, err
    finally:
        bfq.bfq_queue_destroy(q)


@pytest.mark.parametrize("variant", VARIANTS, ids=VNAMES.get)
def test_full_and_empty_counts(variant):
    import torch
    N = 4096
    q = bfq.bfq_queue_create(N, variant)
    try:
        n = 3 * N + 17
        items = np.arange(n, dtype=np.int32)
        epos = _empty(n, torch.int64)
        bfq.bfq_queue_enqueue(q, _t(items), epos, 108, 256)
        epos = epos.cpu().numpy()
        ok = epos >= 0
        assert ok.sum() == N                                  # exactly N granted
        m = N + 999
        out, dpos = _empty(m, torch.int32), _empty(m, torch.int64)
        bfq.bfq_queue_dequeue(q, out, dpos, 108, 256)
        dpos, out = dpos.cpu().numpy(), out.cpu().numpy()
        assert (dpos >= 0).sum() == N                         # exactly N taken
        err = bq.check_fifo_positions(items[ok], epos[ok], out[dpos >= 0], dpos[dpos >= 0])
        assert err is None, err
        st, head, tail, count = bfq.bfq_queue_state(q)
        assert st == bfq.OK and count == 0 and head == tail == N
    finally:
        bfq.bfq_queue_destroy(q)


@pytest.mark.parametrize("variant", VARIANTS, ids=VNAMES.get)
def test_wraparound_many_laps(variant):
    import torch
    N = 1000 if variant not in WARP else 1024
    q = bfq.bfq_queue_create(N, variant)
    try:
        for lap in range(7):
            items = (np.arange(N, dtype=np.int32) + lap * 100_000)
            epos = _empty(N, torch.int64)
            bfq.bfq_queue_enqueue(q, _t(items), epos, 32, 64)
            out, dpos = _empty(N, torch.int32), _empty(N, torch.int64)
            bfq.bfq_queue_dequeue(q, out, dpos, 32, 64)
            e, d, o = epos.cpu().numpy(), dpos.cpu().numpy(), out.cpu().numpy()
            assert np.all(e >= 0) and np.all(d >= 0)
            err = bq.check_fifo_positions(items, e, o, d, base=lap * N)
            assert err is None, err
    finally:
        bfq.bfq_queue_destroy(q)


@pytest.mark.parametrize("variant", VARIANTS, ids=VNAMES.get)
@pytest.mark.parametrize("grid", [2, 64, 216])
def test_mixed(variant, grid):
    import torch
    n_enq, n_deq = 150_000, 150_000
    cap = 1 << 18
    items = np.arange(n_enq, dtype=np.int32) * 3 + 1
    q = bfq.bfq_queue_create(cap, variant)
    try:
        epos = _empty(n_enq, torch.int64)
        out, dpos = _empty(n_deq, torch.int32), _empty(n_deq, torch.int64)
        bfq.bfq_queue_mixed(q, _t(items), out, epos, dpos, grid, 256)
        e, d, o = epos.cpu().numpy(), dpos.cpu().numpy(), out.cpu().numpy()
        assert np.all(e >= 0)                                  # capacity never reached
        got = d >= 0
        err = bq.check_fifo_positions(items, e, o[got], d[got])
        assert err is None, err
        # drain the rest: every item comes out exactly once overall
        rest = n_enq - int(got.sum())
        out2, dpos2 = _empty(rest + 5, torch.int32), _empty(rest + 5, torch.int64)
        bfq.bfq_queue_dequeue(q, out2, dpos2, 64, 256)
        d2, o2 = dpos2.cpu().numpy(), out2.cpu().numpy()
        assert (d2 >= 0).sum() == rest
        all_items = np.concatenate([o[got], o2[d2 >= 0]])
        assert np.array_equal(np.sort(all_items), np.sort(items))
        st, head, tail, count = bfq.bfq_queue_state(q)
        assert st == bfq.OK and count == 0 and head == tail == n_enq
    finally:
        bfq.bfq_queue_destroy(q)


@pytest.mark.parametrize("mode", [0, 1, 2])
def test_atomic_bench_counts_every_operation(mode):
    n = 1 << 20
    ms, tot = bfq.bfq_atomic_bench(mode, n, 152, 256)
    assert tot == n and ms > 0


def test_atomic_bench_rejects_bad_arguments():
    for args in ((3, 1024, 8, 64), (0, 1024, 8, 48), (2, 1000, 8, 64), (0, -1, 8, 64)):
        with pytest.raises(bfq.BfqError):
            bfq.bfq_atomic_bench(*args)


@pytest.mark.parametrize("mode", [0, 1])
def test_relax_bench_runs_and_counts(mode):
    """The relaxation-pattern microbenchmark touches every edge once: with
    labels starting at infinity, at least one edge per distinct label
    lowers it, and no more edges than there are do."""
    n, L = 1 << 20, 1 << 16
    ms, low = bfq.bfq_relax_bench(mode, n, L, 152 * 4, 256)
    assert ms > 0 and L // 2 <= low <= n
    for bad in ((mode, 0, L, 8, 64), (2, n, L, 8, 64), (-1, n, L, 8, 64)):
        with pytest.raises(bfq.BfqError):
            bfq.bfq_relax_bench(*bad)
