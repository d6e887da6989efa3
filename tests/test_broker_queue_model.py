"""Pins for the Broker Queue model (Algorithm 1): sequential runs equal the
bounded-FIFO specification; seeded interleavings of many simulated threads
conserve items and keep FIFO order by ticket position; the garbled slot
release printed in READ_DATA stalls at the first wrap-around, which is why the
model reads it as 2*(Pos//N + 1)."""
import random

import pytest

from oracle import broker_queue as bq


def _run_one(gen):
    try:
        while True:
            assert next(gen) != "wait", "sequential run must never wait"
    except StopIteration as stop:
        return stop.value


@pytest.mark.parametrize("bwd", [False, True])
@pytest.mark.parametrize("seed", range(10))
def test_sequential_equals_spec(seed, bwd):
    rng = random.Random(seed)
    N = rng.choice([1, 2, 3, 4, 8])
    q = bq.BrokerQueueSim(N)
    spec = bq.FifoSpec(N)
    for step in range(300):
        if rng.random() < 0.55:
            x = rng.randrange(1000)
            r, _ = _run_one(q.enqueue(x, bwd=bwd))
            assert r == spec.enqueue(x)
        else:
            r, got = _run_one(q.dequeue(bwd=bwd))
            rs, xs = spec.dequeue()
            assert r == rs
            if r == bq.OK:
                assert got[0] == xs


@pytest.mark.parametrize("seed", range(12))
def test_interleaved_enqdeq_and_mixed(seed):
    """Enqueues and dequeues run concurrently in a seeded random interleaving:
    counters stay consistent, tickets form gap-free ranges and every dequeue
    returns the item enqueued at its ticket position."""
    rng = random.Random(seed)
    N = rng.choice([2, 4, 8, 16])
    q = bq.BrokerQueueSim(N)
    n_enq = rng.randrange(1, 40)
    n_deq = rng.randrange(1, 40)
    ops = [("enq", 1000 + i, q.enqueue(1000 + i)) for i in range(n_enq)]
    ops += [("deq", None, q.dequeue()) for _ in range(n_deq)]
    rng.shuffle(ops)
    res = bq.run_interleaved(q, [(k, g) for k, _, g in ops], seed)
    enq_items, enq_pos, deq_items, deq_pos = [], [], [], []
    for (kind, item, _), (status, val) in zip(ops, res):
        if status != bq.OK:
            continue
        if kind == "enq":
            enq_items.append(item)
            enq_pos.append(val)
        else:
            deq_items.append(val[0])
            deq_pos.append(val[1])
    assert q.tail - q.head == len(enq_pos) - len(deq_pos)
    assert q.count == q.tail - q.head
    err = bq.check_fifo_positions(enq_items, enq_pos, deq_items, deq_pos)
    assert err is None, err


def test_interleaved_items_follow_positions():
    """Enqueue distinct items concurrently, then dequeue concurrently: the item
    at each dequeue position is the one enqueued at that position."""
    for seed in range(8):
        N = 8
        q = bq.BrokerQueueSim(N)
        items = list(range(500, 512))
        enq_ops = [("enq", q.enqueue(x)) for x in items]
        res = bq.run_interleaved(q, enq_ops, seed)
        pos_of = {x: r[1] for x, r in zip(items, res) if r[0] == bq.OK}
        assert len(pos_of) == N                  # capacity reached, rest FULL
        assert sum(r[0] == bq.FULL for r in res) == len(items) - N
        deq_ops = [("deq", q.dequeue()) for _ in range(12)]
        dres = bq.run_interleaved(q, deq_ops, seed + 100)
        got = [r[1] for r in dres if r[0] == bq.OK]
        assert len(got) == N
        err = bq.check_fifo_positions(list(pos_of), list(pos_of.values()),
                                      [x for x, _ in got], [p for _, p in got])
        assert err is None, err


def test_printed_release_ticket_stalls_after_wrap():
    """READ_DATA as printed releases the slot with 2*(Pos + N/N) = 2*(Pos+1);
    the enqueuer of the next lap waits for 2*(Pos//N + 1).  The two agree only
    for Pos = 0, so the second lap stalls on slot 1."""
    N = 4
    q = bq.BrokerQueueSim(N, release_ticket=lambda pos, n: 2 * (pos + n // n))
    for x in range(N):
        r, _ = bq.run_interleaved(q, [("e", q.enqueue(x))], 0)[0]
        assert r == bq.OK
    for _ in range(N):
        r, _ = bq.run_interleaved(q, [("d", q.dequeue())], 0)[0]
        assert r == bq.OK
    # second lap: slot 1's ticket is 4, the enqueuer wants 2
    with pytest.raises(RuntimeError, match="stalled"):
        for x in range(N):
            bq.run_interleaved(q, [("e", q.enqueue(x))], 0, max_steps=10_000)
    # the model's reading completes many laps
    q2 = bq.BrokerQueueSim(N)
    for lap in range(5):
        for x in range(N):
            assert bq.run_interleaved(q2, [("e", q2.enqueue(x))], 0)[0][0] == bq.OK
        for x in range(N):
            r, (item, _) = bq.run_interleaved(q2, [("d", q2.dequeue())], 0)[0]
            assert r == bq.OK and item == x


def test_check_fifo_positions_rejects_mismatch():
    assert bq.check_fifo_positions([1, 2], [0, 1], [2, 1], [1, 0]) is None
    assert bq.check_fifo_positions([1, 2], [0, 1], [1, 2], [1, 0]) is not None
    assert bq.check_fifo_positions([1, 2], [0, 2], [], []) is not None
    assert bq.check_fifo_positions([1], [0], [1, 1], [0, 1]) is not None


def _warp_run(form, seed, n_warps=12, N=16, k_max=8, rounds=3):
    """Warps alternately enqueue and dequeue batches of up to k_max items,
    interleaved at random; returns (results, ops) or raises on a stall."""
    rng = random.Random(seed)
    q = bq.WarpQueueSim(N, form)
    ops = []
    nxt = 0
    for w in range(n_warps):
        for r in range(rounds):
            if (w + r) % 2 == 0:
                k = rng.randint(1, k_max)
                ops.append(("enq", q.enqueue_warp(list(range(nxt, nxt + k)))))
                nxt += k
            else:
                ops.append(("deq", q.dequeue_warp(rng.randint(1, k_max))))
    rng.shuffle(ops)
    return q, ops, bq.run_interleaved(q, ops, seed)


@pytest.mark.parametrize("form", ["exact", "split"])
@pytest.mark.parametrize("seed", range(40))
def test_warp_forms_interleaved(form, seed):
    """The warp-aggregated forms: no wait is ever stranded (the run ends),
    every dequeued item was enqueued at the same ticket position, positions
    are gap-free, and the counters end consistent with the ring."""
    q, ops, res = _warp_run(form, seed)
    enq_items, enq_pos, deq_items, deq_pos = [], [], [], []
    for (kind, _), out in zip(ops, res):
        for item, p in out:
            (enq_items if kind == "enq" else deq_items).append(item)
            (enq_pos if kind == "enq" else deq_pos).append(p)
    assert bq.check_fifo_positions(enq_items, enq_pos, deq_items, deq_pos) is None
    held = len(enq_pos) - len(deq_pos)
    assert q.tail - q.head == held
    if form == "exact":
        assert q.count == held
    else:
        assert q.avail == held and q.free == q.N - held


def test_warp_forms_drain_what_they_hold():
    """After concurrent traffic, every item still held comes out, in ticket
    order, for both forms."""
    for form in ("exact", "split"):
        q, ops, res = _warp_run(form, 5)
        left = q.tail - q.head
        out = bq.run_interleaved(q, [("deq", q.dequeue_warp(q.N))], 0)[0]
        assert len(out) == left
        assert [p for _, p in out] == list(range(q.head - left, q.head))


def test_naive_single_count_can_strand_a_dequeuer():
    """One count moved by fetch-add, the surplus added back afterwards: in
    the window an enqueuer's withdrawn surplus is visible to dequeuers, a
    dequeuer is granted items that no enqueuer will ever publish, and its
    ticket wait never ends even after everyone else has finished.  The
    single-shot form keeps two counters for this reason; both proper forms
    end the same schedule."""
    for form in ("naive", "split", "exact"):
        q = bq.WarpQueueSim(4, form)
        bq.run_interleaved(q, [("enq", q.enqueue_warp([1, 2, 3, 4]))], 0)   # full
        big = q.enqueue_warp([10, 11, 12, 13])     # no room: must withdraw
        next(big)                                  # its reservation step
        thief = q.dequeue_warp(8)
        next(thief)                                # its reservation, before the withdrawal
        if form == "naive":
            with pytest.raises(RuntimeError, match="stalled"):
                bq.run_interleaved(q, [("deq", thief), ("enq", big)], 0)
        else:
            res = bq.run_interleaved(q, [("deq", thief), ("enq", big)], 0)
            assert [x for x, _ in res[0]] == [1, 2, 3, 4] and res[1] == []


def _ring_run(seed, C, n_items=60, n_fill=3, n_take=3, racy=False, max_steps=2_000_000):
    """Fillers publish n_items in batches; takers drain them.  A filler
    reserves room first (at most C items filled or reserved and not taken),
    as the in-queue flag guarantees in the kernel."""
    rng = random.Random(seed)
    q = bq.CtaRingSim(C)
    state = {"live": 0, "next": 0, "taken": []}

    def filler():
        while True:
            # pick a batch and reserve room in one step (no yield in between)
            if state["next"] >= n_items:
                return
            k = min(rng.randint(1, max(1, C // 2)), n_items - state["next"])
            if state["live"] + k > C:
                yield "wait"
                continue
            items = list(range(state["next"], state["next"] + k))
            state["next"] += k
            state["live"] += k
            yield from q.fill(items)

    def taker(kmax):
        while len(state["taken"]) < n_items:
            got = yield from q.take(kmax, racy)
            state["taken"].extend(got)
            state["live"] -= len(got)
            if not got:
                yield "wait"

    ops = [("fill", filler()) for _ in range(n_fill)] + \
          [("take", taker(rng.randint(1, 4))) for _ in range(n_take)]
    bq.run_interleaved(q, ops, seed, max_steps=max_steps)
    return q, state


@pytest.mark.parametrize("C", [4, 8, 16])
@pytest.mark.parametrize("seed", range(30))
def test_cta_ring_conserves_items(C, seed):
    """The single-CTA ring under seeded interleavings: every published item
    is taken exactly once, no wait is stranded, and the tickets end even."""
    q, st = _ring_run(seed, C)
    assert sorted(st["taken"]) == list(range(60))
    assert q.head == q.tail == 60 and all(x is None for x in q.slots)


def test_cta_ring_lap_swaps_are_exercised():
    """Some schedules let two tickets a lap apart meet on one slot, so a
    taker gets the item filled at the other ticket; items are still
    conserved (checked above), and such schedules do occur."""
    swaps = 0
    for seed in range(60):
        q, _ = _ring_run(seed, 4, n_items=80, n_fill=4, n_take=4)
        swaps += sum(q.fill_ticket[x] != q.take_ticket[x] for x in range(80))
    assert swaps > 0


def test_cta_ring_racy_take_breaks_conservation():
    """Reading a slot and emptying it in two steps (no exchange): two takers
    a lap apart can take the same item, and the filler's next item is then
    lost or a taker waits forever.  The kernel takes with one exchange."""
    broken = 0
    for seed in range(80):
        try:
            _, st = _ring_run(seed, 4, n_items=80, n_fill=4, n_take=4, racy=True,
                              max_steps=50_000)
            broken += sorted(st["taken"]) != list(range(80))
        except RuntimeError:                       # a stranded taker
            broken += 1
        if broken:
            break
    assert broken > 0
