"""Broker Queue model -- TEST INFRASTRUCTURE ONLY.

Two things live here, both written from Sec. III-A and Algorithm 1:

``FifoSpec``
    The sequential specification a linearizable bounded FIFO must match:
    capacity N, enqueue fails with FULL when N items are held, dequeue fails
    with EMPTY when none are held, otherwise first in, first out.

``BrokerQueueSim``
    The Broker Queue's shared state (ring, per-slot tickets, head, tail and the
    broker count) and its operations written as Python generators that yield
    after every access to shared state, so that a seeded scheduler can
    interleave many simulated threads.  Steps follow Algorithm 1 in the paper's
    order; the readings taken where the listing is garbled are:

    * ENSURE_DEQUEUE: a fetch-and-decrement of count that returns a value > 0
      grants the dequeue (the listing never sets the grant); otherwise the
      decrement is undone and count re-read -- the mirror of ENSURE_ENQUEUE.
    * READ_DATA releases the slot with ticket 2*(Pos//N + 1), the even ticket
      the enqueuer of the next lap waits for (printed as "2*(Pos + N/N)").
    * head/tail are unbounded counters, so the Full test
      "N <= tail-head < N + MaxThreads/2" and the Empty test
      "N + MaxThreads/2 <= tail-head-1", which rely on 32-bit unsigned
      wrap-around, become tail-head >= N and tail-head <= 0.
    * the ring never overwrites a held item: the broker keeps count <= N.

    ``bwd=True`` gives the Broker Work Distributor variant: the ensure step is
    tried once and its failure is final (Sec. III-A, last paragraph).

``check_fifo_positions``
    The property the GPU queue kernels are checked against: an item dequeued
    at ticket position p is exactly the item enqueued at position p, positions
    form a prefix without gaps or repeats, and no item is lost or duplicated.
"""
from __future__ import annotations

import collections
import random

FULL = "full"
EMPTY = "empty"
OK = "ok"


class FifoSpec:
    """Sequential bounded FIFO (the object Algorithm 1 linearizes to)."""

    def __init__(self, capacity: int):
        self.capacity = capacity
        self.items = collections.deque()

    def enqueue(self, x):
        if len(self.items) >= self.capacity:
            return FULL
        self.items.append(x)
        return OK

    def dequeue(self):
        if not self.items:
            return EMPTY, None
        return OK, self.items.popleft()


class BrokerQueueSim:
    """Shared state of Algorithm 1 plus its operations as step generators."""

    def __init__(self, capacity: int, release_ticket=None):
        self.N = capacity
        # INITIALIZE: counters, tickets and ring start at zero
        self.head = 0
        self.tail = 0
        self.count = 0
        self.tickets = [0] * capacity
        self.ring = [0] * capacity
        # the slot-release ticket of READ_DATA; overridable to show that the
        # literal printed form stalls at the first wrap-around
        self.release_ticket = release_ticket or (lambda pos, n: 2 * (pos // n + 1))

    # --- atomics: each is one step -------------------------------------------
    def _fetch_add(self, field: str, v: int) -> int:
        old = getattr(self, field)
        setattr(self, field, old + v)
        return old

    # --- Algorithm 1 -----------------------------------------------------------
    def _wait_ticket(self, slot: int, expected: int):
        while self.tickets[slot] != expected:
            yield "wait"

    def _ensure_enqueue(self):
        num = self.count
        yield "step"
        while num < self.N:
            old = self._fetch_add("count", 1)
            yield "step"
            if old < self.N:
                return True
            num = self._fetch_add("count", -1) - 1
            yield "step"
        return False

    def _ensure_dequeue(self):
        num = self.count
        yield "step"
        while num > 0:
            old = self._fetch_add("count", -1)
            yield "step"
            if old > 0:
                return True
            self._fetch_add("count", 1)
            yield "step"
            num = self.count
            yield "step"
        return False

    def _put_data(self, item, log):
        pos = self._fetch_add("tail", 1)
        yield "step"
        slot, lap = pos % self.N, pos // self.N
        yield from self._wait_ticket(slot, 2 * lap)
        self.ring[slot] = item
        yield "step"
        self.tickets[slot] = 2 * lap + 1
        yield "step"
        log.append(pos)

    def _read_data(self, log):
        pos = self._fetch_add("head", 1)
        yield "step"
        slot, lap = pos % self.N, pos // self.N
        yield from self._wait_ticket(slot, 2 * lap + 1)
        item = self.ring[slot]
        yield "step"
        self.tickets[slot] = self.release_ticket(pos, self.N)
        yield "step"
        log.append(pos)
        return item

    def enqueue(self, item, bwd: bool = False):
        """Generator for one ENQUEUE; returns (OK, pos) or (FULL, None)."""
        while True:
            ensured = yield from self._ensure_enqueue()
            if ensured:
                break
            if bwd:
                return FULL, None
            if self.tail - self.head >= self.N:
                return FULL, None
            yield "step"
        log = []
        yield from self._put_data(item, log)
        return OK, log[0]

    def dequeue(self, bwd: bool = False):
        """Generator for one DEQUEUE; returns (OK, (item, pos)) or (EMPTY, None)."""
        while True:
            ensured = yield from self._ensure_dequeue()
            if ensured:
                break
            if bwd:
                return EMPTY, None
            if self.tail - self.head <= 0:
                return EMPTY, None
            yield "step"
        log = []
        item = yield from self._read_data(log)
        return OK, (item, log[0])


def run_interleaved(q: BrokerQueueSim, ops, seed: int, max_steps: int = 2_000_000):
    """Run generators ``ops`` (list of (name, generator)) under a seeded random
    scheduler.  Returns the list of results in op order, or raises
    ``RuntimeError('stalled')`` if every live thread is waiting on a ticket or
    the step budget runs out."""
    rng = random.Random(seed)
    live = {i: g for i, (_, g) in enumerate(ops)}
    results = [None] * len(ops)
    waiting_rounds = 0
    steps = 0
    while live:
        steps += 1
        if steps > max_steps:
            raise RuntimeError("stalled")
        i = rng.choice(list(live))
        try:
            r = next(live[i])
            if r == "wait":
                waiting_rounds += 1
                if waiting_rounds > 50 * (len(live) + 1) ** 2:
                    raise RuntimeError("stalled")
            else:
                waiting_rounds = 0
        except StopIteration as stop:
            results[i] = stop.value
            del live[i]
            waiting_rounds = 0
    return results


def check_fifo_positions(enq_items, enq_pos, deq_items, deq_pos, base: int = 0):
    """Position-based FIFO/linearizability check used on GPU queue output.

    enq_items/enq_pos: successful enqueues with the tail ticket each took.
    deq_items/deq_pos: successful dequeues with the head ticket each took.
    Tickets handed out are a gap-free range starting at ``base``; a dequeue
    at position p returns the item enqueued at p.  Returns an error string or
    None when everything holds."""
    enq_pos = [int(p) for p in enq_pos]
    deq_pos = [int(p) for p in deq_pos]
    if sorted(enq_pos) != list(range(base, base + len(enq_pos))):
        return "enqueue positions are not a gap-free range"
    if sorted(deq_pos) != list(range(base, base + len(deq_pos))):
        return "dequeue positions are not a gap-free range"
    if len(deq_pos) > len(enq_pos):
        return "more dequeues than enqueues"
    at = dict(zip(enq_pos, (int(x) for x in enq_items)))
    for item, p in zip(deq_items, deq_pos):
        if at[p] != int(item):
            return f"position {p}: dequeued {int(item)}, enqueued {at[p]}"
    return None
