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

``WarpQueueSim``
    The warp-aggregated forms the GPU worklist uses (exact-count and
    single-shot split counters) as step generators, for the same seeded
    interleavings.

``CtaRingSim``
    The single-CTA path's shared-memory ring (take and fill tickets, slots
    filled by compare-and-swap from empty and taken by exchange) as step
    generators.

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


class WarpQueueSim:
    """Warp-aggregated forms of the Broker Queue (one reservation and one
    ticket range for up to 32 items), the forms the GPU worklist uses; the
    same ring, slot tickets and head/tail as BrokerQueueSim.

    ``form="exact"``: one broker count moved by compare-and-swap to an exact
    value (retried while the count changes under it), then the ticket range.
    Every ticket wait is then on an operation already granted.

    ``form="split"``: single-shot reservations (the BWD idea of Sec. III-A,
    warp-aggregated): two counters, ``free`` (places an enqueuer may take,
    initially N) and ``avail`` (items a dequeuer may take).  An enqueuer
    fetch-subtracts k from free, keeps min(max(old, 0), k) and adds the
    surplus back; takes its tail tickets; publishes the items; then adds its
    grant to avail.  A dequeuer does the same on avail, takes head tickets, reads and
    releases the slots, then adds its grant to free.  A transient surplus
    only understates a counter, and each counter is read by one side only,
    so no grant exceeds what the other side has already provided; no retry.

    ``form="naive"``: one count moved by fetch-add with the surplus added
    back -- kept to show that it can strand a waiter (a dequeuer granted an
    item that the enqueuer then withdraws)."""

    def __init__(self, capacity: int, form: str = "exact"):
        assert form in ("exact", "split", "naive")
        self.N = capacity
        self.form = form
        self.head = 0
        self.tail = 0
        self.count = 0          # exact / naive
        self.free = capacity    # split
        self.avail = 0          # split
        self.tickets = [0] * capacity
        self.ring = [0] * capacity

    def _fetch_add(self, field: str, v: int) -> int:
        old = getattr(self, field)
        setattr(self, field, old + v)
        return old

    def _reserve(self, k: int, deq: bool):
        """Returns how many of k operations were granted."""
        if self.form == "exact":
            c = self.count
            yield "step"
            while True:
                room = c if deq else self.N - c
                if room <= 0:
                    return 0
                take = min(room, k)
                nc = c - take if deq else c + take
                if self.count == c:              # compare-and-swap
                    self.count = nc
                    yield "step"
                    return take
                c = self.count
                yield "step"
        if self.form == "naive":
            old = self._fetch_add("count", -k if deq else k)
            yield "step"
            got = min(max(old, 0), k) if deq else min(max(self.N - old, 0), k)
            if got < k:
                self._fetch_add("count", (k - got) if deq else -(k - got))
                yield "step"
            return got
        field = "avail" if deq else "free"
        old = self._fetch_add(field, -k)
        yield "step"
        got = min(max(old, 0), k)
        if got < k:
            self._fetch_add(field, k - got)
            yield "step"
        return got

    def enqueue_warp(self, items):
        """Generator: enqueue up to len(items) items at once; returns the
        list of (item, pos) placed (the first ones)."""
        got = yield from self._reserve(len(items), deq=False)
        if got == 0:
            return []
        pos = self._fetch_add("tail", got)
        yield "step"
        placed = []
        for i in range(got):
            p = pos + i
            slot, lap = p % self.N, p // self.N
            while self.tickets[slot] != 2 * lap:
                yield "wait"
            self.ring[slot] = items[i]
            self.tickets[slot] = 2 * lap + 1
            yield "step"
            placed.append((items[i], p))
        if self.form == "split":
            self._fetch_add("avail", got)          # published: dequeuers may take them
            yield "step"
        return placed

    def dequeue_warp(self, k: int):
        """Generator: dequeue up to k items at once; returns [(item, pos)]."""
        got = yield from self._reserve(k, deq=True)
        if got == 0:
            return []
        pos = self._fetch_add("head", got)
        yield "step"
        out = []
        for i in range(got):
            p = pos + i
            slot, lap = p % self.N, p // self.N
            while self.tickets[slot] != 2 * lap + 1:
                yield "wait"
            out.append((self.ring[slot], p))
            self.tickets[slot] = 2 * (lap + 1)
            yield "step"
        if self.form == "split":
            self._fetch_add("free", got)
            yield "step"
        return out


class CtaRingSim:
    """The vertex ring of the single-CTA path (one CTA, shared memory) as
    step generators: a take ticket (head) and a fill ticket (tail) over C
    slots; a warp reserves up to k items with one compare-and-swap on head
    (the warp-aggregated ensure of Algorithm 1, at CTA scope), a filler takes
    its tickets with one fetch-add on tail; a slot is filled by compare-and-
    swap from empty and taken by exchange with empty.  Two tickets a lap
    apart that meet on one slot may swap items, but no item is taken twice
    or lost.  The caller keeps at most C items filled-or-reserved and not
    yet taken (in the kernel the in-queue flag does: a vertex is queued at
    most once, and C >= V), so a filler only ever waits for a taker that has
    already reserved the item in its slot."""

    def __init__(self, capacity: int):
        self.C = capacity
        self.head = 0
        self.tail = 0
        self.slots = [None] * capacity
        self.fill_ticket = {}        # item -> ticket it was filled at
        self.take_ticket = {}        # item -> ticket it was taken at

    def fill(self, items):
        """Generator: publish items; returns their first ticket."""
        p = self.tail                # fetch-add on the fill ticket
        self.tail += len(items)
        yield "step"
        for i, x in enumerate(items):
            s = (p + i) % self.C
            while self.slots[s] is not None:       # compare-and-swap fails: full
                yield "wait"
            self.slots[s] = x                      # compare-and-swap succeeds
            self.fill_ticket[x] = p + i
            yield "step"
        return p

    def take(self, kmax: int, racy: bool = False):
        """Generator: take up to kmax items; returns them ([] if none).
        racy=True reads a slot and empties it in two steps instead of one
        exchange (kept to show that two takers meeting on a slot can then
        both take its item)."""
        h = self.head
        yield "step"
        while True:
            avail = self.tail - h
            if avail <= 0:
                return []
            k = min(avail, kmax)
            if self.head == h:                     # compare-and-swap on head
                self.head = h + k
                yield "step"
                break
            h = self.head
            yield "step"
        out = []
        for i in range(k):
            s = (h + i) % self.C
            while True:
                if racy:
                    x = self.slots[s]
                    yield "step"
                    self.slots[s] = None
                else:
                    x, self.slots[s] = self.slots[s], None     # exchange with empty
                if x is not None:
                    self.take_ticket[x] = h + i
                    out.append(x)
                    yield "step"
                    break
                yield "wait"
        return out


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
