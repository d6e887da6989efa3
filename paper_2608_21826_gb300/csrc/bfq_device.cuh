// Device primitives shared by the SSSP and queue kernels: memory-ordering
// helpers (inline PTX), bounded waits, and the Broker Queue operations of
// Sec. III-A / Algorithm 1 in the two forms the library uses:
//
//   * per-thread (Algorithm 1 as printed, with the readings listed below),
//     used by the standalone queue benchmark for BFQ_QUEUE_BQ / BFQ_QUEUE_BWD;
//   * warp-aggregated (BFQ_QUEUE_BQ_WARP and the SSSP worklist): one broker
//     reservation and one head/tail ticket per warp for up to 32 items.
//
// Readings of Algorithm 1 (the listing is garbled in places):
//   - ENSURE_DEQUEUE grants the dequeue when its fetch-and-decrement of count
//     returned a value > 0 (the listing never sets the grant).
//   - READ_DATA releases the slot with ticket 2*(Pos/N + 1), the even ticket
//     the next lap's enqueuer waits for.
//   - head/tail are 64-bit and never wrap, so "Full" is tail-head >= N and
//     "Empty" is tail-head <= 0.
// Warp-aggregated forms: a warp reserves k items at once.  Exact-count form:
// the broker count is moved with compare-and-swap to an exact value instead
// of the paper's add-then-undo; every ticket wait is then on an operation
// that has already been granted (see the proof sketch at wq_reserve), so no
// waiter can be stranded by a reservation that is later withdrawn.
// Single-shot form (BWD's ensure-once): one fetch-add on one of two
// counters, each read by one side only, so a withdrawn surplus is never
// visible to the other side (also at wq_reserve).
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace bfq {

constexpr unsigned kFullMask = 0xffffffffu;
constexpr int kInf32 = 2147483647;

// Status bits collected while a run executes.
enum : int {
  kStNegCycle = 1,
  kStRange = 2,
  kStTimeout = 4,
  kStQueue = 8,      // internal: no sub-queue had room (cannot happen when
                     // total capacity >= number of vertices)
};

// ---------------------------------------------------------------------------
// memory-ordering helpers (PTX memory model, .gpu scope)
// ---------------------------------------------------------------------------
__device__ __forceinline__ unsigned long long ld_acquire_u64(const unsigned long long* p) {
  unsigned long long v;
  asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ unsigned long long ld_relaxed_u64(const unsigned long long* p) {
  unsigned long long v;
  asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ long long ld_relaxed_s64(const long long* p) {
  long long v;
  asm volatile("ld.relaxed.gpu.global.s64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ int ld_relaxed_s32(const int* p) {
  int v;
  asm volatile("ld.relaxed.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ unsigned ld_relaxed_u32(const unsigned* p) {
  unsigned v;
  asm volatile("ld.relaxed.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ int ld_acquire_s32(const int* p) {
  int v;
  asm volatile("ld.acquire.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ unsigned ld_acquire_u32(const unsigned* p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void st_release_u64(unsigned long long* p, unsigned long long v) {
  asm volatile("st.release.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}
__device__ __forceinline__ void st_relaxed_u64(unsigned long long* p, unsigned long long v) {
  asm volatile("st.relaxed.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}
__device__ __forceinline__ void st_release_u32(unsigned* p, unsigned v) {
  asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ void st_relaxed_s32(int* p, int v) {
  asm volatile("st.relaxed.gpu.global.s32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ void fence_acq_rel_gpu() {
  asm volatile("fence.acq_rel.gpu;" ::: "memory");
}
// fetch-and-add with release semantics: orders every earlier access of this
// thread (and, through __syncwarp, of its warp) before the update.
__device__ __forceinline__ int atom_add_release_s32(int* p, int v) {
  int old;
  asm volatile("atom.release.gpu.global.add.s32 %0, [%1], %2;"
               : "=r"(old) : "l"(p), "r"(v) : "memory");
  return old;
}
// fire-and-forget add (no value returned, so the warp does not wait)
__device__ __forceinline__ void red_add_relaxed_s32(int* p, int v) {
  asm volatile("red.relaxed.gpu.global.add.s32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ unsigned long long globaltimer_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Label word of a vertex: dist (int32) in the high half, hops (31 bits) in
// bits 1..31, and the in-queue flag in bit 0.  With the flag cleared, signed
// 64-bit order is lexicographic (dist, hops) order, so comparing words
// compares labels.  Keeping the flag in the label word lets a producer lower
// the label and claim the enqueue in one compare-and-swap, and a consumer
// clear the flag and read the label in one atomicAnd: a single memory
// location, so no fence is needed to order the two.
constexpr long long kQueuedBit = 1LL;
constexpr long long kInfLabel = 0x7ffffffffffffffeLL;   // (INT32_MAX, 2^31-1), not queued
// (INT32_MIN, 0): minus infinity, below every other label; only written when
// negative cycles are resolved (a finite dist never reaches INT32_MIN).
constexpr long long kNegInfLabel = (long long)0x8000000000000000ULL;
constexpr int kNegInf32 = (int)0x80000000u;

__device__ __forceinline__ long long pack_label(int dist, unsigned hops) {
  return (long long)(((unsigned long long)(unsigned)dist << 32) |
                     ((unsigned long long)hops << 1));
}
__device__ __forceinline__ int label_dist(long long l) { return (int)(l >> 32); }
__device__ __forceinline__ unsigned label_hops(long long l) {
  return ((unsigned)(unsigned long long)l) >> 1;
}
__device__ __forceinline__ long long label_key(long long l) { return l & ~kQueuedBit; }

// ---------------------------------------------------------------------------
// warp-aggregated Broker Queue (sub-queue of the SSSP worklist)
// ---------------------------------------------------------------------------
// One sub-queue's counters, each on its own 128-byte line.  Within one line
// the atomics of the four counters serialise (the single-shot warp queue ran
// at 11.2 G ops/s with its counters 32 bytes apart, 21.1 G with them on
// separate lines; the counters of a line most likely share one L2 slice).
struct alignas(128) QueueMeta {
  int count;                    // exact form: broker count, items granted and
                                //   not yet taken; single-shot form: items
                                //   published and not yet granted to dequeuers
  int pad0[31];
  unsigned long long head;      // dequeue ticket counter
  unsigned long long pad1[15];
  unsigned long long tail;      // enqueue ticket counter
  unsigned long long pad2[15];
  int used;                     // single-shot form: places granted to
                                //   enqueuers and not yet released by dequeuers
  int pad3[31];
};
static_assert(sizeof(QueueMeta) == 512, "QueueMeta layout");

// Slot word: (ticket << 32) | item.  Ticket 2*lap means "free for the
// enqueuer of lap `lap`", 2*lap+1 "holds the item of lap `lap`"; packing the
// ticket with the item publishes both with one 8-byte store.
// split: 0 = exact-count reservations (compare-and-swap on count), 1 =
// single-shot reservations on two counters (see wq_reserve).
struct QueueSet {
  QueueMeta* meta;              // [Q]
  unsigned long long* slots;    // [Q << cap_log2]
  int Q;
  int cap_log2;
  int split;
};

// Leader-lane reservation on the broker count of one sub-queue.
// is_deq: take up to `want` items (count -> count - got);
// else:   grant up to `want` free places (count -> count + got, <= cap).
// Then take `got` consecutive head (or tail) tickets.  Returns got; *pos is
// the first ticket.
//
// Why exact counts make every ticket wait finite: let E and D be the numbers
// of granted enqueues and dequeues.  count = E - D stays in [0, cap].  A
// dequeuer holding head ticket p had D <= E when granted, so ticket p's
// enqueue was granted and will publish.  An enqueuer holding tail ticket p
// had E - D <= cap when it took the ticket, so ticket p - cap's dequeue was
// granted and will free the slot.  Every wait is on an earlier ticket that is
// already granted, hence no cycle of waits.
//
// Single-shot form (split = 1; the Broker Work Distributor's "ensure once"
// of Sec. III-A, warp-aggregated): two counters, each read by one side only.
// A dequeuer fetch-subtracts `want` from count (published items), keeps
// min(max(old, 0), want) and adds the surplus back; an enqueuer does the same
// on used (granted places) against cap.  One atomic and no retry: a
// transient surplus only understates what the other warps of the same side
// see (they take less, or move on), never what the opposite side sees.  The
// enqueuer adds its grant to count after publishing (wq_after_put) and the
// dequeuer releases its places from used after freeing the slots
// (wq_after_take).  Finite waits, by induction on tickets: grants never
// exceed the counter's true value, so at all times (dequeues granted) <=
// (items published) <= (tail tickets taken) and (enqueues granted) <= cap +
// (places released) <= cap + (head tickets taken).  A dequeuer's head ticket
// p therefore has its tail ticket taken, by an enqueuer whose own wait is on
// ticket p - cap < p; an enqueuer's tail ticket p >= cap has head ticket
// p - cap taken, by a dequeuer whose wait is on the item of that earlier
// ticket, after which it frees the slot.
__device__ __forceinline__ int wq_reserve(QueueMeta* m, int want, bool is_deq, int cap,
                                          unsigned long long* pos, int c_hint = -1,
                                          int split = 0) {
  int got = 0;
  if (split) {
    int* ctr = is_deq ? &m->count : &m->used;
    const int old = atomicAdd(ctr, is_deq ? -want : want);
    got = is_deq ? min(max(old, 0), want) : min(max(cap - old, 0), want);
    if (got < want) red_add_relaxed_s32(ctr, is_deq ? want - got : got - want);
  } else {
    int c = c_hint >= 0 ? c_hint : ld_relaxed_s32(&m->count);
    for (;;) {
      int room = is_deq ? c : cap - c;
      if (room <= 0) break;
      int take = min(room, want);
      int nc = is_deq ? c - take : c + take;
      int old = atomicCAS(&m->count, c, nc);
      if (old == c) { got = take; break; }
      c = old;
    }
  }
  if (got) *pos = atomicAdd(is_deq ? &m->head : &m->tail, (unsigned long long)got);
  return got;
}

// Single-shot form only: after an enqueuer has published `got` items, make
// them available to dequeuers; after a dequeuer has freed `got` slots, give
// the places back to enqueuers.  Called by one lane after a __syncwarp.
__device__ __forceinline__ void wq_after_put(QueueMeta* m, int got, int split) {
  if (split && got) red_add_relaxed_s32(&m->count, got);
}
__device__ __forceinline__ void wq_after_take(QueueMeta* m, int got, int split) {
  if (split && got) red_add_relaxed_s32(&m->used, -got);
}

// Publish `item` at ticket p of a sub-queue (wait for the slot's free ticket,
// then one release store).  Returns false if the wait ran out.
__device__ __forceinline__ bool wq_put(unsigned long long* qslots, int cap_log2,
                                       unsigned long long p, unsigned item,
                                       long long spin_limit) {
  unsigned long long* s = qslots + (p & ((1ull << cap_log2) - 1));
  const unsigned lap_ticket = 2u * (unsigned)(p >> cap_log2);
  unsigned long long w = ld_relaxed_u64(s);
  long long spins = 0;
  while ((unsigned)(w >> 32) != lap_ticket) {
    if (++spins > spin_limit) return false;
    __nanosleep(64);
    w = ld_relaxed_u64(s);
  }
  st_release_u64(s, ((unsigned long long)(lap_ticket + 1u) << 32) | item);
  return true;
}

// Take the item at ticket p (wait for the full ticket with acquire, then free
// the slot for the next lap).  Returns false if the wait ran out.
__device__ __forceinline__ bool wq_take(unsigned long long* qslots, int cap_log2,
                                        unsigned long long p, unsigned* item,
                                        long long spin_limit) {
  unsigned long long* s = qslots + (p & ((1ull << cap_log2) - 1));
  const unsigned full_ticket = 2u * (unsigned)(p >> cap_log2) + 1u;
  unsigned long long w = ld_acquire_u64(s);
  long long spins = 0;
  while ((unsigned)(w >> 32) != full_ticket) {
    if (++spins > spin_limit) return false;
    __nanosleep(64);
    w = ld_acquire_u64(s);
  }
  *item = (unsigned)w;
  st_relaxed_u64(s, (unsigned long long)(full_ticket + 1u) << 32);
  return true;
}

// Warp-collective dequeue of up to `want` items from sub-queue q.  Lanes
// [0, got) receive an item.  Returns got, or -1 if a ticket wait ran out.
__device__ __forceinline__ int wq_dequeue_warp(const QueueSet& qs, int q, int want, int lane,
                                               unsigned* item, long long spin_limit,
                                               int c_hint = -1) {
  unsigned long long pos = 0;
  int got = 0;
  if (lane == 0)
    got = wq_reserve(qs.meta + q, want, true, 1 << qs.cap_log2, &pos, c_hint, qs.split);
  got = __shfl_sync(kFullMask, got, 0);
  if (got == 0) return 0;
  pos = __shfl_sync(kFullMask, pos, 0);
  bool ok = true;
  if (lane < got)
    ok = wq_take(qs.slots + ((size_t)q << qs.cap_log2), qs.cap_log2, pos + lane, item,
                 spin_limit);
  if (__any_sync(kFullMask, !ok)) return -1;
  if (qs.split) {
    __syncwarp();
    if (lane == 0) wq_after_take(qs.meta + q, got, 1);
  }
  return got;
}

// ---------------------------------------------------------------------------
// per-thread Broker Queue / Broker Work Distributor (Algorithm 1)
// ---------------------------------------------------------------------------
struct alignas(128) BQState {
  int count;
  int pad0[31];
  unsigned long long head;
  unsigned long long pad1[15];
  unsigned long long tail;
  unsigned long long pad2[15];
  int error;                     // kStTimeout once a ticket wait ran out
  int pad3[31];
};

// WAIT_FOR_TICKET with a bound; acquire so the data written before the
// ticket (PUT_DATA) or read before it (READ_DATA) is ordered.
__device__ __forceinline__ bool bq_wait_ticket(const unsigned* t, unsigned expected,
                                               long long spin_limit) {
  long long spins = 0;
  while (ld_acquire_u32(t) != expected) {
    if (++spins > spin_limit) return false;
    __nanosleep(32);
  }
  return true;
}

// ENSURE_ENQUEUE: reserve one place with fetch-and-add, undo if the queue
// was full, retry while the re-read count shows room.
__device__ __forceinline__ bool bq_ensure_enqueue(BQState* q, int N) {
  int num = ld_relaxed_s32(&q->count);
  while (num < N) {
    if (atomicAdd(&q->count, 1) < N) return true;
    num = atomicSub(&q->count, 1) - 1;
  }
  return false;
}

// ENSURE_DEQUEUE (reading: grant when the decrement found an item).
__device__ __forceinline__ bool bq_ensure_dequeue(BQState* q) {
  int num = ld_relaxed_s32(&q->count);
  while (num > 0) {
    if (atomicSub(&q->count, 1) > 0) return true;
    atomicAdd(&q->count, 1);
    num = ld_relaxed_s32(&q->count);
  }
  return false;
}

}  // namespace bfq
