// Warp-level building blocks shared by the single-query and the batched
// persistent SSSP kernels: warp scans, the owner search of a merged edge
// list, sub-queue probing, warp-aggregated enqueue of lanes or of a buffer,
// and the label compare-and-swap.
#pragma once

#include "bfq_internal.h"

namespace bfq {
namespace {

constexpr int kBlock = 256;
#ifndef BFQ_MIN_CTAS_PER_SM
#define BFQ_MIN_CTAS_PER_SM 4
#endif

__device__ __forceinline__ void raise_status(Control* ctl, int bits) {
  atomicOr(&ctl->status, bits);
  st_relaxed_s32(&ctl->stop, 1);
}

__device__ __forceinline__ unsigned long long warp_sum_u64(unsigned long long x) {
#pragma unroll
  for (int o = 16; o; o >>= 1) x += __shfl_down_sync(kFullMask, x, o);
  return x;
}

// Exclusive prefix of `x` over the warp; *total receives the sum.
__device__ __forceinline__ int warp_excl_scan(int x, int lane, int* total) {
  int incl = x;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    int n = __shfl_up_sync(kFullMask, incl, o);
    if (lane >= o) incl += n;
  }
  *total = __shfl_sync(kFullMask, incl, 31);
  return incl - x;
}

// For position t of a merged list, the owning lane: the largest j < n with
// excl_j <= t (excl non-decreasing over lanes).
__device__ __forceinline__ int owner_lane(int excl, int t, int n) {
  int j = 0;
#pragma unroll
  for (int step = 16; step >= 1; step >>= 1) {
    const int cand = j + step;
    const int ex = __shfl_sync(kFullMask, excl, cand & 31);
    if (cand < n && ex <= t) j = cand;
  }
  return j;
}

__device__ __forceinline__ unsigned lanemask_le() {
  unsigned m;
  asm("mov.u32 %0, %%lanemask_le;" : "=r"(m));
  return m;
}
__device__ __forceinline__ unsigned lanemask_lt() {
  unsigned m;
  asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
  return m;
}

// A warp's batch staged for the merged edge walk.  The items that have
// edges to relax are compacted, in lane order, into slots 0..k-1; edge t of
// the merged list (positions excl_j .. excl_j + deg_j - 1 belong to the
// item of lane j) is adj[off[r] + t] for the item's slot r, and key0[r] is
// (dist, hops + 1) of the item's tail label, the candidate key before the
// edge weight is added.
struct BatchStage {
  long long key0[32];
  int off[32];
  int tail[32];
};

// Slot (in the compacted order) of the item that owns position P + lane of
// the merged list, for a warp-uniform P.  has/excl are the lane's item flag
// and exclusive edge prefix; slots are consecutive along the list, so the
// owner is the slot of position P plus the number of item starts in
// (P, P + lane], read from a 32-bit mask of the starts in (P, P + 32).
__device__ __forceinline__ int staged_owner(bool has, int excl, int P) {
  const unsigned bit = (has && excl > P && excl < P + 32) ? (1u << (excl - P)) : 0u;
  const unsigned starts = __reduce_or_sync(kFullMask, bit);
  const int o0 = __popc(__ballot_sync(kFullMask, has && excl <= P)) - 1;
  return o0 + __popc(starts & lanemask_le());
}

// Candidate label of an edge of weight w out of a tail whose key0 is
// (dist, hops + 1): (dist + w, hops + 1), or minus infinity from a
// minus-infinity tail.  Returns 0 (no candidate: dist + w cannot be stored),
// 1 (candidate in *key) or -1 (dist + w is below the int32 range).
__device__ __forceinline__ int edge_candidate(long long key0, int w, long long* key) {
  const int d = label_dist(key0);
  if (d == kNegInf32) {
    *key = kNegInfLabel;
    return 1;
  }
  const long long nd = (long long)d + (long long)w;
  if (nd >= (long long)kInf32) return 0;
  if (nd <= -2147483648LL) return -1;
  *key = key0 + (long long)((unsigned long long)(long long)w << 32);
  return 1;
}

// Lanes probe up to 64 sub-queues starting at `start`; returns the fullest
// non-empty one seen, or -1.
__device__ __forceinline__ int probe_queues(const QueueSet& qs, int start, int skip, int lane) {
  for (int r = 0; r < 2 && r * 32 < qs.Q; ++r) {
    const int i = r * 32 + lane;
    const int q = (start + i) % qs.Q;
    const int c = (i < qs.Q && q != skip) ? ld_relaxed_s32(&qs.meta[q].count) : 0;
    const int m = __reduce_max_sync(kFullMask, c);
    if (m > 0) {
      const unsigned who = __ballot_sync(kFullMask, c == m);
      return __shfl_sync(kFullMask, q, __ffs(who) - 1);
    }
  }
  return -1;
}

// Warp-collective enqueue of the lanes with `active` into the sub-queues of
// qs, starting at `home` and moving on while a sub-queue is full, for at most
// max_tries reservations.  Returns the number of items placed (the active
// lanes of lowest rank), or -1 if a ticket wait ran out.
__device__ __forceinline__ int enqueue_warp(const QueueSet& qs, int home, bool active,
                                            unsigned item, int lane, long long spin_limit,
                                            long long max_tries) {
  const unsigned mask = __ballot_sync(kFullMask, active);
  if (!mask) return 0;
  const int k = __popc(mask);
  const int rank = __popc(mask & ((1u << lane) - 1u));
  const int cap = 1 << qs.cap_log2;
  int done = 0;
  int q = home;
  for (long long tries = 0; done < k && tries < max_tries; ++tries) {
    unsigned long long pos = 0;
    int got = 0;
    if (lane == 0) got = wq_reserve(qs.meta + q, k - done, false, cap, &pos, -1, qs.split);
    got = __shfl_sync(kFullMask, got, 0);
    if (got) {
      pos = __shfl_sync(kFullMask, pos, 0);
      const int r = rank - done;
      bool ok = true;
      if (active && r >= 0 && r < got)
        ok = wq_put(qs.slots + ((size_t)q << qs.cap_log2), qs.cap_log2, pos + r, item,
                    spin_limit);
      if (__any_sync(kFullMask, !ok)) return -1;
      if (lane == 0) wq_after_put(qs.meta + q, got, qs.split);
      done += got;
    }
    q = (q + 1 == qs.Q) ? 0 : q + 1;
  }
  return done;
}

// Per-warp statistics of one launch (32 bits: they stay far below 2^32 per
// warp; the launch totals are 64-bit).
struct WarpCounters {
  unsigned deq = 0, rel = 0, upd = 0, enq = 0, steal = 0, chunk = 0, idle = 0;
};

constexpr int kChildBuf = 256;   // claimed children buffered per warp

// Publish `count` items from the warp's buffer to the sub-queues of qs,
// starting at `home`: one broker reservation (and one tail ticket range) per
// sub-queue visited, every lane writing a share of the slots.  Returns false
// if no room was found within the bounds or a ticket wait ran out.
__device__ __forceinline__ bool enqueue_buffer(const QueueSet& qs, int home,
                                               const unsigned* buf, int count, int lane,
                                               long long spin_limit, long long max_tries) {
  const int cap = 1 << qs.cap_log2;
  int done = 0;
  int q = home;
  for (long long tries = 0; done < count && tries < max_tries; ++tries) {
    unsigned long long pos = 0;
    int got = 0;
    if (lane == 0) got = wq_reserve(qs.meta + q, count - done, false, cap, &pos, -1, qs.split);
    got = __shfl_sync(kFullMask, got, 0);
    if (got) {
      pos = __shfl_sync(kFullMask, pos, 0);
      unsigned long long* qslots = qs.slots + ((size_t)q << qs.cap_log2);
      bool ok = true;
      for (int i = lane; i < got; i += 32)
        ok = wq_put(qslots, qs.cap_log2, pos + i, buf[done + i], spin_limit) && ok;
      if (__any_sync(kFullMask, !ok)) return false;
      if (lane == 0) wq_after_put(qs.meta + q, got, qs.split);
      done += got;
    }
    q = (q + 1 == qs.Q) ? 0 : q + 1;
  }
  return done == count;
}

// Lower label[v] to `key` unless it is already at least as small; on success
// set the in-queue flag in the same compare-and-swap.  Returns 0 (no
// change), 1 (lowered, flag was already set) or 2 (lowered and this caller
// must enqueue v).
__device__ __forceinline__ int lower_label(long long* label_v, long long key, long long seen) {
  long long old = seen;
  while (key < label_key(old)) {
    const long long prev = (long long)atomicCAS((unsigned long long*)label_v,
                                                (unsigned long long)old,
                                                (unsigned long long)(key | kQueuedBit));
    if (prev == old) return (old & kQueuedBit) ? 1 : 2;
    old = prev;
  }
  return 0;
}

#ifndef BFQ_EDGE_GROUPS
#define BFQ_EDGE_GROUPS 2
#endif
constexpr int kGroups = BFQ_EDGE_GROUPS;   // edge groups of 32 in flight per warp step

// Negative-cycle accelerator.  A successful relaxation that gives v a label
// of walk0 / 2 hops or more (walk0: the run's first walk threshold) records
// its edge (tail, weight) in cyc[v], one 8-byte store.  When a label reaches
// the lane's walk threshold (walk0 at first, twice the label's hops after a
// failed walk) the lane walks
// the recorded edges backwards from v (Brent's cycle finding, at most
// kCycWalk steps).  If they close a cycle, the weights are re-read around it:
// a closed walk of real edges with negative total weight, through vertices
// that hold finite labels in this run, proves a reachable negative cycle.
// Nothing else is concluded from the walk, so a racy or stale record can
// only make a proof fail, never make one up; the hops >= V test remains the
// exact fallback.
constexpr int kCycWalk = 32;

__device__ __forceinline__ long long pack_edge(int tail, int w) {
  return (long long)(((unsigned long long)(unsigned)w << 32) | (unsigned)tail);
}

__device__ __noinline__ bool prove_negative_cycle(const long long* cyc,
                                                  const long long* label, int v, int V) {
  long long e = ld_relaxed_s64(cyc + v);
  int hare = (int)(unsigned)e;
  if (hare < 0 || hare >= V) return false;
  int tort = v, power = 1, lam = 1, steps = 1;
  while (tort != hare) {
    if (++steps > kCycWalk) return false;
    if (power == lam) {
      tort = hare;
      power <<= 1;
      lam = 0;
    }
    e = ld_relaxed_s64(cyc + hare);
    hare = (int)(unsigned)e;
    ++lam;
    if (hare < 0 || hare >= V) return false;
  }
  long long sum = 0;
  int x = hare;
  for (int i = 0; i < lam; ++i) {
    if (label_dist(ld_relaxed_s64(label + x)) == kInf32) return false;
    e = ld_relaxed_s64(cyc + x);
    const int y = (int)(unsigned)e;
    if (y < 0 || y >= V) return false;
    sum += (long long)(int)(e >> 32);
    x = y;
  }
  return x == hare && sum < 0;
}

__device__ __forceinline__ int share_of(int cnt, int max_items, int share) {
  return min(max_items, max(1, (cnt + share - 1) / share));
}

}  // namespace
}  // namespace bfq
