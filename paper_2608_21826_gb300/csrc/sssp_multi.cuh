// Multi-query building blocks shared by the batched and the serving kernels:
// a warp's batch may hold items of several queries, each query with its own
// label slice, in-flight counter and status bits.
#pragma once

#include "sssp_common.cuh"

// Registers of the multi-query kernels (batched, serving) and edge groups of
// their merged walk.  With the staged walk (per-query fields in shared
// memory, not in registers) 4 CTAs per SM at 64 registers and 2 groups in
// flight are fastest on the batched mix (34.6 ms per launch against 39.8 at
// 3 CTAs per SM with 3 groups).
#ifndef BFQ_MULTI_CTAS_PER_SM
#define BFQ_MULTI_CTAS_PER_SM 4
#endif
#ifndef BFQ_MULTI_EDGE_GROUPS
#define BFQ_MULTI_EDGE_GROUPS 2
#endif

namespace bfq {
namespace {

constexpr int kCounterStride = 32;  // one 128-byte line per query counter (4 per line
                                     // serialise: batched mix 34.8 against 32.9 ms)
constexpr int kMultiGroups = BFQ_MULTI_EDGE_GROUPS;

// Where the per-query state lives.
struct MultiEnv {
  long long* pool;              // label pool; an item is an index into it
  long long* cyc;               // recorded relaxation edges, indexed like pool (or null)
  int* inflight;                // [query * kCounterStride]
  int* qstatus;                 // [query] kStNegCycle / kStRange
  int* gstatus;                 // launch-wide kSt* bits
  int* gstop;                   // launch-wide stop flag
  QueueSet qs;                  // vertex sub-queues
  long long spin_limit;
  unsigned cyc_walk0;           // first cycle-walk threshold (hops); records from half
};

// Count the buffered children in their queries' in-flight counters, then
// publish them (one broker reservation per sub-queue visited).
__device__ __forceinline__ bool flush_multi(const MultiEnv& e, int home, unsigned* buf,
                                            unsigned short* bufq, int& nbuf, int lane,
                                            WarpCounters& wc) {
  if (nbuf == 0) return true;
  __syncwarp();
  for (int i = 0; i < nbuf; i += 32) {
    const int idx = i + lane;
    const int q = idx < nbuf ? (int)bufq[idx] : -1;
    const unsigned m = __match_any_sync(kFullMask, q);
    if (q >= 0 && lane == __ffs(m) - 1)
      red_add_relaxed_s32(&e.inflight[q * kCounterStride], __popc(m));
  }
  if (lane == 0) wc.enq += nbuf;
  __syncwarp();
  const bool ok = enqueue_buffer(e.qs, home, buf, nbuf, lane, e.spin_limit, 4LL * e.qs.Q + 64);
  __syncwarp();
  if (!ok && lane == 0) {
    atomicOr(e.gstatus, kStQueue);
    st_relaxed_s32(e.gstop, 1);
  }
  nbuf = 0;
  return ok;
}

// A mixed batch staged for the merged edge walk (as BatchStage, with the
// per-query fields): slot r holds the item of the r-th lane with edges.
struct MultiStage {
  long long ebase[32];          // address of merged-list position 0 for this item
  long long* lbase[32];         // the item's query's labels
  long long key0[32];           // (dist, hops + 1) of the tail's label
  int q[32];                    // query
  int vq[32];                   // the query graph's vertex count
  int tail[32];
};

// Merged relaxation of a mixed batch: lane j owns edges [0, deg_j) at eptr_j
// of a tail with label lab_j in query q_j, whose labels start at lbase_j in
// the pool and which has V_j vertices.  The items with edges are staged in
// shared memory and each edge position finds its item's slot with
// staged_owner; the next step's edge loads are issued before this step's
// label atomics.  MIN: one atomicMin per edge lowers the label and claims the
// in-queue flag (keys are even, so key | 1 is below a label exactly when key
// is below its key part); for labels that stay in L2, since every atomic
// dirties its line.  Otherwise load, then the same atomicMin only when the
// key is below the loaded label (a stale load is only ever too high).
template <int U, bool MIN>
__device__ __forceinline__ bool relax_multi(const MultiEnv& e, int n, const int2* eptr, int deg,
                                            long long lab, long long* lbase, int Vq, int q,
                                            int tail, int lane, int home, WarpCounters& wc,
                                            unsigned* buf, unsigned short* bufq, int& nbuf,
                                            unsigned& walk_at, MultiStage* st) {
  const bool has = lane < n && deg > 0;
  const unsigned hm = __ballot_sync(kFullMask, has);
  if (!hm) return true;
  int total = 0;
  const int excl = warp_excl_scan(has ? deg : 0, lane, &total);
  wc.rel += (lane == 0) ? (unsigned)total : 0u;
  if (has) {
    const int r = __popc(hm & lanemask_lt());
    st->ebase[r] = (long long)(size_t)eptr - (long long)sizeof(int2) * excl;
    st->lbase[r] = lbase;
    st->key0[r] = pack_label(label_dist(lab), label_hops(lab) + 1u);
    st->q[r] = q;
    st->vq[r] = Vq;
    st->tail[r] = tail;
  }
  __syncwarp();
  int2 nx_cw[U];
  int nx_own[U];
  bool nx_act[U];
#pragma unroll
  for (int g = 0; g < U; ++g) {
    nx_act[g] = false;
    nx_cw[g] = make_int2(0, 0);
    nx_own[g] = 0;
    const int P = 32 * g;
    if (P < total) {
      nx_own[g] = staged_owner(has, excl, P);
      if (P + lane < total) {
        nx_act[g] = true;
        nx_cw[g] = __ldg((const int2*)(size_t)(st->ebase[nx_own[g]] +
                                                (long long)sizeof(int2) * (P + lane)));
      }
    }
  }
  for (int base = 0; base < total; base += 32 * U) {
    int2 cw[U];
    int own[U];
    bool act[U];
#pragma unroll
    for (int g = 0; g < U; ++g) {
      cw[g] = nx_cw[g];
      own[g] = nx_own[g];
      act[g] = nx_act[g];
      nx_act[g] = false;
      const int P = base + 32 * U + 32 * g;
      if (P < total) {                      // warp-uniform
        nx_own[g] = staged_owner(has, excl, P);
        if (P + lane < total) {
          nx_act[g] = true;
          nx_cw[g] = __ldg((const int2*)(size_t)(st->ebase[nx_own[g]] +
                                                  (long long)sizeof(int2) * (P + lane)));
        }
      }
    }
    long long key[U], cur[U];
#pragma unroll
    for (int g = 0; g < U; ++g) {
      key[g] = 0;
      cur[g] = 0;
      if (act[g]) {
        const int c = edge_candidate(st->key0[own[g]], cw[g].y, &key[g]);
        if (c < 0) atomicOr(&e.qstatus[st->q[own[g]]], kStRange);
        act[g] = c > 0;
        if (act[g] && !MIN) cur[g] = ld_relaxed_s64(st->lbase[own[g]] + cw[g].x);
      }
    }
    if (MIN) {
#pragma unroll
      for (int g = 0; g < U; ++g)
        if (act[g]) cur[g] = atomicMin(st->lbase[own[g]] + cw[g].x, key[g] | kQueuedBit);
    } else {
#pragma unroll
      for (int g = 0; g < U; ++g) {
        if (act[g] && key[g] < label_key(cur[g]))
          cur[g] = atomicMin(st->lbase[own[g]] + cw[g].x, key[g] | kQueuedBit);
        else
          act[g] = false;
      }
    }
    bool enq[U];
#pragma unroll
    for (int g = 0; g < U; ++g) {
      enq[g] = false;
      if (act[g]) {
        long long* lb = st->lbase[own[g]];
        const int r = key[g] < label_key(cur[g]) ? ((cur[g] & kQueuedBit) ? 1 : 2) : 0;
        if (r) {
          ++wc.upd;
          const unsigned nh = label_hops(key[g]);
          const int vq = st->vq[own[g]];
          if (nh >= (unsigned)vq) {
            atomicOr(&e.qstatus[st->q[own[g]]], kStNegCycle);
          } else {
            enq[g] = (r == 2);
            if (e.cyc && nh >= (e.cyc_walk0 >> 1)) {
              long long* cb = e.cyc + (lb - e.pool);
              st_relaxed_u64((unsigned long long*)(cb + cw[g].x),
                             (unsigned long long)pack_edge(st->tail[own[g]], cw[g].y));
              if (nh >= walk_at) {
                if (prove_negative_cycle(cb, lb, cw[g].x, vq))
                  atomicOr(&e.qstatus[st->q[own[g]]], kStNegCycle);
                else
                  walk_at = nh * 2;
              }
            }
          }
        }
      }
    }
#pragma unroll
    for (int g = 0; g < U; ++g) {
      const unsigned m = __ballot_sync(kFullMask, enq[g]);
      if (m) {
        if (nbuf + __popc(m) > kChildBuf) {
          if (!flush_multi(e, home, buf, bufq, nbuf, lane, wc)) return false;
        }
        if (enq[g]) {
          const int slot = nbuf + __popc(m & lanemask_lt());
          buf[slot] = (unsigned)((st->lbase[own[g]] - e.pool) + cw[g].x);
          bufq[slot] = (unsigned short)st->q[own[g]];
        }
        nbuf += __popc(m);
      }
    }
  }
  __syncwarp();                         // stage free for the next batch
  return true;
}

// Retire the lanes' items (q = -1 for lanes without one): per query one
// subtraction; returns, in the lane that made it, the query it emptied (or
// -1 everywhere else).
__device__ __forceinline__ int retire_multi(const MultiEnv& e, int q, int lane) {
  const unsigned m = __match_any_sync(kFullMask, q);
  int emptied = -1;
  if (q >= 0 && lane == __ffs(m) - 1) {
    const int cnt = __popc(m);
    const int old = atomicAdd(&e.inflight[q * kCounterStride], -cnt);
    if (old == cnt) emptied = q;
  }
  return emptied;
}

}  // namespace
}  // namespace bfq
