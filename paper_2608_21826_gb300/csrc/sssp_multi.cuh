// Multi-query building blocks shared by the batched and the serving kernels:
// a warp's batch may hold items of several queries, each query with its own
// label slice, in-flight counter and status bits.
#pragma once

#include "sssp_common.cuh"

// The multi-query kernels (batched, serving) keep more state per warp: their
// registers are sized for 3 CTAs per SM (80 per thread), which halves their
// spills (the batched mix: 45 against 48 ms per launch at 4 CTAs per SM).
#ifndef BFQ_MULTI_CTAS_PER_SM
#define BFQ_MULTI_CTAS_PER_SM 3
#endif

namespace bfq {
namespace {

constexpr int kCounterStride = 8;   // one 32-byte sector per query counter

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

// Merged relaxation of a mixed batch: lane j owns edges [0, deg_j) at eptr_j
// of a tail with label lab_j in query q_j, whose labels start at lbase_j in
// the pool and which has V_j vertices.  MIN: one atomicMin per edge lowers
// the label and claims the in-queue flag (keys are even, so key | 1 is below
// a label exactly when key is below its key part); for labels that stay in
// L2, since every atomic dirties its line.  Otherwise load, then
// compare-and-swap when lower.
template <int U, bool MIN>
__device__ __forceinline__ bool relax_multi(const MultiEnv& e, int n, const int2* eptr, int deg,
                                            long long lab, long long* lbase, int Vq, int q,
                                            int tail, int lane, int home, WarpCounters& wc,
                                            unsigned* buf, unsigned short* bufq, int& nbuf,
                                            unsigned& walk_at) {
  int total = 0;
  const int excl = warp_excl_scan(deg, lane, &total);
  wc.rel += (lane == 0) ? (unsigned)total : 0u;
  for (int base = 0; base < total; base += 32 * U) {
    int2 cw[U];
    long long lab_t[U];
    long long* lb[U];
    int qq[U], vv[U], tl[U];
    bool act[U];
#pragma unroll
    for (int g = 0; g < U; ++g) {
      act[g] = false;
      cw[g] = make_int2(0, 0);
      lab_t[g] = 0;
      lb[g] = nullptr;
      qq[g] = 0;
      vv[g] = 0;
      tl[g] = 0;
      if (base + 32 * g < total) {          // warp-uniform
        const int t = base + 32 * g + lane;
        const int j = owner_lane(excl, t, n);
        const int ex_j = __shfl_sync(kFullMask, excl, j);
        const int2* ep = (const int2*)__shfl_sync(kFullMask, (unsigned long long)eptr, j);
        lb[g] = (long long*)__shfl_sync(kFullMask, (unsigned long long)lbase, j);
        lab_t[g] = __shfl_sync(kFullMask, lab, j);
        qq[g] = __shfl_sync(kFullMask, q, j);
        vv[g] = __shfl_sync(kFullMask, Vq, j);
        tl[g] = __shfl_sync(kFullMask, tail, j);
        if (t < total) {
          act[g] = true;
          cw[g] = __ldg(ep + (t - ex_j));
        }
      }
    }
    long long key[U], cur[U];
#pragma unroll
    for (int g = 0; g < U; ++g) {
      key[g] = 0;
      cur[g] = 0;
      if (act[g]) {
        const long long nd = (long long)label_dist(lab_t[g]) + (long long)cw[g].y;
        if (nd >= (long long)kInf32) {
          act[g] = false;
        } else if (nd <= -2147483648LL) {
          atomicOr(&e.qstatus[qq[g]], kStRange);
          act[g] = false;
        } else {
          key[g] = pack_label((int)nd, label_hops(lab_t[g]) + 1u);
          if (!MIN) cur[g] = ld_relaxed_s64(lb[g] + cw[g].x);
        }
      }
    }
    long long prev[U];
    if (MIN) {
#pragma unroll
      for (int g = 0; g < U; ++g) {
        prev[g] = 0;
        if (act[g]) cur[g] = atomicMin(lb[g] + cw[g].x, key[g] | kQueuedBit);
      }
    } else {
      // first compare-and-swap of every group back to back (they overlap);
      // a failed one retries through lower_label
#pragma unroll
      for (int g = 0; g < U; ++g) {
        prev[g] = cur[g];
        if (act[g] && key[g] < label_key(cur[g]))
          prev[g] = (long long)atomicCAS((unsigned long long*)(lb[g] + cw[g].x),
                                         (unsigned long long)cur[g],
                                         (unsigned long long)(key[g] | kQueuedBit));
        else
          act[g] = false;
      }
    }
    bool enq[U];
#pragma unroll
    for (int g = 0; g < U; ++g) {
      enq[g] = false;
      if (act[g]) {
        const int r =
            MIN ? (key[g] < label_key(cur[g]) ? ((cur[g] & kQueuedBit) ? 1 : 2) : 0)
                : (prev[g] == cur[g]) ? ((cur[g] & kQueuedBit) ? 1 : 2)
                                      : lower_label(lb[g] + cw[g].x, key[g], prev[g]);
        if (r) {
          ++wc.upd;
          const unsigned nh = label_hops(key[g]);
          if (nh >= (unsigned)vv[g]) {
            atomicOr(&e.qstatus[qq[g]], kStNegCycle);
          } else {
            enq[g] = (r == 2);
            if (e.cyc && nh >= (e.cyc_walk0 >> 1)) {
              long long* cb = e.cyc + (lb[g] - e.pool);
              st_relaxed_u64((unsigned long long*)(cb + cw[g].x),
                             (unsigned long long)pack_edge(tl[g], cw[g].y));
              if (nh >= walk_at) {
                if (prove_negative_cycle(cb, lb[g], cw[g].x, vv[g]))
                  atomicOr(&e.qstatus[qq[g]], kStNegCycle);
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
          const int slot = nbuf + __popc(m & ((1u << lane) - 1u));
          buf[slot] = (unsigned)((lb[g] - e.pool) + cw[g].x);
          bufq[slot] = (unsigned short)qq[g];
        }
        nbuf += __popc(m);
      }
    }
  }
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
