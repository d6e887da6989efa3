// Queue-driven Bellman-Ford SSSP on one GPU (Sec. III-C, Algorithm 3).
//
// One persistent kernel runs the whole query.  Every warp loops:
//   dequeue a batch of up to 32 items (warp-aggregated Broker Queue,
//   own sub-queue first, then stealing), relax their out-edges as one merged,
//   lane-contiguous edge stream, enqueue the vertices whose label dropped and
//   whose in-queue bit it won, and retire the batch from the in-flight count.
// The run ends when the in-flight count reaches zero (this replaces the
// paper's per-round change count and cross-GPU reduction), when a label with
// hops >= V is accepted (negative cycle), or on a range error or timeout.
//
// Labels are (dist, hops) packed in 64 bits and lowered with one atomicMin
// (while the labels fit in L2) or a load and a compare-and-swap; the
// relaxation test is the one of PARALLEL_RELAX_EDGES (Algorithm 3) applied to
// the lexicographic label and made atomic (the listing's fetch / compare /
// put sequence would lose concurrent updates).
//
// Vertices of out-degree > hub_degree are split into chunks of chunk_edges
// edges published to a second set of sub-queues, so many warps share a hub.
#include "sssp_common.cuh"

namespace bfq {

namespace {

// Count the buffered children as in flight (before any becomes visible),
// then publish them.  retire (> 0 only once the warp's batch is fully
// relaxed) is the batch's item count, taken off in the same update: the
// single in-flight counter is the kernel's most contended address, so a
// batch changes it once, not twice.
__device__ __forceinline__ bool flush_children(const SsspArgs& a, int home, unsigned* buf,
                                               int& nbuf, int lane, WarpCounters& wc,
                                               int retire = 0) {
  if (nbuf == 0) {
    if (retire && lane == 0) red_add_relaxed_s32(&a.ctl->inflight, -retire);
    return true;
  }
  __syncwarp();                         // buffer writes visible to all lanes
  if (lane == 0) {
    red_add_relaxed_s32(&a.ctl->inflight, nbuf - retire);
    wc.enq += nbuf;
  }
  __syncwarp();
  const bool ok = enqueue_buffer(a.qs, home, buf, nbuf, lane, a.spin_limit, 4LL * a.qs.Q + 64);
  __syncwarp();                         // buffer free for reuse
  if (!ok && lane == 0) atomicOr(&a.ctl->status, kStQueue);
  nbuf = 0;
  return ok;
}

// Relax the merged edge lists of the items held by lanes [0, n): lane j owns
// edges [beg_j, beg_j + deg_j) of a tail whose label is lab_j.  The items
// with edges are staged in shared memory (BatchStage) and the edges walked
// lane-contiguously, U groups of 32 per step so that the loads of the
// groups overlap; the next step's edge loads are issued before this step's
// label atomics, so the two round trips overlap.  Returns false on a timeout.
// Claimed children are appended to the warp's buffer `buf` (nbuf items,
// capacity kChildBuf) and published in bulk by flush_children.
// Relaxation forms of the single-query kernel (SsspArgs::relax_min).
constexpr int kRelaxCas = 0;      // load, then compare-and-swap when lower
constexpr int kRelaxMin = 1;      // one atomicMin per edge
constexpr int kRelaxFilter = 2;   // load, then atomicMin only when lower

template <int U, int RX>
__device__ __forceinline__ bool relax_merged(const SsspArgs& a, int n, int beg, int deg,
                                             long long lab, int tail, int lane, int home,
                                             WarpCounters& wc, unsigned* buf, int& nbuf,
                                             unsigned& walk_at, BatchStage* st) {
  const bool has = lane < n && deg > 0;
  const unsigned hm = __ballot_sync(kFullMask, has);
  if (!hm) return true;
  int total = 0;
  const int excl = warp_excl_scan(has ? deg : 0, lane, &total);
  wc.rel += (lane == 0) ? (unsigned)total : 0u;
  if (has) {
    const int r = __popc(hm & lanemask_lt());
    st->key0[r] = pack_label(label_dist(lab), label_hops(lab) + 1u);
    st->off[r] = beg - excl;
    st->tail[r] = tail;
  }
  __syncwarp();
  const unsigned V = (unsigned)a.V;
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
        nx_cw[g] = __ldg(&a.adj[st->off[nx_own[g]] + P + lane]);
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
          nx_cw[g] = __ldg(&a.adj[st->off[nx_own[g]] + P + lane]);
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
        if (c < 0) raise_status(a.ctl, kStRange);
        act[g] = c > 0;
        if (act[g] && RX != kRelaxMin) cur[g] = ld_relaxed_s64(&a.label[cw[g].x]);
      }
    }
    long long prev[U];
    if (RX == kRelaxMin) {
      // One atomicMin per edge lowers the label and claims the in-queue flag
      // at once: keys are even (bit 0 is the flag), so key | 1 is below a
      // label exactly when key is below the label's key part, and the
      // minimum then carries the flag.  Used while the label array sits in
      // L2: every atomic, lowering or not, dirties its line.
#pragma unroll
      for (int g = 0; g < U; ++g) {
        prev[g] = 0;
        if (act[g]) cur[g] = atomicMin(&a.label[cw[g].x], key[g] | kQueuedBit);
      }
    } else if (RX == kRelaxFilter) {
      // The same atomicMin, issued only where the label just loaded is
      // above the key (labels only fall, so a stale load can only let an
      // atomic through, never hold back a lowering one): where most
      // relaxations fail, as on power-law graphs, loads take the place of
      // atomics at L2; each lowering relaxation costs one round trip more.
#pragma unroll
      for (int g = 0; g < U; ++g) {
        prev[g] = 0;
        if (act[g] && key[g] < label_key(cur[g]))
          cur[g] = atomicMin(&a.label[cw[g].x], key[g] | kQueuedBit);
      }
    } else {
      // Load, then the first compare-and-swap of every group back to back
      // (the independent atomics overlap); a failed one (another lane
      // changed the label in between) retries through lower_label.
#pragma unroll
      for (int g = 0; g < U; ++g) {
        prev[g] = cur[g];
        if (act[g] && key[g] < label_key(cur[g]))
          prev[g] = (long long)atomicCAS((unsigned long long*)&a.label[cw[g].x],
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
            RX != kRelaxCas ? (key[g] < label_key(cur[g]) ? ((cur[g] & kQueuedBit) ? 1 : 2) : 0)
                        : (prev[g] == cur[g]) ? ((cur[g] & kQueuedBit) ? 1 : 2)
                                              : lower_label(&a.label[cw[g].x], key[g], prev[g]);
        if (r) {
          ++wc.upd;
          const unsigned nh = label_hops(key[g]);
          bool proven = nh >= V;          // a walk of >= V edges that still improved
          if (!proven && a.cyc && nh >= (a.cyc_walk0 >> 1)) {
            st_relaxed_u64((unsigned long long*)(a.cyc + cw[g].x),
                           (unsigned long long)pack_edge(st->tail[own[g]], cw[g].y));
            if (nh >= walk_at) {
              if (prove_negative_cycle(a.cyc, a.label, cw[g].x, a.V))
                proven = true;
              else
                walk_at = nh * 2;
            }
          }
          if (!proven) {
            enq[g] = (r == 2);
          } else if (a.mark_neg_inf) {
            // the head is reached from a negative cycle: minus infinity.  The
            // second lowering may claim the in-queue flag again if a consumer
            // took the vertex in between; either claim queues it once more.
            atomicOr(&a.ctl->status, kStNegCycle);
            const int r2 = lower_label(&a.label[cw[g].x], kNegInfLabel, key[g] | kQueuedBit);
            enq[g] = (r == 2) || (r2 == 2);
          } else {
            raise_status(a.ctl, kStNegCycle);
          }
        }
      }
    }
#pragma unroll
    for (int g = 0; g < U; ++g) {
      const unsigned m = __ballot_sync(kFullMask, enq[g]);
      if (m) {
        if (nbuf + __popc(m) > kChildBuf) {
          if (!flush_children(a, home, buf, nbuf, lane, wc)) return false;
        }
        if (enq[g]) buf[nbuf + __popc(m & lanemask_lt())] = (unsigned)cw[g].x;
        nbuf += __popc(m);
      }
    }
  }
  __syncwarp();                         // stage free for the next batch
  return true;
}

// Publish the hub chunks [c0_j, c0_j + nch_j) of the lanes with nch > 0 to
// the chunk sub-queues.  Chunks that find no room are relaxed right here.
template <int RX>
__device__ __forceinline__ bool push_chunks(const SsspArgs& a, int nch, int c0, int lane,
                                            int home, int chome, WarpCounters& wc,
                                            unsigned* buf, int& nbuf, unsigned& walk_at,
                                            BatchStage* st) {
  int K = 0;
  const int excl = warp_excl_scan(nch, lane, &K);
  if (K == 0) return true;
  if (lane == 0) red_add_relaxed_s32(&a.ctl->inflight, K);
  __syncwarp();
  for (int base = 0; base < K; base += 32) {
    const int t = base + lane;
    const int j = owner_lane(excl, t, 32);
    const int ex_j = __shfl_sync(kFullMask, excl, j);
    const int c0_j = __shfl_sync(kFullMask, c0, j);
    const bool act = t < K;
    const unsigned id = (unsigned)(c0_j + (t - ex_j));
    const int placed = enqueue_warp(a.cq, chome, act, id, lane, a.spin_limit, 2LL * a.cq.Q);
    if (placed < 0) return false;
    // leftovers (no room anywhere): relax them inline, one chunk at a time
    const unsigned act_mask = __ballot_sync(kFullMask, act);
    const int rank = __popc(act_mask & ((1u << lane) - 1u));
    unsigned left = __ballot_sync(kFullMask, act && rank >= placed);
    while (left) {
      const int src_lane = __ffs(left) - 1;
      left &= left - 1;
      const unsigned cid = __shfl_sync(kFullMask, id, src_lane);
      int beg = 0, deg = 0, tail = 0;
      long long lab = 0;
      if (lane == 0) {
        const int4 ct = a.chunk_tab[cid];
        beg = ct.y;
        deg = ct.z - ct.y;
        tail = ct.x;
        lab = label_key(ld_relaxed_s64(&a.label[ct.x]));
      }
      if (!relax_merged<kGroups, RX>(a, 1, beg, deg, lab, tail, lane, home, wc, buf, nbuf,
                                      walk_at, st) ||
          !flush_children(a, home, buf, nbuf, lane, wc))
        return false;
      if (lane == 0) red_add_relaxed_s32(&a.ctl->inflight, -1);
    }
  }
  return true;
}

// RX: the relaxation form (kRelax*, see relax_merged).  CTAS:
// the CTAs per SM the register budget is sized for: kCtasNarrow (64
// registers per thread, more warps in flight) or kCtasWide (80 registers,
// fewer spills; faster on low-degree graphs, whose warps spend more of each
// step in queue operations).  All six forms are compiled; the launcher
// picks one per run.
constexpr int kCtasNarrow = BFQ_MIN_CTAS_PER_SM;
constexpr int kCtasWide = 3;
template <int RX, int CTAS>
__global__ void __launch_bounds__(kBlock, CTAS) sssp_persistent_kernel(SsspArgs a) {
  const int lane = threadIdx.x & 31;
  const int wid = threadIdx.x >> 5;
  const int nwarps = blockDim.x >> 5;
  const int home = (blockIdx.x * a.queues_per_cta + wid % a.queues_per_cta) % a.qs.Q;
  const int chome = blockIdx.x % a.cq.Q;
  const int share = a.share_div > 0 ? a.share_div : max(1, nwarps / a.queues_per_cta);
  WarpCounters wc;
  const unsigned long long t_start = globaltimer_ns();
  unsigned rng = 0x9e3779b9u * (blockIdx.x * 64u + wid + 1u);
  int idle = 0;
  bool timed_out = false;

  __shared__ unsigned s_children[kBlock / 32][kChildBuf];
  __shared__ BatchStage s_stage[kBlock / 32];
  unsigned* buf = s_children[wid];
  BatchStage* st = &s_stage[wid];
  int nbuf = 0;
  unsigned walk_at = a.cyc_walk0;     // per lane: hops that trigger a cycle walk
  for (;;) {
    unsigned item = 0;
    int got = 0;
    bool is_chunk = false;
    // hub chunks first (they sit on the critical path), then the own vertex
    // sub-queue, then stealing; both home counts are read in one step
    // (the stop flag is read in the same step, so retiring a batch needs no
    // load of its own)
    int c = 0;
    if (lane == 0) c = ld_relaxed_s32(&a.cq.meta[chome].count);
    else if (lane == 1) c = ld_relaxed_s32(&a.qs.meta[home].count);
    else if (lane == 2) c = ld_relaxed_s32(&a.ctl->stop);
    const int c_chunk = __shfl_sync(kFullMask, c, 0);
    const int c_vert = __shfl_sync(kFullMask, c, 1);
    if (__shfl_sync(kFullMask, c, 2)) break;
    if (c_chunk > 0) {
      is_chunk = true;
      got = wq_dequeue_warp(a.cq, chome, a.chunk_batch, lane, &item, a.spin_limit, c_chunk);
    }
    if (got == 0 && c_vert > 0) {
      is_chunk = false;
      got = wq_dequeue_warp(a.qs, home, share_of(c_vert, a.batch_items, share), lane, &item,
                            a.spin_limit, c_vert);
    }
    if (got == 0) {
      rng = rng * 1664525u + 1013904223u;
      int q = probe_queues(a.cq, (int)(rng % (unsigned)a.cq.Q), chome, lane);
      if (q >= 0) {
        is_chunk = true;
        got = wq_dequeue_warp(a.cq, q, a.chunk_batch, lane, &item, a.spin_limit);
      } else {
        q = probe_queues(a.qs, (int)((rng >> 7) % (unsigned)a.qs.Q), home, lane);
        if (q >= 0) {
          is_chunk = false;
          int cq_cnt = 0;
          if (lane == 0) cq_cnt = ld_relaxed_s32(&a.qs.meta[q].count);
          cq_cnt = __shfl_sync(kFullMask, cq_cnt, 0);
          if (cq_cnt > 0)
            got = wq_dequeue_warp(a.qs, q, share_of(cq_cnt, a.batch_items, share), lane, &item,
                                  a.spin_limit, cq_cnt);
        }
      }
      if (got > 0) ++wc.steal;
    }
    if (got < 0) { timed_out = true; break; }
    if (got == 0) {
      // lane 0 decides whether the warp leaves (done, or out of time) and
      // the warp follows as one: lanes may run apart after a sleep
      int done = 0;
      if (lane == 0) {
        done = (ld_relaxed_s32(&a.ctl->inflight) == 0) || ld_relaxed_s32(&a.ctl->stop);
        if (!done && ((idle + 1) & 31) == 0 &&
            (long long)(globaltimer_ns() - t_start) > a.time_limit_ns)
          done = 2;
      }
      done = __shfl_sync(kFullMask, done, 0);
      if (done) {
        timed_out = done == 2;
        break;
      }
      ++wc.idle;
      __nanosleep(min(32u << min(idle, 6), 2048u));
      ++idle;
      continue;
    }
    idle = 0;
    wc.deq += (lane == 0) ? (unsigned)got : 0u;
    if (is_chunk) wc.chunk += (lane == 0) ? (unsigned)got : 0u;

    int beg = 0, deg = 0, nch = 0, c0 = 0, tail = 0;
    long long lab = 0;
    if (lane < got) {
      if (is_chunk) {
        const int4 ct = a.chunk_tab[item];
        beg = ct.y;
        deg = ct.z - ct.y;
        tail = ct.x;
        lab = label_key(ld_relaxed_s64(&a.label[ct.x]));
      } else {
        const unsigned u = item;
        tail = (int)u;
        // clear the in-queue flag and read the label in one atomic: any
        // later improvement sees the flag clear and queues u again
        lab = label_key((long long)atomicAnd((unsigned long long*)&a.label[u],
                                             ~(unsigned long long)kQueuedBit));
        beg = __ldg(&a.row_ptr[u]);
        deg = __ldg(&a.row_ptr[u + 1]) - beg;
        if (deg > a.hub_degree) {
          nch = (deg + a.chunk_edges - 1) / a.chunk_edges;
          c0 = __ldg(&a.hub_chunk0[u]);
          deg = 0;
        }
      }
    }
    if (__any_sync(kFullMask, nch > 0)) {
      if (!push_chunks<RX>(a, nch, c0, lane, home, chome, wc, buf, nbuf, walk_at, st)) {
        timed_out = true;
        break;
      }
    }
    // relax, then publish the children and retire the batch in one update
    // of the in-flight count: its children are counted before any becomes
    // visible, and the batch is done with; the labels are read by the
    // epilogue kernel, after this kernel has ended.
    if (!relax_merged<kGroups, RX>(a, got, beg, deg, lab, tail, lane, home, wc, buf, nbuf,
                                    walk_at, st) ||
        !flush_children(a, home, buf, nbuf, lane, wc, got)) {
      timed_out = true;
      break;
    }
  }
  if (timed_out && lane == 0) raise_status(a.ctl, kStTimeout);

  const unsigned long long upd_sum = warp_sum_u64(wc.upd);
  if (lane == 0) {
    if (wc.deq) atomicAdd(&a.ctl->ctr[kCtrDeq], (unsigned long long)wc.deq);
    if (wc.rel) atomicAdd(&a.ctl->ctr[kCtrRel], (unsigned long long)wc.rel);
    if (upd_sum) atomicAdd(&a.ctl->ctr[kCtrUpd], upd_sum);
    if (wc.enq) atomicAdd(&a.ctl->ctr[kCtrEnq], (unsigned long long)wc.enq);
    if (wc.steal) atomicAdd(&a.ctl->ctr[kCtrSteal], (unsigned long long)wc.steal);
    if (wc.chunk) atomicAdd(&a.ctl->ctr[kCtrChunk], (unsigned long long)wc.chunk);
    if (wc.idle) atomicAdd(&a.ctl->ctr[kCtrIdle], (unsigned long long)wc.idle);
  }
}

// Epilogue: unpack the labels into dist / hops (pred to -1 for the optional
// predecessor pass), and turn the status bits into the run's status code,
// also kept for the next run's init.  Runs after the persistent kernel, so
// every label write is visible; after an early stop the results are
// unspecified.
__global__ void sssp_epilogue_kernel(SsspArgs a, int32_t* status_dev, const int* bad) {
  const long long tid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const long long nth = (long long)gridDim.x * blockDim.x;
  for (long long v = tid; v < a.V; v += nth) {
    const long long l = a.label[v];
    const int d = label_dist(l);
    a.dist[v] = d;
    if (a.hops) a.hops[v] = (d == kInf32) ? -1 : (d == kNegInf32) ? -2 : (int)label_hops(l);
    if (a.pred) a.pred[v] = -1;
  }
  if (tid == 0) {
    const int st = a.ctl->status;
    int code = BFQ_OK;
    if (bad && *bad) code = BFQ_ERR_INVALID;
    else if (st & (kStTimeout | kStQueue)) code = BFQ_ERR_TIMEOUT;
    else if (a.mark_neg_inf && (st & kStRange)) code = BFQ_RANGE;   // labels incomplete
    else if (st & kStNegCycle) code = BFQ_NEG_CYCLE;
    else if (st & kStRange) code = BFQ_RANGE;
    a.ctl->last_status = code;
    if (status_dev) *status_dev = code;
  }
}

// Labels start at (INT32_MAX, -) and not queued, the source at (0, 0) and
// queued in vertex sub-queue 0.  If the previous run ended early
// (last_status != 0) all sub-queues are reset first; a clean run leaves every
// sub-queue empty and every in-queue flag clear.
__global__ void sssp_init_kernel(SsspArgs a) {
  const bool dirty = a.ctl->last_status != 0;
  const long long tid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const long long nth = (long long)gridDim.x * blockDim.x;
  for (long long v = tid; v < a.V; v += nth)
    a.label[v] = (v == a.src) ? (pack_label(0, 0) | kQueuedBit) : kInfLabel;
  if (dirty) {
    // every allocated sub-queue, also those a run of the other register form
    // used: a clean run leaves all of its sub-queues empty, so after this
    // reset the ones outside qs.Q / cq.Q stay empty for later runs
    const int q_all = a.q_alloc > 0 ? a.q_alloc : a.qs.Q;
    const int cq_all = a.cq_alloc > 0 ? a.cq_alloc : a.cq.Q;
    const long long nslots = (long long)q_all << a.qs.cap_log2;
    for (long long i = tid; i < nslots; i += nth)
      a.qs.slots[i] = (i == 0) ? ((1ull << 32) | (unsigned)a.src) : 0ull;
    const long long ncslots = (long long)cq_all << a.cq.cap_log2;
    for (long long i = tid; i < ncslots; i += nth) a.cq.slots[i] = 0ull;
    for (long long q = tid; q < q_all; q += nth) {
      a.qs.meta[q].count = (q == 0) ? 1 : 0;
      a.qs.meta[q].used = (q == 0) ? 1 : 0;
      a.qs.meta[q].head = 0;
      a.qs.meta[q].tail = (q == 0) ? 1 : 0;
    }
    for (long long q = tid; q < cq_all; q += nth) {
      a.cq.meta[q].count = 0;
      a.cq.meta[q].used = 0;
      a.cq.meta[q].head = 0;
      a.cq.meta[q].tail = 0;
    }
  } else if (tid == 0) {
    QueueMeta* m = a.qs.meta;
    const unsigned long long p = m->tail;
    const unsigned lap = (unsigned)(p >> a.qs.cap_log2);
    a.qs.slots[p & ((1ull << a.qs.cap_log2) - 1)] =
        ((unsigned long long)(2u * lap + 1u) << 32) | (unsigned)a.src;
    m->tail = p + 1;
    m->count = 1;
    m->used = 1;          // one place taken (single-shot form; unused otherwise)
  }
  if (tid == 0) {
    a.ctl->inflight = 1 + a.phantom;
    a.ctl->status = 0;
    a.ctl->stop = 0;
    for (int i = 0; i < 8; ++i) a.ctl->ctr[i] = 0;
  }
}

// Predecessor post-pass: for each reached u and edge (u, v, w) with
// dist[u] + w == dist[v] and hops[u] + 1 == hops[v], pred[v] = u.  Any such u
// is valid; following pred strictly lowers hops, so the tree is acyclic.
__global__ void sssp_pred_kernel(const int* __restrict__ row_ptr, const int2* __restrict__ adj,
                                 const long long* __restrict__ label, int V, int* pred,
                                 const Control* ctl, int allow_neg_cycle) {
  // labels are final after a clean run, and after a run that resolved its
  // negative cycles (minus-infinity vertices match no tight edge below)
  if (ctl && ctl->last_status != 0 &&
      !(allow_neg_cycle && ctl->last_status == BFQ_NEG_CYCLE))
    return;
  const int lane = threadIdx.x & 31;
  const long long warp = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const long long nw = ((long long)gridDim.x * blockDim.x) >> 5;
  for (long long u = warp; u < V; u += nw) {
    const long long lu = label_key(label[u]);
    if (label_dist(lu) == kInf32 || label_dist(lu) == kNegInf32) continue;
    const int b = row_ptr[u], e = row_ptr[u + 1];
    for (int i = b + lane; i < e; i += 32) {
      const int2 cw = adj[i];
      const long long nd = (long long)label_dist(lu) + cw.y;
      if (nd >= kInf32) continue;
      const long long lv = label_key(label[cw.x]);
      if (label_dist(lv) == (int)nd && label_hops(lv) == label_hops(lu) + 1u) pred[cw.x] = (int)u;
    }
  }
}

__global__ void reached_edges_kernel(const int* __restrict__ row_ptr,
                                     const long long* __restrict__ label, int V,
                                     unsigned long long* out2) {
  unsigned long long m = 0, r = 0;
  for (long long v = (long long)blockIdx.x * blockDim.x + threadIdx.x; v < V;
       v += (long long)gridDim.x * blockDim.x) {
    if (label_dist(label[v]) != kInf32) {
      m += (unsigned long long)(row_ptr[v + 1] - row_ptr[v]);
      ++r;
    }
  }
  m = warp_sum_u64(m);
  r = warp_sum_u64(r);
  if ((threadIdx.x & 31) == 0) {
    atomicAdd(&out2[0], m);
    atomicAdd(&out2[1], r);
  }
}

__global__ void pack_adj_kernel(const int* __restrict__ col, const int* __restrict__ w,
                                int2* __restrict__ adj, long long E) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < E;
       i += (long long)gridDim.x * blockDim.x)
    adj[i] = make_int2(col[i], w[i]);
}

__global__ void validate_csr_kernel(const int* __restrict__ row_ptr, const int* __restrict__ col,
                                    int V, long long E, int* bad) {
  const long long tid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const long long nth = (long long)gridDim.x * blockDim.x;
  if (tid == 0 && (row_ptr[0] != 0 || (long long)row_ptr[V] != E)) atomicOr(bad, 1);
  for (long long v = tid; v < V; v += nth)
    if (row_ptr[v + 1] < row_ptr[v]) atomicOr(bad, 2);
  for (long long i = tid; i < E; i += nth)
    if (col[i] < 0 || col[i] >= V) atomicOr(bad, 4);
}

__global__ void queue_reset_kernel(QueueSet qs) {
  const long long tid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const long long nth = (long long)gridDim.x * blockDim.x;
  const long long n = (long long)qs.Q << qs.cap_log2;
  for (long long i = tid; i < n; i += nth) qs.slots[i] = 0ull;
  for (long long q = tid; q < qs.Q; q += nth) {
    qs.meta[q].count = 0;
    qs.meta[q].used = 0;
    qs.meta[q].head = 0;
    qs.meta[q].tail = 0;
  }
}

// The persistent kernel in the form a.relax_min / a.wide name, with the L2
// access-policy window as a launch attribute when one is given.
template <int RX, int CTAS>
cudaError_t launch_persistent_as(const SsspArgs& a, LaunchShape sh, cudaStream_t s,
                                 const cudaAccessPolicyWindow* l2win) {
  if (!l2win) {
    sssp_persistent_kernel<RX, CTAS><<<sh.grid, sh.block, 0, s>>>(a);
    return cudaGetLastError();
  }
  cudaLaunchConfig_t cfg{};
  cfg.gridDim = dim3(sh.grid);
  cfg.blockDim = dim3(sh.block);
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeAccessPolicyWindow;
  attr[0].val.accessPolicyWindow = *l2win;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, sssp_persistent_kernel<RX, CTAS>, a);
}

cudaError_t launch_persistent(const SsspArgs& a, LaunchShape sh, cudaStream_t s,
                              const cudaAccessPolicyWindow* l2win) {
  switch (a.relax_min * 2 + (a.wide ? 1 : 0)) {
    case 0: return launch_persistent_as<kRelaxCas, kCtasNarrow>(a, sh, s, l2win);
    case 1: return launch_persistent_as<kRelaxCas, kCtasWide>(a, sh, s, l2win);
    case 2: return launch_persistent_as<kRelaxMin, kCtasNarrow>(a, sh, s, l2win);
    case 3: return launch_persistent_as<kRelaxMin, kCtasWide>(a, sh, s, l2win);
    case 4: return launch_persistent_as<kRelaxFilter, kCtasNarrow>(a, sh, s, l2win);
    case 5: return launch_persistent_as<kRelaxFilter, kCtasWide>(a, sh, s, l2win);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace

int sssp_max_ctas_per_sm(int block, int wide) {
  int n = 0;
  const cudaError_t e =
      wide ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(
                 &n, sssp_persistent_kernel<kRelaxMin, kCtasWide>, block, 0)
           : cudaOccupancyMaxActiveBlocksPerMultiprocessor(
                 &n, sssp_persistent_kernel<kRelaxMin, kCtasNarrow>, block, 0);
  if (e != cudaSuccess) return 1;
  return n < 1 ? 1 : n;
}

cudaError_t launch_sssp(const SsspArgs& a, LaunchShape init_shape, LaunchShape run_shape,
                        int32_t* status_dev, cudaEvent_t ev0, cudaEvent_t ev1,
                        cudaStream_t s, const cudaAccessPolicyWindow* l2win) {
  sssp_init_kernel<<<init_shape.grid, init_shape.block, 0, s>>>(a);
  if (ev0) cudaEventRecord(ev0, s);
  const cudaError_t e = launch_persistent(a, run_shape, s, l2win);
  if (e != cudaSuccess) return e;
  if (ev1) cudaEventRecord(ev1, s);
  sssp_epilogue_kernel<<<init_shape.grid, init_shape.block, 0, s>>>(a, status_dev, nullptr);
  if (a.pred)
    sssp_pred_kernel<<<init_shape.grid, init_shape.block, 0, s>>>(a.row_ptr, a.adj, a.label, a.V,
                                                                 a.pred, a.ctl, a.mark_neg_inf);
  return cudaGetLastError();
}

cudaError_t launch_pred_pass(const int* row_ptr, const int2* adj, const long long* label, int V,
                             int* pred, cudaStream_t s) {
  sssp_pred_kernel<<<1024, 256, 0, s>>>(row_ptr, adj, label, V, pred, nullptr, 0);
  return cudaGetLastError();
}

cudaError_t launch_sssp_pred(const SsspArgs& a, cudaStream_t s) {
  sssp_pred_kernel<<<1024, 256, 0, s>>>(a.row_ptr, a.adj, a.label, a.V, a.pred, a.ctl,
                                        a.mark_neg_inf);
  return cudaGetLastError();
}

cudaError_t launch_reached_edges(const int* row_ptr, const long long* label, int V,
                                 unsigned long long* out2, cudaStream_t s) {
  cudaError_t e = cudaMemsetAsync(out2, 0, 2 * sizeof(unsigned long long), s);
  if (e != cudaSuccess) return e;
  reached_edges_kernel<<<1024, 256, 0, s>>>(row_ptr, label, V, out2);
  return cudaGetLastError();
}

cudaError_t launch_pack_adj(const int* col, const int* w, int2* adj, long long E, cudaStream_t s) {
  if (E == 0) return cudaSuccess;
  pack_adj_kernel<<<2048, 256, 0, s>>>(col, w, adj, E);
  return cudaGetLastError();
}

cudaError_t launch_validate_csr(const int* row_ptr, const int* col, int V, long long E, int* bad,
                                cudaStream_t s) {
  validate_csr_kernel<<<1024, 256, 0, s>>>(row_ptr, col, V, E, bad);
  return cudaGetLastError();
}

cudaError_t launch_queue_reset(QueueSet qs, cudaStream_t s) {
  queue_reset_kernel<<<1024, 256, 0, s>>>(qs);
  return cudaGetLastError();
}

cudaError_t launch_sssp_persistent_only(const SsspArgs& a, LaunchShape run_shape,
                                        cudaStream_t s) {
  return launch_persistent(a, run_shape, s, nullptr);
}

cudaError_t launch_sssp_epilogue(const SsspArgs& a, LaunchShape shape, int32_t* status_dev,
                                 const int* bad, cudaStream_t s) {
  sssp_epilogue_kernel<<<shape.grid, shape.block, 0, s>>>(a, status_dev, bad);
  return cudaGetLastError();
}

}  // namespace bfq
