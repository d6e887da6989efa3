// Serving: continuous batching of single-source queries on a resident
// persistent kernel (the queue-driven relaxation of Sec. III-C, fed by a
// request stream).
//
// The host admission thread keeps submitted requests in FIFO order and admits
// one when a slot is free and the label pool (the device-memory budget) has a
// contiguous page run for its V labels.  It writes an admission command into
// a ring in mapped pinned host memory.  On the device, a warp that finds no
// work takes the next command and turns it into init tasks (labels of the
// slot's run to infinity, page owners); the last init task queues the source.
// From then on the query's vertices and hub chunks flow through the same
// sub-queues as every other running query, so requests that arrive while
// others run overlap with them on the device.  When a query's in-flight count
// reaches zero its unpack tasks write dist/hops, and the last one posts a
// completion record to a second mapped ring, which the host thread consumes
// (freeing the slot and the pages).
//
// Every device wait is bounded.  The kernel leaves when the host asks it to,
// after idle_exit_ms without work, or after time_limit_ms; the host relaunches
// it when there is work again, and the device state carries over.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <new>
#include <thread>
#include <unordered_map>
#include <vector>

#include "sssp_multi.cuh"

namespace bfq {

struct GraphView {
  const int* row_ptr;
  const int2* adj;
  const int* hub_chunk0;
  const int4* chunk_tab;
  int V, n_chunks, hub_degree, chunk_edges;
};
int graph_view(bfq_graph_t g, GraphView* out);

namespace {

constexpr int kPageLog2 = 12;            // label pool page: 4096 labels
constexpr int kTaskLog2 = 14;            // init / unpack task: 16384 labels
constexpr int kMaxHelpers = 128;         // helper items queued per init / unpack phase
constexpr int kChunkIdBits = 20;         // chunk item = slot << 20 | chunk
constexpr int kMaxSlots = 2048;          // 11 bits of slot in task items

struct alignas(16) SlotDesc {
  const int* row_ptr;
  const int2* adj;
  const int* hub_chunk0;
  const int4* chunk_tab;
  int* dist;
  int* hops;
  int V, src, hub_degree, chunk_edges;
  int label_off, n_tasks, n_chunks, pad0;
  long long req_id;
  long long pad1;
};

struct alignas(16) ServeCmd {            // mapped host memory, host -> device
  SlotDesc d;
  int slot;
  unsigned seq;                          // position + 1, written last
  int pad[2];
};

struct alignas(16) ServeDone {           // mapped host memory, device -> host
  long long req_id;
  unsigned long long t_gpu_ns;
  int slot, status;
  unsigned seq;                          // position + 1, written last
  int pad;
};

struct alignas(128) ServeCtl {
  unsigned cmd_head;                     // next command to take
  int pad0[31];
  unsigned done_tail;                    // next completion record to fill
  int pad1[31];
  int active;                            // admitted, not yet completed
  int pad2[31];
  int stop;
  int pad3[31];
  int status;                            // kSt* bits of the launch
  int pad4[31];
  unsigned long long ctr[8];
  unsigned long long pad5[8];
  int bad_where;                         // first failed range check (0 = none)
  unsigned bad_value;
  int pad6[30];
  unsigned long long poll_ns;            // last look at the host rings (0: look now)
  unsigned long long pad7[15];
};

// Reads of the mapped host rings cross the chip-to-host link; at most one
// warp looks at a time, and not more often than this.
constexpr unsigned long long kHostPollGapNs = 2000;

// Claim the next look at the host memory: true for one warp per gap.
__device__ __forceinline__ bool claim_host_poll(ServeCtl* ctl) {
  const unsigned long long now = globaltimer_ns();
  const unsigned long long last = ld_relaxed_u64(&ctl->poll_ns);
  if (last != 0 && now - last < kHostPollGapNs) return false;
  return atomicCAS(&ctl->poll_ns, last, now) == last;
}

struct ServeArgs {
  SlotDesc* slots;                       // [S]
  int* inflight;                         // [S * kCounterStride]
  int* qstatus;                          // [S]
  int* pending;                          // [S * kCounterStride] init/unpack tasks left
  int* page_owner;                       // [pool pages]
  long long* label;                      // pool
  long long* cyc;                        // recorded relaxation edges, like the pool
  QueueSet qs, cq, tq;                   // vertices, hub chunks, tasks
  ServeCmd* cmd;                         // mapped ring [R]
  ServeDone* done;                       // mapped ring [R]
  const int* shutdown;                   // mapped flag
  ServeCtl* ctl;
  int ring;
  int max_slots;
  int pool_pages;
  int queues_per_cta;
  int share_div, chunk_batch, batch_items;
  unsigned cyc_walk0;                    // first cycle-walk threshold (hops)
  long long spin_limit, time_limit_ns, idle_exit_ns;
};

__device__ __forceinline__ int ld_acquire_sys_s32(const int* p) {
  int v;
  asm volatile("ld.acquire.sys.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ unsigned ld_acquire_sys_u32(const unsigned* p) {
  unsigned v;
  asm volatile("ld.acquire.sys.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void st_release_sys_u32(unsigned* p, unsigned v) {
  asm volatile("st.release.sys.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ int atom_add_acq_rel_s32(int* p, int v) {
  int old;
  asm volatile("atom.acq_rel.gpu.global.add.s32 %0, [%1], %2;"
               : "=r"(old) : "l"(p), "r"(v) : "memory");
  return old;
}

__device__ __forceinline__ void serve_fail(const ServeArgs& a) {
  atomicOr(&a.ctl->status, kStTimeout);
  st_relaxed_s32(&a.ctl->stop, 1);
}

// A decoded item or task out of range: record the first one, stop the
// launch, and let the caller skip the access.
__device__ __noinline__ void serve_bad(const ServeArgs& a, int where, unsigned value) {
  if (atomicCAS(&a.ctl->bad_where, 0, where) == 0) a.ctl->bad_value = value;
  atomicOr(&a.ctl->status, kStQueue);
  st_relaxed_s32(&a.ctl->stop, 1);
}

// Publish `n` helper items (kind, slot, 0..n-1) to the task queue.
__device__ __forceinline__ bool push_tasks(const ServeArgs& a, int kind, int slot, int n,
                                           int lane) {
  for (int base = 0; base < n; base += 32) {
    const int t = base + lane;
    const bool act = t < n;
    const unsigned id = ((unsigned)kind << 30) | ((unsigned)slot << 19) | (unsigned)t;
    const int placed = enqueue_warp(a.tq, 0, act, id, lane, a.spin_limit, 64);
    if (placed != min(32, n - base)) return false;
  }
  return true;
}

// Take the next admission command, if one is ready, into its slot.
__device__ __forceinline__ bool admit_one(const ServeArgs& a, int lane) {
  int slot = -1, n_tasks = 0;
  if (lane == 0 && claim_host_poll(a.ctl)) {
    const unsigned pos = ld_relaxed_s32((const int*)&a.ctl->cmd_head);
    ServeCmd* c = a.cmd + (pos % (unsigned)a.ring);
    if (ld_acquire_sys_u32(&c->seq) == pos + 1 &&
        atomicCAS(&a.ctl->cmd_head, pos, pos + 1) == pos) {
      st_relaxed_u64(&a.ctl->poll_ns, 0ull);   // commands come in bursts: look again now
      slot = c->slot;
      SlotDesc d = c->d;
      d.n_tasks = (d.V + (1 << kTaskLog2) - 1) >> kTaskLog2;
      a.slots[slot] = d;
      a.qstatus[slot] = 0;
      a.inflight[slot * kCounterStride] = 0;
      n_tasks = min(d.n_tasks, kMaxHelpers);        // helper items
      a.pending[slot * kCounterStride] = n_tasks;
      a.pending[slot * kCounterStride + 1] = 0;     // task cursor
      atomicAdd(&a.ctl->active, 1);
      __threadfence();               // slot state before its tasks are visible
    }
  }
  __syncwarp();
  slot = __shfl_sync(kFullMask, slot, 0);
  if (slot < 0) return false;
  n_tasks = __shfl_sync(kFullMask, n_tasks, 0);
  if (!push_tasks(a, 0, slot, n_tasks, lane)) serve_fail(a);
  return true;
}

// Init and unpack phases of a slot: the slot's V labels are cut into tasks
// of 16384; the phase queues min(tasks, kMaxHelpers) helper items, and a warp
// holding one claims tasks from the slot's cursor (pending[slot * stride + 1],
// an atomicAdd, no retries) until none is left, so a large graph needs few
// queue operations.  The phase ends when every helper has left (helpers'
// count in pending[slot * stride]); no helper of it is running afterwards,
// so the slot's next phase may reset the cursor.
// Init task: labels of [t * 16384, ...) to infinity (the source to (0, 0),
// queued), page owners; the last helper queues the source.
// Unpack task: dist / hops out; the last helper posts the completion.
__device__ __forceinline__ bool run_task(const ServeArgs& a, unsigned id, int lane, int home) {
  const int kind = (int)(id >> 30);
  const int slot = (int)((id >> 19) & (kMaxSlots - 1));
  const int h = (int)(id & ((1u << 19) - 1));
  if (slot >= a.max_slots) {
    if (lane == 0) serve_bad(a, 1, id);
    return false;
  }
  const SlotDesc d = a.slots[slot];
  if (h >= kMaxHelpers || d.label_off < 0 ||
      ((long long)d.label_off + d.V) > ((long long)a.pool_pages << kPageLog2)) {
    if (lane == 0) serve_bad(a, 2, id);
    return false;
  }
  long long* lab = a.label + d.label_off;
  for (;;) {
    int t = 0;
    if (lane == 0) t = atomicAdd(&a.pending[slot * kCounterStride + 1], 1);
    t = __shfl_sync(kFullMask, t, 0);
    if (t >= d.n_tasks) break;
    const int lo = t << kTaskLog2;
    const int hi = min(d.V, lo + (1 << kTaskLog2));
    if (kind == 0) {
      for (int i = lo + lane; i < hi; i += 32)
        lab[i] = (i == d.src) ? (pack_label(0, 0) | kQueuedBit) : kInfLabel;
      const int p0 = (d.label_off + lo) >> kPageLog2, p1 = (d.label_off + hi - 1) >> kPageLog2;
      for (int p = p0 + lane; p <= p1; p += 32) a.page_owner[p] = slot;
    } else if (d.dist || d.hops) {
      // sixteen labels in flight per lane, read as 16-byte pairs (the slot's
      // labels start on a page, so even indices are 16-byte aligned)
      for (int i0 = lo + 2 * lane; i0 < hi; i0 += 64 * 8) {
        long long l[16];
#pragma unroll
        for (int k = 0; k < 8; ++k) {
          const int i = i0 + 64 * k;
          if (i + 1 < hi) {
            const longlong2 v = *reinterpret_cast<const longlong2*>(lab + i);
            l[2 * k] = v.x;
            l[2 * k + 1] = v.y;
          } else {
            l[2 * k] = (i < hi) ? lab[i] : 0;
            l[2 * k + 1] = 0;
          }
        }
#pragma unroll
        for (int k = 0; k < 16; ++k) {
          const int i = i0 + 64 * (k >> 1) + (k & 1);
          if (i >= hi) continue;
          const int dd = label_dist(l[k]);
          if (d.dist) d.dist[i] = dd;
          if (d.hops) d.hops[i] = (dd == kInf32) ? -1 : (int)label_hops(l[k]);
        }
      }
    }
  }
  __syncwarp();
  int last = 0;
  if (lane == 0) last = atom_add_acq_rel_s32(&a.pending[slot * kCounterStride], -1) == 1;
  last = __shfl_sync(kFullMask, last, 0);
  if (!last) return true;
  if (kind == 0) {
    // every init write is ordered before this point (acq_rel chain); the
    // source becomes visible only after its in-flight count
    unsigned src_item = (unsigned)(d.label_off + d.src);
    if (lane == 0) a.inflight[slot * kCounterStride] = 1;
    __syncwarp();
    return enqueue_warp(a.qs, home, lane == 0, src_item, lane, a.spin_limit,
                        4LL * a.qs.Q + 64) == 1;
  }
  if (lane == 0) {
    const int st = a.qstatus[slot];
    int code = BFQ_OK;
    if (st & kStNegCycle) code = BFQ_NEG_CYCLE;
    else if (st & kStRange) code = BFQ_RANGE;
    __threadfence_system();
    const unsigned pos = atomicAdd(&a.ctl->done_tail, 1u);
    ServeDone* r = a.done + (pos % (unsigned)a.ring);
    r->req_id = d.req_id;
    r->t_gpu_ns = globaltimer_ns();
    r->slot = slot;
    r->status = code;
    st_release_sys_u32(&r->seq, pos + 1);
    atomicAdd(&a.ctl->active, -1);
  }
  return true;
}

__global__ void __launch_bounds__(kBlock, BFQ_MULTI_CTAS_PER_SM) serve_kernel(ServeArgs a) {
  __shared__ unsigned s_children[kBlock / 32][kChildBuf];
  __shared__ unsigned short s_childq[kBlock / 32][kChildBuf];
  __shared__ MultiStage s_mstage[kBlock / 32];
  const int lane = threadIdx.x & 31;
  const int wid = threadIdx.x >> 5;
  const int nwarps = blockDim.x >> 5;
  const int home = (blockIdx.x * a.queues_per_cta + wid % a.queues_per_cta) % a.qs.Q;
  const int chome = blockIdx.x % a.cq.Q;
  const int share = a.share_div > 0 ? a.share_div : max(1, nwarps / a.queues_per_cta);
  unsigned* buf = s_children[wid];
  unsigned short* bufq = s_childq[wid];
  int nbuf = 0;
  WarpCounters wc;
  const MultiEnv env{a.label, a.cyc, a.inflight, a.qstatus, &a.ctl->status, &a.ctl->stop,
                     a.qs, a.spin_limit, a.cyc_walk0};
  unsigned walk_at = env.cyc_walk0;     // per lane: hops that trigger a cycle walk
  const unsigned long long t_start = globaltimer_ns();
  unsigned long long t_idle = t_start;
  unsigned rng = 0x9e3779b9u * (blockIdx.x * 64u + wid + 1u);
  int idle = 0;
  bool failed = false;

  int since_admit = 0;
  for (;;) {
    // 0) busy warps also take admissions now and then, so that arrivals do
    // not wait for the device to run dry
    if (++since_admit >= 16) {
      since_admit = 0;
      if (admit_one(a, lane)) idle = 0;
    }
    // 1) init / unpack tasks (the one task sub-queue is looked at every
    // eighth step of a busy warp: its counter line is shared by all warps)
    unsigned item = 0;
    int c = 0;
    if (lane == 0) c = ((since_admit & 7) == 0 || idle) ? ld_relaxed_s32(&a.tq.meta[0].count) : 0;
    else if (lane == 1) c = ld_relaxed_s32(&a.cq.meta[chome].count);
    else if (lane == 2) c = ld_relaxed_s32(&a.qs.meta[home].count);
    const int c_task = __shfl_sync(kFullMask, c, 0);
    const int c_chunk = __shfl_sync(kFullMask, c, 1);
    const int c_vert = __shfl_sync(kFullMask, c, 2);
    if (c_task > 0) {
      const int g = wq_dequeue_warp(a.tq, 0, 1, lane, &item, a.spin_limit, c_task);
      if (g < 0) { failed = true; break; }
      if (g == 1) {
        const unsigned id = __shfl_sync(kFullMask, item, 0);
        if (!run_task(a, id, lane, home)) { failed = true; break; }
        idle = 0;
        continue;
      }
    }
    // 2) hub chunks, then vertices (own sub-queue, then stealing)
    int got = 0;
    bool is_chunk = false;
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
          int cnt = 0;
          if (lane == 0) cnt = ld_relaxed_s32(&a.qs.meta[q].count);
          cnt = __shfl_sync(kFullMask, cnt, 0);
          if (cnt > 0)
            got = wq_dequeue_warp(a.qs, q, share_of(cnt, a.batch_items, share), lane, &item,
                                  a.spin_limit, cnt);
        }
      }
      if (got > 0) ++wc.steal;
    }
    if (got < 0) { failed = true; break; }
    if (got == 0) {
      // 3) admission, then idle
      if (admit_one(a, lane)) { idle = 0; continue; }
      if (idle == 0) t_idle = globaltimer_ns();
      // leaving is decided for the whole launch (a warp sets the stop flag,
      // every warp follows), so the kernel never lingers with a few warps
      int leave = 0;
      if (lane == 0) {
        const unsigned long long now = globaltimer_ns();
        if (ld_relaxed_s32(&a.ctl->stop)) {
          leave = 1;
        } else if ((claim_host_poll(a.ctl) && ld_acquire_sys_s32(a.shutdown)) ||
                   (long long)(now - t_start) > a.time_limit_ns ||
                   (ld_relaxed_s32(&a.ctl->active) == 0 &&
                    (long long)(now - t_idle) > a.idle_exit_ns)) {
          st_relaxed_s32(&a.ctl->stop, 1);
          leave = 1;
        }
      }
      if (__shfl_sync(kFullMask, leave, 0)) break;
      ++wc.idle;
      __nanosleep(min(32u << min(idle, 5), 1024u));
      ++idle;
      continue;
    }
    idle = 0;
    wc.deq += (lane == 0) ? (unsigned)got : 0u;
    if (is_chunk) wc.chunk += (lane == 0) ? (unsigned)got : 0u;

    int q = -1, deg = 0, nch = 0, c0 = 0, Vq = 0, tail = 0;
    long long lab = 0;
    long long* lbase = nullptr;
    const int2* eptr = nullptr;
    bool bad = false;
    if (lane < got) {
      if (is_chunk) {
        q = (int)(item >> kChunkIdBits);
        const unsigned ci = item & ((1u << kChunkIdBits) - 1);
        if (q >= a.max_slots || (int)ci >= a.slots[q].n_chunks) {
          serve_bad(a, 3, item);
          bad = true;
        } else {
          const SlotDesc& d = a.slots[q];
          const int4 ct = d.chunk_tab[ci];
          tail = ct.x;
          lbase = a.label + d.label_off;
          lab = label_key(ld_relaxed_s64(lbase + ct.x));
          eptr = d.adj + ct.y;
          deg = ct.z - ct.y;
          Vq = d.V;
        }
      } else {
        // the item is a pool index: its page names the slot (each load once)
        const unsigned page = item >> kPageLog2;
        const int po = page < (unsigned)a.pool_pages ? a.page_owner[page] : -1;
        const SlotDesc* dp = a.slots + ((unsigned)po < (unsigned)a.max_slots ? po : 0);
        const int loff = dp->label_off, Vd = dp->V;
        const int u = (int)item - loff;
        if ((unsigned)po >= (unsigned)a.max_slots || u < 0 || u >= Vd) {
          serve_bad(a, 4, item);
          bad = true;
        } else {
          q = po;
          tail = u;
          lbase = a.label + loff;
          lab = label_key((long long)atomicAnd((unsigned long long*)(lbase + u),
                                               ~(unsigned long long)kQueuedBit));
          const int* rp = dp->row_ptr;
          const int beg = __ldg(rp + u);
          deg = __ldg(rp + u + 1) - beg;
          eptr = dp->adj + beg;
          Vq = Vd;
          if (deg > dp->hub_degree) {
            nch = (deg + dp->chunk_edges - 1) / dp->chunk_edges;
            c0 = (q << kChunkIdBits) + __ldg(dp->hub_chunk0 + u);
            deg = 0;
          }
        }
      }
      if (!bad && (ld_relaxed_s32(&a.qstatus[q]) & (kStNegCycle | kStRange))) {
        deg = 0;
        nch = 0;
      }
    }
    if (__any_sync(kFullMask, bad)) break;      // the launch stops; nothing was touched
    if (__any_sync(kFullMask, nch > 0)) {
      const int qn = nch > 0 ? q : -1;
      const unsigned m = __match_any_sync(kFullMask, qn);
      const int sum_q = (int)__reduce_add_sync(m, (unsigned)nch);
      if (qn >= 0 && lane == __ffs(m) - 1)
        red_add_relaxed_s32(&a.inflight[qn * kCounterStride], sum_q);
      __syncwarp();
      int K = 0;
      const int excl = warp_excl_scan(nch, lane, &K);
      for (int base = 0; base < K && !failed; base += 32) {
        const int t = base + lane;
        const int j = owner_lane(excl, t, 32);
        const int ex_j = __shfl_sync(kFullMask, excl, j);
        const int c0_j = __shfl_sync(kFullMask, c0, j);
        const bool act = t < K;
        const unsigned id = (unsigned)(c0_j + (t - ex_j));
        const int placed = enqueue_warp(a.cq, chome, act, id, lane, a.spin_limit, 2LL * a.cq.Q);
        if (placed < 0) { failed = true; break; }
        const unsigned act_mask = __ballot_sync(kFullMask, act);
        const int rank = __popc(act_mask & ((1u << lane) - 1u));
        unsigned left = __ballot_sync(kFullMask, act && rank >= placed);
        while (left) {
          const unsigned cid = __shfl_sync(kFullMask, id, __ffs(left) - 1);
          left &= left - 1;
          int cs = -1, cdeg = 0, cV = 0, ctail = 0;
          long long clab = 0;
          long long* clb = nullptr;
          const int2* cep = nullptr;
          if (lane == 0) {
            cs = (int)(cid >> kChunkIdBits);
            const SlotDesc& d = a.slots[cs];
            const int4 ct = d.chunk_tab[cid & ((1u << kChunkIdBits) - 1)];
            clb = a.label + d.label_off;
            clab = label_key(ld_relaxed_s64(clb + ct.x));
            cep = d.adj + ct.y;
            cdeg = ct.z - ct.y;
            cV = d.V;
            ctail = ct.x;
          }
          if (!relax_multi<kMultiGroups, false>(env, 1, cep, cdeg, clab, clb, cV, cs, ctail, lane, home, wc,
                                    buf, bufq, nbuf, walk_at, &s_mstage[wid]) ||
              !flush_multi(env, home, buf, bufq, nbuf, lane, wc)) {
            failed = true;
            break;
          }
          __syncwarp();
          if (lane == 0) red_add_relaxed_s32(&a.inflight[cs * kCounterStride], -1);
        }
      }
      if (failed) break;
    }
    if (!relax_multi<kMultiGroups, false>(env, got, eptr, deg, lab, lbase, Vq, q, tail, lane, home, wc,
                              buf, bufq, nbuf, walk_at, &s_mstage[wid]) ||
        !flush_multi(env, home, buf, bufq, nbuf, lane, wc)) {
      failed = true;
      break;
    }
    __syncwarp();
    const int emptied = retire_multi(env, lane < got ? q : -1, lane);
    // queries this batch finished: queue their unpack tasks
    unsigned fin = __ballot_sync(kFullMask, emptied >= 0);
    while (fin) {
      const int src_lane = __ffs(fin) - 1;
      fin &= fin - 1;
      const int s = __shfl_sync(kFullMask, emptied, src_lane);
      int n_tasks = 0;
      if (lane == 0) {
        n_tasks = min(a.slots[s].n_tasks, kMaxHelpers);   // helper items
        a.pending[s * kCounterStride] = n_tasks;
        a.pending[s * kCounterStride + 1] = 0;              // task cursor
        __threadfence();
      }
      __syncwarp();
      n_tasks = __shfl_sync(kFullMask, n_tasks, 0);
      if (!push_tasks(a, 1, s, n_tasks, lane)) { failed = true; break; }
    }
    if (failed) break;
    int stop = 0;
    if (lane == 0) stop = ld_relaxed_s32(&a.ctl->stop);
    if (__shfl_sync(kFullMask, stop, 0)) break;
  }
  if (failed && lane == 0) serve_fail(a);
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

__global__ void serve_reset_kernel(ServeArgs a) {
  const long long tid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const long long nth = (long long)gridDim.x * blockDim.x;
  const QueueSet* sets[3] = {&a.qs, &a.cq, &a.tq};
  for (int k = 0; k < 3; ++k) {
    const QueueSet& s = *sets[k];
    const long long n = (long long)s.Q << s.cap_log2;
    for (long long i = tid; i < n; i += nth) s.slots[i] = 0ull;
    for (long long q = tid; q < s.Q; q += nth) {
      s.meta[q].count = 0; s.meta[q].head = 0; s.meta[q].tail = 0;
    }
  }
  if (tid == 0) {
    a.ctl->active = 0;
    a.ctl->stop = 0;
    a.ctl->status = 0;
    a.ctl->poll_ns = 0;
  }
}

int ceil_log2_s(long long x) {
  int l = 0;
  while ((1LL << l) < x) ++l;
  return l;
}

}  // namespace
}  // namespace bfq

using namespace bfq;

struct ServeRequest {
  int64_t id;
  int graph;
  int src;
  int32_t* dist;
  int32_t* hops;
  int64_t t_submit;
};

struct ServeRecord {
  int status = BFQ_PENDING;
  int64_t t_submit = 0, t_done = 0;
};

struct bfq_server {
  std::vector<bfq_graph_t> graphs;
  std::vector<GraphView> views;
  int S = 0;
  int ring = 0;
  long long pool_entries = 0;
  bfq_tune tune{};
  ServeArgs args{};
  ServeCmd* cmd_host = nullptr;
  ServeDone* done_host = nullptr;
  int* shutdown_host = nullptr;
  cudaStream_t stream = nullptr;
  cudaEvent_t kernel_done = nullptr;
  bool launched = false;
  int grid = 0;
  int device = 0;
  std::vector<void*> dev_allocs;
  // host-side state (mutex-protected)
  std::mutex mu;
  std::condition_variable cv;
  std::deque<ServeRequest> pending;
  std::unordered_map<int64_t, ServeRecord> records;
  struct Admitted {
    int slot;
    long long start, pages;    // page run of its labels
    bool large;
  };
  std::unordered_map<int64_t, Admitted> admitted;
  // Requests whose labels exceed a quarter of L2 keep a GPU busy alone and,
  // run side by side, push each other's labels out of L2: at most one runs
  // at a time, and smaller requests may pass one that waits for its turn.
  long long large_vertices = 0;
  int large_active = 0;
  // The other requests are admitted while their labels fit a budget (half
  // of L2 by default), so the labels being relaxed stay in L2.
  long long small_budget = 0;
  long long small_labels = 0;
  int small_active = 0;
  // A large request runs alone through the single-query kernel on its
  // graph's handle: the resident kernel is stopped between batches (its
  // queued work stays queued), the query runs, the resident kernel resumes.
  int solo_state = 0;                    // 0 none, 1 stopping the resident kernel, 2 running
  ServeRequest solo_rq{};
  bool stop_requested = false;
  cudaStream_t side = nullptr;           // writes the stop flag while the kernel runs
  cudaEvent_t solo_done = nullptr;
  int32_t* solo_status = nullptr;        // pinned: the solo query's status code
  int32_t* solo_status_dev = nullptr;
  int* one_host = nullptr;               // pinned 1, for the stop flag
  int32_t* solo_scratch = nullptr;       // dist for a request that asked for none
  long long solo_scratch_n = 0;
  std::vector<int> free_slots;
  std::map<long long, long long> free_pages;        // start page -> page count
  int64_t next_id = 1;
  unsigned cmd_tail = 0, done_head = 0;
  bool stopping = false;
  int fatal = 0;
  long long relaunches = 0, completed = 0, peak_active = 0;
  long long completed_at_launch = 0;
  int stalled_launches = 0;
  int cuda_error = 0;
  int bad_where = 0;
  unsigned bad_value = 0;
  std::thread th;

  ~bfq_server() {
    if (th.joinable()) {
      {
        std::lock_guard<std::mutex> lk(mu);
        stopping = true;
      }
      cv.notify_all();
      th.join();
    }
    if (stream) cudaStreamSynchronize(stream);
    if (side) cudaStreamSynchronize(side);
    if (solo_done) cudaEventDestroy(solo_done);
    if (side) cudaStreamDestroy(side);
    if (solo_status) cudaFreeHost(solo_status);
    if (one_host) cudaFreeHost(one_host);
    if (solo_scratch) cudaFree(solo_scratch);
    if (kernel_done) cudaEventDestroy(kernel_done);
    if (stream) cudaStreamDestroy(stream);
    for (void* p : dev_allocs) cudaFree(p);
    if (cmd_host) cudaFreeHost(cmd_host);
    if (done_host) cudaFreeHost(done_host);
    if (shutdown_host) cudaFreeHost(shutdown_host);
  }

  int dalloc(void** p, size_t n) {
    cudaError_t e = cudaMalloc(p, n ? n : 16);
    if (e != cudaSuccess) return cuda_fail(e, "cudaMalloc", __FILE__, __LINE__);
    dev_allocs.push_back(*p);
    return BFQ_OK;
  }

  static int64_t now_ns() {
    return std::chrono::duration_cast<std::chrono::nanoseconds>(
               std::chrono::steady_clock::now().time_since_epoch())
        .count();
  }

  // Every admitted and waiting request ends with `code`.
  void fail_all(int code) {
    for (auto& kv : admitted) {
      auto rec = records.find(kv.first);
      if (rec != records.end()) {
        rec->second.status = code;
        rec->second.t_done = now_ns();
      }
    }
    admitted.clear();
    large_active = 0;
    small_labels = 0;
    small_active = 0;
    if (solo_state == 1) {
      auto rec = records.find(solo_rq.id);
      if (rec != records.end()) {
        rec->second.status = code;
        rec->second.t_done = now_ns();
      }
      solo_state = 0;
    }
    for (auto& rq : pending) {
      auto rec = records.find(rq.id);
      if (rec != records.end()) {
        rec->second.status = code;
        rec->second.t_done = now_ns();
      }
    }
    pending.clear();
  }

  bool alloc_pages(long long need, long long* start) {
    for (auto it = free_pages.begin(); it != free_pages.end(); ++it) {
      if (it->second >= need) {
        *start = it->first;
        const long long rest = it->second - need, rs = it->first + need;
        free_pages.erase(it);
        if (rest > 0) free_pages[rs] = rest;
        return true;
      }
    }
    return false;
  }

  void free_run(long long start, long long n) {
    auto it = free_pages.emplace(start, n).first;
    auto nx = std::next(it);
    if (nx != free_pages.end() && it->first + it->second == nx->first) {
      it->second += nx->second;
      free_pages.erase(nx);
    }
    if (it != free_pages.begin()) {
      auto pv = std::prev(it);
      if (pv->first + pv->second == it->first) {
        pv->second += it->second;
        free_pages.erase(it);
      }
    }
  }

  // Consume completion records; admit pending requests; keep the kernel up.
  void loop() {
    cudaSetDevice(device);
    std::unique_lock<std::mutex> lk(mu);
    while (true) {
      bool progressed = false;
      // completions
      for (;;) {
        volatile ServeDone* r = done_host + (done_head % (unsigned)ring);
        if (__atomic_load_n(&r->seq, __ATOMIC_ACQUIRE) != done_head + 1) break;
        const long long id = r->req_id;
        const int st = r->status;
        ++done_head;
        progressed = true;
        auto ad = admitted.find(id);
        if (ad != admitted.end()) {
          free_slots.push_back(ad->second.slot);
          free_run(ad->second.start, ad->second.pages);
          if (ad->second.large) {
            --large_active;
          } else {
            --small_active;
            small_labels -= ad->second.pages << kPageLog2;
          }
          admitted.erase(ad);
        }
        auto rec = records.find(id);
        if (rec != records.end()) {
          rec->second.status = st;
          rec->second.t_done = now_ns();
        }
        ++completed;
      }
      // admissions in FIFO order: a request waits until it fits, and those
      // behind it wait too, except behind a large request that waits for the
      // large one running now
      for (size_t i = 0; i < pending.size() && i < 1024 && !free_slots.empty() && !fatal;) {
        ServeRequest& rq = pending[i];
        const GraphView& gv = views[rq.graph];
        const bool large = gv.V >= large_vertices;
        const long long need = ((long long)gv.V + (1 << kPageLog2) - 1) >> kPageLog2;
        if (large && large_active > 0) {
          ++i;
          continue;
        }
        if (large) {
          // run it alone through the single-query kernel (see solo_state)
          solo_rq = rq;
          solo_state = 1;
          ++large_active;
          pending.erase(pending.begin() + (long)i);
          if (launched && !stop_requested) {
            cudaMemcpyAsync(&args.ctl->stop, one_host, sizeof(int), cudaMemcpyHostToDevice, side);
            stop_requested = true;
          }
          progressed = true;
          continue;
        }
        if (!large && small_active > 0 && small_labels + (need << kPageLog2) > small_budget)
          break;
        long long start = 0;
        if (!alloc_pages(need, &start)) break;
        const int slot = free_slots.back();
        free_slots.pop_back();
        ServeCmd* c = cmd_host + (cmd_tail % (unsigned)ring);
        SlotDesc d{};
        d.row_ptr = gv.row_ptr;
        d.adj = gv.adj;
        d.hub_chunk0 = gv.hub_chunk0;
        d.chunk_tab = gv.chunk_tab;
        d.dist = rq.dist;
        d.hops = rq.hops;
        d.V = gv.V;
        d.src = rq.src;
        d.hub_degree = gv.hub_degree;
        d.chunk_edges = gv.chunk_edges;
        d.label_off = (int)(start << kPageLog2);
        d.n_chunks = gv.n_chunks;
        d.req_id = rq.id;
        c->d = d;
        c->slot = slot;
        __atomic_store_n(&c->seq, cmd_tail + 1, __ATOMIC_RELEASE);
        ++cmd_tail;
        admitted[rq.id] = Admitted{slot, start, need, large};
        if (large) {
          ++large_active;
        } else {
          ++small_active;
          small_labels += need << kPageLog2;
        }
        pending.erase(pending.begin() + (long)i);
        progressed = true;
        peak_active = std::max<long long>(peak_active, (long long)admitted.size());
      }
      // the kernel runs while anything is admitted
      cudaError_t qe = launched ? cudaEventQuery(kernel_done) : cudaSuccess;
      if (launched && qe != cudaSuccess && qe != cudaErrorNotReady) {
        // the launch failed outright: nothing more can run on this context
        cuda_error = (int)qe;
        fail_all(BFQ_ERR_CUDA);
        launched = false;
        stopping = true;
      }
      if (launched && qe == cudaSuccess) {
        launched = false;
        ServeCtl c;
        cudaMemcpy(&c, args.ctl, sizeof(c), cudaMemcpyDeviceToHost);
        // a launch that ran to its time limit without completing anything
        // while requests were admitted counts as stuck (not one stopped for
        // a large request)
        stalled_launches = (completed == completed_at_launch && !admitted.empty() &&
                            !stop_requested)
                               ? stalled_launches + 1 : 0;
        stop_requested = false;
        if (c.bad_where) {
          bad_where = c.bad_where;
          bad_value = c.bad_value;
        }
        if ((c.status & (kStTimeout | kStQueue)) || stalled_launches >= 3) {
          stalled_launches = 0;
          // a bounded wait ran out, or the kernel made no progress: fail what
          // was admitted and reset the queues
          for (auto& kv : admitted) {
            auto rec = records.find(kv.first);
            if (rec != records.end()) {
              rec->second.status = BFQ_ERR_TIMEOUT;
              rec->second.t_done = now_ns();
            }
            free_slots.push_back(kv.second.slot);
            free_run(kv.second.start, kv.second.pages);
          }
          admitted.clear();
          large_active = 0;
          small_labels = 0;
          small_active = 0;
          serve_reset_kernel<<<1024, 256, 0, stream>>>(args);
          cudaMemcpyAsync(&args.ctl->cmd_head, &cmd_tail, sizeof(unsigned), cudaMemcpyHostToDevice,
                          stream);
          cudaStreamSynchronize(stream);
        }
      }
      // the solo query: start it once the resident kernel is down, finish it
      if (solo_state == 1 && !launched) {
        const GraphView& gv = views[solo_rq.graph];
        int32_t* dist = solo_rq.dist;
        int rc = BFQ_OK;
        if (!dist) {
          if (solo_scratch_n < gv.V) {
            if (solo_scratch) cudaFree(solo_scratch);
            solo_scratch = nullptr;
            solo_scratch_n = 0;
            if (cudaMalloc((void**)&solo_scratch, sizeof(int32_t) * (size_t)gv.V) == cudaSuccess)
              solo_scratch_n = gv.V;
            else
              rc = BFQ_ERR_OOM;
          }
          dist = solo_scratch;
        }
        if (rc == BFQ_OK)
          rc = bfq_sssp_async(graphs[solo_rq.graph], solo_rq.src, dist, solo_rq.hops, nullptr,
                              solo_status_dev, stream);
        if (rc == BFQ_OK) {
          cudaMemcpyAsync(solo_status, solo_status_dev, sizeof(int32_t), cudaMemcpyDeviceToHost,
                          stream);
          cudaEventRecord(solo_done, stream);
          solo_state = 2;
        } else {
          auto rec = records.find(solo_rq.id);
          if (rec != records.end()) {
            rec->second.status = rc;
            rec->second.t_done = now_ns();
          }
          ++completed;
          --large_active;
          solo_state = 0;
        }
        progressed = true;
      }
      if (solo_state == 2) {
        const cudaError_t se = cudaEventQuery(solo_done);
        if (se != cudaErrorNotReady) {
          // nothing else runs now: persisting lines the large query's L2
          // window left behind become normal lines again before the
          // resident kernel resumes
          int lpct = 0;
          bfq_tune lt{};
          if (bfq_graph_get_tune(graphs[solo_rq.graph], &lt) == BFQ_OK) lpct = lt.l2_persist_pct;
          if (lpct > 0) cudaCtxResetPersistingL2Cache();
          auto rec = records.find(solo_rq.id);
          if (rec != records.end()) {
            rec->second.status = se == cudaSuccess ? *solo_status : BFQ_ERR_CUDA;
            rec->second.t_done = now_ns();
          }
          if (se != cudaSuccess) cuda_error = (int)se;
          ++completed;
          --large_active;
          solo_state = 0;
          progressed = true;
        }
      }
      if (!launched && !admitted.empty() && !stopping && solo_state == 0) {
        completed_at_launch = completed;
        // a stop written from the side stream must land before it is cleared
        cudaStreamSynchronize(side);
        cudaMemsetAsync(&args.ctl->stop, 0, sizeof(int), stream);
        serve_kernel<<<grid, kBlock, 0, stream>>>(args);
        cudaEventRecord(kernel_done, stream);
        launched = true;
        ++relaunches;
      }
      if (stopping && admitted.empty() && pending.empty() && solo_state == 0) break;
      if (stopping && !launched && solo_state == 0) break;
      if (!progressed) {
        cv.wait_for(lk, std::chrono::microseconds(20));
      }
    }
    __atomic_store_n(shutdown_host, 1, __ATOMIC_RELEASE);
    lk.unlock();
    cudaStreamSynchronize(stream);
  }
};

static int s_invalid(const char* m) {
  set_error(m);
  return BFQ_ERR_INVALID;
}

extern "C" {

int bfq_server_create(bfq_server_t* out, const bfq_graph_t* graphs, int32_t ngraphs,
                      int64_t hbm_budget_bytes, int32_t max_slots, const bfq_tune* tune) {
  if (!out) return s_invalid("bfq_server_create: out is null");
  *out = nullptr;
  if (!graphs || ngraphs < 1) return s_invalid("bfq_server_create: no graphs");
  if (max_slots < 1 || max_slots > kMaxSlots)
    return s_invalid("bfq_server_create: max_slots must be in [1, 2048]");
  bfq_server* sv = new (std::nothrow) bfq_server();
  if (!sv) return s_invalid("bfq_server_create: host allocation failed");
  bfq_tune_default(&sv->tune);
  if (tune) {
    if (tune->share_div) sv->tune.share_div = tune->share_div;
    if (tune->chunk_batch) sv->tune.chunk_batch = tune->chunk_batch;
    if (tune->batch_items) sv->tune.batch_items = tune->batch_items;
    if (tune->spin_limit) sv->tune.spin_limit = tune->spin_limit;
    if (tune->time_limit_ms) sv->tune.time_limit_ms = tune->time_limit_ms;
    if (tune->cycle_walk_hops >= 2 && tune->cycle_walk_hops <= (1 << 30))
      sv->tune.cycle_walk_hops = tune->cycle_walk_hops;
  }
  long long maxC = 0;
  for (int i = 0; i < ngraphs; ++i) {
    GraphView gv;
    if (graph_view(graphs[i], &gv) != BFQ_OK) { delete sv; return s_invalid("bfq_server_create: bad graph handle"); }
    if (gv.n_chunks >= (1 << kChunkIdBits)) { delete sv; return s_invalid("bfq_server_create: a graph has too many hub chunks (>= 2^20)"); }
    sv->graphs.push_back(graphs[i]);
    sv->views.push_back(gv);
    maxC = std::max<long long>(maxC, gv.n_chunks);
  }
  // budget: 8 B of label + 8 B of recorded edge + 16 B of sub-queue slots
  // per pooled label
  long long entries = hbm_budget_bytes / 32;
  entries = (entries >> kPageLog2) << kPageLog2;
  if (entries < (1 << kPageLog2) || entries >= (1LL << 31))
    { delete sv; return s_invalid("bfq_server_create: budget must cover 4096..2^31 labels"); }
  sv->pool_entries = entries;
  sv->S = max_slots;
  sv->ring = 2 * max_slots;
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  sv->device = dev;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  int per_sm = 1;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, serve_kernel, kBlock, 0) != cudaSuccess ||
      per_sm < 1)
    per_sm = 1;
  sv->grid = sms * per_sm;
  int l2 = 0;
  cudaDeviceGetAttribute(&l2, cudaDevAttrL2CacheSize, dev);
  {
    const int k = tune ? tune->batch_budget_klabels : 0;
    sv->small_budget = k < 0 ? (1LL << 62) : k > 0 ? (long long)k << 10
                                                   : (long long)l2 / 2 / (long long)sizeof(long long);
    // large: labels over a quarter of L2, or over half of the budget
    sv->large_vertices = std::min<long long>((long long)l2 / 4 / (long long)sizeof(long long),
                                             std::max<long long>(1, sv->small_budget / 2));
  }
  ServeArgs& a = sv->args;
  a.queues_per_cta = 1;
  a.qs.Q = sv->grid;
  // total vertex-queue capacity in [E, 2E): at least every pooled label
  // (at most that many items are queued at once), at most 16 B per label
  int ql = 10;
  while ((1LL << (ql + 1)) <= (2 * entries) / a.qs.Q) ++ql;
  a.qs.cap_log2 = ql;
  a.cq.Q = sv->grid;
  a.cq.cap_log2 = std::min(14, std::max(8, ceil_log2_s((maxC * max_slots + a.cq.Q - 1) / a.cq.Q)));
  a.tq.Q = 1;
  long long max_tasks = 1;
  for (const GraphView& gv : sv->views)
    max_tasks = std::max<long long>(max_tasks, (gv.V + (1LL << kTaskLog2) - 1) >> kTaskLog2);
  a.tq.cap_log2 = std::max(10, ceil_log2_s((long long)max_slots *
                                           std::min<long long>(max_tasks, kMaxHelpers)));
  a.ring = sv->ring;
  a.max_slots = max_slots;
  a.pool_pages = (int)(entries >> kPageLog2);
  a.share_div = sv->tune.share_div;
  a.chunk_batch = sv->tune.chunk_batch;
  a.batch_items = sv->tune.batch_items;
  a.cyc_walk0 = (unsigned)sv->tune.cycle_walk_hops;
  a.spin_limit = sv->tune.spin_limit;
  a.time_limit_ns = sv->tune.time_limit_ms * 1000000LL;
  a.idle_exit_ns = 5LL * 1000000LL;
  const long long pages = entries >> kPageLog2;
  int rc = BFQ_OK;
#define S_TRY(x) do { rc = (x); if (rc != BFQ_OK) { delete sv; return rc; } } while (0)
  S_TRY(sv->dalloc((void**)&a.slots, sizeof(SlotDesc) * max_slots));
  S_TRY(sv->dalloc((void**)&a.inflight, sizeof(int) * kCounterStride * max_slots));
  S_TRY(sv->dalloc((void**)&a.qstatus, sizeof(int) * max_slots));
  S_TRY(sv->dalloc((void**)&a.pending, sizeof(int) * kCounterStride * max_slots));
  S_TRY(sv->dalloc((void**)&a.page_owner, sizeof(int) * pages));
  S_TRY(sv->dalloc((void**)&a.label, sizeof(long long) * entries));
  S_TRY(sv->dalloc((void**)&a.cyc, sizeof(long long) * entries));
  S_TRY(sv->dalloc((void**)&a.qs.meta, sizeof(QueueMeta) * a.qs.Q));
  S_TRY(sv->dalloc((void**)&a.qs.slots, sizeof(unsigned long long) * ((size_t)a.qs.Q << a.qs.cap_log2)));
  S_TRY(sv->dalloc((void**)&a.cq.meta, sizeof(QueueMeta) * a.cq.Q));
  S_TRY(sv->dalloc((void**)&a.cq.slots, sizeof(unsigned long long) * ((size_t)a.cq.Q << a.cq.cap_log2)));
  S_TRY(sv->dalloc((void**)&a.tq.meta, sizeof(QueueMeta)));
  S_TRY(sv->dalloc((void**)&a.tq.slots, sizeof(unsigned long long) * ((size_t)1 << a.tq.cap_log2)));
  S_TRY(sv->dalloc((void**)&a.ctl, sizeof(ServeCtl)));
  S_TRY(sv->dalloc((void**)&sv->solo_status_dev, sizeof(int32_t)));
#undef S_TRY
#define S_CUDA(x) do { cudaError_t e__ = (x); if (e__ != cudaSuccess) { int r__ = cuda_fail(e__, #x, __FILE__, __LINE__); delete sv; return r__; } } while (0)
  S_CUDA(cudaHostAlloc((void**)&sv->cmd_host, sizeof(ServeCmd) * sv->ring, cudaHostAllocMapped));
  S_CUDA(cudaHostAlloc((void**)&sv->done_host, sizeof(ServeDone) * sv->ring, cudaHostAllocMapped));
  S_CUDA(cudaHostAlloc((void**)&sv->shutdown_host, sizeof(int), cudaHostAllocMapped));
  std::memset(sv->cmd_host, 0, sizeof(ServeCmd) * sv->ring);
  std::memset(sv->done_host, 0, sizeof(ServeDone) * sv->ring);
  *sv->shutdown_host = 0;
  S_CUDA(cudaHostGetDevicePointer((void**)&a.cmd, sv->cmd_host, 0));
  S_CUDA(cudaHostGetDevicePointer((void**)&a.done, sv->done_host, 0));
  S_CUDA(cudaHostGetDevicePointer((void**)&a.shutdown, sv->shutdown_host, 0));
  S_CUDA(cudaMemset(a.ctl, 0, sizeof(ServeCtl)));
  S_CUDA(cudaMemset(a.cyc, 0xff, sizeof(long long) * entries));
  S_CUDA(cudaMemset(a.inflight, 0, sizeof(int) * kCounterStride * max_slots));
  S_CUDA(cudaStreamCreateWithFlags(&sv->stream, cudaStreamNonBlocking));
  S_CUDA(cudaEventCreateWithFlags(&sv->kernel_done, cudaEventDisableTiming));
  S_CUDA(cudaStreamCreateWithFlags(&sv->side, cudaStreamNonBlocking));
  S_CUDA(cudaEventCreateWithFlags(&sv->solo_done, cudaEventDisableTiming));
  S_CUDA(cudaMallocHost((void**)&sv->solo_status, sizeof(int32_t)));
  S_CUDA(cudaMallocHost((void**)&sv->one_host, sizeof(int)));
  *sv->one_host = 1;
  serve_reset_kernel<<<1024, 256, 0, sv->stream>>>(a);
  S_CUDA(cudaGetLastError());
  S_CUDA(cudaStreamSynchronize(sv->stream));
#undef S_CUDA
  for (int s = max_slots - 1; s >= 0; --s) sv->free_slots.push_back(s);
  sv->free_pages[0] = pages;
  sv->th = std::thread([sv] { sv->loop(); });
  *out = sv;
  return BFQ_OK;
}

int bfq_server_submit(bfq_server_t sv, int32_t graph_id, int32_t src, int32_t* dist,
                      int32_t* hops, int64_t* req_id) {
  if (!sv || !req_id) return s_invalid("bfq_server_submit: null argument");
  if (graph_id < 0 || graph_id >= (int)sv->graphs.size())
    return s_invalid("bfq_server_submit: graph id out of range");
  const GraphView& gv = sv->views[graph_id];
  if (src < 0 || src >= gv.V) return s_invalid("bfq_server_submit: source out of range");
  const long long need = ((long long)gv.V + (1 << kPageLog2) - 1) >> kPageLog2;
  if ((need << kPageLog2) > sv->pool_entries) {
    set_error("bfq_server_submit: the graph's labels can never fit the memory budget");
    return BFQ_ERR_BUDGET;
  }
  {
    std::lock_guard<std::mutex> lk(sv->mu);
    if (sv->stopping) return s_invalid("bfq_server_submit: server is shutting down");
    if (sv->cuda_error) {
      set_error("bfq_server_submit: the server stopped after a CUDA error");
      return BFQ_ERR_CUDA;
    }
    const int64_t id = sv->next_id++;
    const int64_t t = bfq_server::now_ns();
    sv->pending.push_back({id, graph_id, src, dist, hops, t});
    ServeRecord r;
    r.t_submit = t;
    sv->records[id] = r;
    *req_id = id;
  }
  sv->cv.notify_all();
  return BFQ_OK;
}

int bfq_server_poll(bfq_server_t sv, int64_t req_id, int32_t* status, int64_t* t_submit_ns,
                    int64_t* t_done_ns) {
  if (!sv) return s_invalid("bfq_server_poll: null handle");
  std::lock_guard<std::mutex> lk(sv->mu);
  auto it = sv->records.find(req_id);
  if (it == sv->records.end()) return s_invalid("bfq_server_poll: unknown request id");
  if (status) *status = it->second.status;
  if (t_submit_ns) *t_submit_ns = it->second.t_submit;
  if (t_done_ns) *t_done_ns = it->second.t_done;
  return it->second.status == BFQ_PENDING ? BFQ_PENDING : BFQ_OK;
}

int bfq_server_wait(bfq_server_t sv, int64_t req_id, int64_t timeout_ms, int32_t* status) {
  if (!sv) return s_invalid("bfq_server_wait: null handle");
  const auto limit = std::chrono::steady_clock::now() + std::chrono::milliseconds(timeout_ms);
  for (;;) {
    int32_t st = BFQ_PENDING;
    int rc = bfq_server_poll(sv, req_id, &st, nullptr, nullptr);
    if (rc < 0) return rc;
    if (st != BFQ_PENDING) {
      if (status) *status = st;
      return BFQ_OK;
    }
    if (std::chrono::steady_clock::now() > limit) return BFQ_PENDING;
    std::this_thread::sleep_for(std::chrono::microseconds(20));
  }
}

int bfq_server_stats(bfq_server_t sv, int64_t* completed, int64_t* relaunches,
                     int64_t* peak_active) {
  if (!sv) return s_invalid("bfq_server_stats: null handle");
  std::lock_guard<std::mutex> lk(sv->mu);
  if (completed) *completed = sv->completed;
  if (relaunches) *relaunches = sv->relaunches;
  if (peak_active) *peak_active = sv->peak_active;
  return BFQ_OK;
}

int bfq_server_state(bfq_server_t sv, int64_t* out, int32_t n) {
  if (!sv || !out || n < 1) return s_invalid("bfq_server_state: null argument");
  std::lock_guard<std::mutex> lk(sv->mu);
  long long largest = 0;
  for (auto& kv : sv->free_pages) largest = std::max(largest, kv.second);
  const int64_t v[10] = {(int64_t)sv->pending.size(), (int64_t)sv->admitted.size(),
                         (int64_t)sv->free_slots.size(), largest << kPageLog2,
                         sv->relaunches, sv->completed, sv->launched ? 1 : 0,
                         sv->cuda_error, sv->bad_where, (int64_t)sv->bad_value};
  for (int i = 0; i < n && i < 10; ++i) out[i] = v[i];
  return BFQ_OK;
}

int bfq_server_destroy(bfq_server_t sv) {
  if (!sv) return s_invalid("bfq_server_destroy: null handle");
  delete sv;
  return BFQ_OK;
}

}  // extern "C"
