// Batched queue-driven Bellman-Ford: many single-source queries, over many
// resident graphs, in one persistent launch (Sec. III-C's algorithm, run for
// a query table instead of one source).
//
// Every query q owns a slice [label_off[q], label_off[q] + V_q) of one label
// pool; a queue item is a global label index, so one set of sub-queues carries
// the work of all queries and a warp's batch may mix queries.  The query of
// an item is found by binary search over the offsets (kept in shared memory).
// Each query has its own in-flight counter and status bits: a query whose
// label reaches hops >= V_q (negative cycle) or leaves the int32 range is
// drained -- its remaining items are taken and dropped -- while the others go
// on.  The launch ends when every query's in-flight count is zero.
//
// The whole run (staging copy of the query table, reset, init, persistent
// kernel, epilogue, status copy-back) is captured once into a CUDA graph and
// replayed per call; per-call parameters travel in the staging block.
#include <algorithm>
#include <cstring>
#include <new>
#include <vector>

#include "sssp_multi.cuh"

namespace bfq {

struct alignas(16) QueryDesc {
  const int* row_ptr;
  const int2* adj;
  const int* hub_chunk0;
  const int4* chunk_tab;
  int* dist;
  int* hops;
  int V, src, hub_degree, chunk_edges;
  int label_off, chunk_off, pad0, pad1;
};

// Host-written block copied to the device before every run.
struct alignas(16) StageHeader {
  int nq;
  int share_div, chunk_batch, batch_items, phantom;
  int cyc_walk0;                // first cycle-walk threshold (hops)
  int window;                   // queries started by the init kernel
  int pad;
  long long time_limit_ns, spin_limit;
  long long budget;             // labels of the queries running at once (soft)
  long long pad1;
};

struct alignas(128) BatchCtl {
  int remaining;                // queries with work left
  int pad0[31];
  int stop;                     // whole-launch stop (timeout)
  int pad1[31];
  int status;                   // whole-launch kSt* bits
  int pad2[31];
  unsigned long long ctr[8];
  unsigned long long pad3[8];
  int last_status;              // 0, or an error code that needs a queue reset
  int pad4[31];
  int next_q;                   // next query to start
  int pad5[31];
  int active;                   // queries started and not finished
  int pad6[31];
  long long active_labels;      // their labels
  long long pad7[15];
};

struct BatchArgs {
  const StageHeader* hdr;       // device copy of the staging block
  const int* loff;              // [nq + 1] label offsets
  const int* coff;              // [nq + 1] chunk-item offsets
  const QueryDesc* desc;        // [nq]
  long long* label;             // pool
  long long* cyc;               // recorded relaxation edges, like the pool
  QueueSet qs, cq;
  int* inflight;                // [maxq * kCounterStride]
  int* qstatus;                 // [maxq]
  int* qcode;                   // [maxq] status codes out
  BatchCtl* ctl;
  int maxq;
  int queues_per_cta;
};

namespace {

__device__ __forceinline__ int find_query(const int* off, int nq, int x) {
  int lo = 0, hi = nq - 1;                  // largest q with off[q] <= x
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (off[mid] <= x) lo = mid; else hi = mid - 1;
  }
  return lo;
}

__device__ __forceinline__ void batch_timeout(const BatchArgs& a) {
  atomicOr(&a.ctl->status, kStTimeout);
  st_relaxed_s32(&a.ctl->stop, 1);
}

// Queries start in order while the labels of the running ones stay within
// the budget (half of L2 by default): the labels of a few dozen running
// queries then stay in L2 instead of all of them being touched at random
// in HBM.  A query that finishes frees its share and starts the next ones;
// one always runs.  Returns false if a source could not be queued.
__device__ __forceinline__ bool start_queries(const BatchArgs& a, const StageHeader& hdr,
                                              const int* s_loff, int lane, int home) {
  for (;;) {
    int q = -1;
    if (lane == 0) {
      const int n = ld_relaxed_s32(&a.ctl->next_q);
      if (n < hdr.nq) {
        const long long v = (long long)s_loff[n + 1] - s_loff[n];
        if (ld_relaxed_s32(&a.ctl->active) == 0 ||
            (long long)ld_relaxed_u64((unsigned long long*)&a.ctl->active_labels) + v <= hdr.budget) {
          if (atomicCAS(&a.ctl->next_q, n, n + 1) == n) {
            atomicAdd((unsigned long long*)&a.ctl->active_labels, (unsigned long long)v);
            atomicAdd(&a.ctl->active, 1);
            a.inflight[n * kCounterStride] = 1 + hdr.phantom;
            q = n;
          } else {
            q = -2;                                // lost the race: look again
          }
        }
      }
    }
    q = __shfl_sync(kFullMask, q, 0);
    if (q == -2) continue;
    if (q < 0) return true;
    __syncwarp();                                  // in-flight count before the source
    const unsigned item = (unsigned)(s_loff[q] + a.desc[q].src);
    if (enqueue_warp(a.qs, home, lane == 0, item, lane, hdr.spin_limit, 4LL * a.qs.Q + 64) != 1)
      return false;
  }
}

// MIN: relax with atomicMin (the running queries' labels fit in L2 under
// the label budget); both forms are compiled, capture() picks one.
template <bool MIN>
__global__ void __launch_bounds__(kBlock, BFQ_MULTI_CTAS_PER_SM) batch_persistent_kernel(BatchArgs a) {
  extern __shared__ int s_off[];                // loff[nq+1], coff[nq+1]
  __shared__ unsigned s_children[kBlock / 32][kChildBuf];
  __shared__ unsigned short s_childq[kBlock / 32][kChildBuf];
  __shared__ MultiStage s_mstage[kBlock / 32];
  const StageHeader hdr = *a.hdr;
  const int nq = hdr.nq;
  int* s_loff = s_off;
  int* s_coff = s_off + nq + 1;
  for (int i = threadIdx.x; i <= nq; i += blockDim.x) {
    s_loff[i] = a.loff[i];
    s_coff[i] = a.coff[i];
  }
  __syncthreads();
  if (nq == 0) return;

  const int lane = threadIdx.x & 31;
  const int wid = threadIdx.x >> 5;
  const int nwarps = blockDim.x >> 5;
  const int home = (blockIdx.x * a.queues_per_cta + wid % a.queues_per_cta) % a.qs.Q;
  const int chome = blockIdx.x % a.cq.Q;
  const int share = hdr.share_div > 0 ? hdr.share_div : max(1, nwarps / a.queues_per_cta);
  unsigned* buf = s_children[wid];
  unsigned short* bufq = s_childq[wid];
  int nbuf = 0;
  WarpCounters wc;
  const MultiEnv env{a.label, a.cyc, a.inflight, a.qstatus, &a.ctl->status, &a.ctl->stop,
                     a.qs, hdr.spin_limit, (unsigned)hdr.cyc_walk0};
  unsigned walk_at = env.cyc_walk0;     // per lane: hops that trigger a cycle walk
  const unsigned long long t_start = globaltimer_ns();
  unsigned rng = 0x9e3779b9u * (blockIdx.x * 64u + wid + 1u);
  int idle = 0;
  bool timed_out = false;

  for (;;) {
    unsigned item = 0;
    int got = 0;
    bool is_chunk = false;
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
      got = wq_dequeue_warp(a.cq, chome, hdr.chunk_batch, lane, &item, hdr.spin_limit, c_chunk);
    }
    if (got == 0 && c_vert > 0) {
      is_chunk = false;
      got = wq_dequeue_warp(a.qs, home, share_of(c_vert, hdr.batch_items, share), lane, &item,
                            hdr.spin_limit, c_vert);
    }
    if (got == 0) {
      rng = rng * 1664525u + 1013904223u;
      int q = probe_queues(a.cq, (int)(rng % (unsigned)a.cq.Q), chome, lane);
      if (q >= 0) {
        is_chunk = true;
        got = wq_dequeue_warp(a.cq, q, hdr.chunk_batch, lane, &item, hdr.spin_limit);
      } else {
        q = probe_queues(a.qs, (int)((rng >> 7) % (unsigned)a.qs.Q), home, lane);
        if (q >= 0) {
          is_chunk = false;                 // whatever the home probes set
          int cnt = 0;
          if (lane == 0) cnt = ld_relaxed_s32(&a.qs.meta[q].count);
          cnt = __shfl_sync(kFullMask, cnt, 0);
          if (cnt > 0)
            got = wq_dequeue_warp(a.qs, q, share_of(cnt, hdr.batch_items, share), lane, &item,
                                  hdr.spin_limit, cnt);
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
        done = (ld_relaxed_s32(&a.ctl->remaining) <= 0) || ld_relaxed_s32(&a.ctl->stop);
        if (!done && ((idle + 1) & 31) == 0 &&
            (long long)(globaltimer_ns() - t_start) > hdr.time_limit_ns)
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

    // decode the lanes' items
    int q = -1, deg = 0, nch = 0, c0 = 0, Vq = 0, tail = 0;
    long long lab = 0;
    long long* lbase = nullptr;
    const int2* eptr = nullptr;
    if (lane < got) {
      if (is_chunk) {
        q = find_query(s_coff, nq, (int)item);
        const QueryDesc& d = a.desc[q];
        const int4 ct = d.chunk_tab[(int)item - s_coff[q]];
        tail = ct.x;
        lbase = a.label + s_loff[q];
        lab = label_key(ld_relaxed_s64(lbase + ct.x));
        eptr = d.adj + ct.y;
        deg = ct.z - ct.y;
        Vq = d.V;
      } else {
        q = find_query(s_loff, nq, (int)item);
        const int u = (int)item - s_loff[q];
        tail = u;
        const QueryDesc& d = a.desc[q];
        lbase = a.label + s_loff[q];
        lab = label_key((long long)atomicAnd((unsigned long long*)(lbase + u),
                                             ~(unsigned long long)kQueuedBit));
        const int beg = __ldg(d.row_ptr + u);
        deg = __ldg(d.row_ptr + u + 1) - beg;
        eptr = d.adj + beg;
        Vq = d.V;
        if (deg > d.hub_degree) {
          nch = (deg + d.chunk_edges - 1) / d.chunk_edges;
          c0 = s_coff[q] + __ldg(d.hub_chunk0 + u);
          deg = 0;
        }
      }
      if (ld_relaxed_s32(&a.qstatus[q]) & (kStNegCycle | kStRange)) {   // drained query
        deg = 0;
        nch = 0;
      }
    }
    // hub chunks of this batch, counted per query before they are published;
    // chunks that find no room are relaxed right here
    if (__any_sync(kFullMask, nch > 0)) {
      const int qn = nch > 0 ? q : -1;
      const unsigned m = __match_any_sync(kFullMask, qn);
      const int sum_q = (int)__reduce_add_sync(m, (unsigned)nch);
      if (qn >= 0 && lane == __ffs(m) - 1) red_add_relaxed_s32(&a.inflight[qn * kCounterStride], sum_q);
      __syncwarp();
      int K = 0;
      const int excl = warp_excl_scan(nch, lane, &K);
      for (int base = 0; base < K && !timed_out; base += 32) {
        const int t = base + lane;
        const int j = owner_lane(excl, t, 32);
        const int ex_j = __shfl_sync(kFullMask, excl, j);
        const int c0_j = __shfl_sync(kFullMask, c0, j);
        const bool act = t < K;
        const unsigned id = (unsigned)(c0_j + (t - ex_j));
        const int placed = enqueue_warp(a.cq, chome, act, id, lane, hdr.spin_limit, 2LL * a.cq.Q);
        if (placed < 0) { timed_out = true; break; }
        const unsigned act_mask = __ballot_sync(kFullMask, act);
        const int rank = __popc(act_mask & ((1u << lane) - 1u));
        unsigned left = __ballot_sync(kFullMask, act && rank >= placed);
        while (left) {
          const unsigned cid = __shfl_sync(kFullMask, id, __ffs(left) - 1);
          left &= left - 1;
          int cq_q = -1, cdeg = 0, cV = 0, ctail = 0;
          long long clab = 0;
          long long* clb = nullptr;
          const int2* cep = nullptr;
          if (lane == 0) {
            cq_q = find_query(s_coff, nq, (int)cid);
            const QueryDesc& d = a.desc[cq_q];
            const int4 ct = d.chunk_tab[(int)cid - s_coff[cq_q]];
            clb = a.label + s_loff[cq_q];
            clab = label_key(ld_relaxed_s64(clb + ct.x));
            cep = d.adj + ct.y;
            cdeg = ct.z - ct.y;
            cV = d.V;
            ctail = ct.x;
          }
          if (!relax_multi<kMultiGroups, MIN>(env, 1, cep, cdeg, clab, clb, cV, cq_q, ctail, lane, home,
                                    wc, buf, bufq, nbuf, walk_at, &s_mstage[wid]) ||
              !flush_multi(env, home, buf, bufq, nbuf, lane, wc)) {
            timed_out = true;
            break;
          }
          __syncwarp();
          if (lane == 0) red_add_relaxed_s32(&a.inflight[cq_q * kCounterStride], -1);
        }
      }
      if (timed_out) break;
    }
    if (!relax_multi<kMultiGroups, MIN>(env, got, eptr, deg, lab, lbase, Vq, q, tail, lane, home, wc,
                              buf, bufq, nbuf, walk_at, &s_mstage[wid]) ||
        !flush_multi(env, home, buf, bufq, nbuf, lane, wc)) {
      timed_out = true;
      break;
    }
    __syncwarp();
    const int emptied = retire_multi(env, lane < got ? q : -1, lane);
    if (emptied >= 0) {
      atomicAdd(&a.ctl->remaining, -1);
      atomicAdd((unsigned long long*)&a.ctl->active_labels,
                (unsigned long long)(-((long long)s_loff[emptied + 1] - s_loff[emptied])));
      atomicAdd(&a.ctl->active, -1);
    }
    if (__any_sync(kFullMask, emptied >= 0) && !start_queries(a, hdr, s_loff, lane, home)) {
      timed_out = true;
      break;
    }
  }
  if (timed_out && lane == 0) batch_timeout(a);
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

// After a launch that timed out the sub-queues may hold stale items: clear
// them (only then; a normal launch leaves every sub-queue empty).
__global__ void batch_reset_kernel(BatchArgs a) {
  if (a.ctl->last_status == 0) return;
  const long long tid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const long long nth = (long long)gridDim.x * blockDim.x;
  const long long ns = (long long)a.qs.Q << a.qs.cap_log2;
  for (long long i = tid; i < ns; i += nth) a.qs.slots[i] = 0ull;
  const long long nc = (long long)a.cq.Q << a.cq.cap_log2;
  for (long long i = tid; i < nc; i += nth) a.cq.slots[i] = 0ull;
  for (long long i = tid; i < a.qs.Q; i += nth) {
    a.qs.meta[i].count = 0; a.qs.meta[i].head = 0; a.qs.meta[i].tail = 0;
  }
  for (long long i = tid; i < a.cq.Q; i += nth) {
    a.cq.meta[i].count = 0; a.cq.meta[i].head = 0; a.cq.meta[i].tail = 0;
  }
}

// Labels of every query to (INF, -), each source to (0, 0) and queued in
// sub-queue q % Q; per-query counters and the launch counters reset.
__global__ void batch_init_kernel(BatchArgs a) {
  extern __shared__ int s_off[];
  const int nq = a.hdr->nq;
  for (int i = threadIdx.x; i <= nq; i += blockDim.x) s_off[i] = a.loff[i];
  __syncthreads();
  const long long tid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const long long nth = (long long)gridDim.x * blockDim.x;
  const long long total = s_off[nq];
  for (long long i = tid; i < total; i += nth) {
    const int q = find_query(s_off, nq, (int)i);
    const bool is_src = (i - s_off[q]) == a.desc[q].src;
    a.label[i] = is_src ? (pack_label(0, 0) | kQueuedBit) : kInfLabel;
  }
  const int window = a.hdr->window;
  for (long long q = tid; q < nq; q += nth) {
    a.qstatus[q] = 0;
    if (q >= window) {                       // started later by start_queries
      a.inflight[q * kCounterStride] = 0;
      continue;
    }
    QueueMeta* m = a.qs.meta + (q % a.qs.Q);
    const unsigned long long p = atomicAdd(&m->tail, 1ull);
    const unsigned lap = (unsigned)(p >> a.qs.cap_log2);
    a.qs.slots[((q % a.qs.Q) << a.qs.cap_log2) + (p & ((1ull << a.qs.cap_log2) - 1))] =
        ((unsigned long long)(2u * lap + 1u) << 32) | (unsigned)(s_off[q] + a.desc[q].src);
    atomicAdd(&m->count, 1);
    a.inflight[q * kCounterStride] = 1 + a.hdr->phantom;
  }
  if (tid == 0) {
    a.ctl->remaining = nq;
    a.ctl->next_q = window;
    a.ctl->active = window;
    a.ctl->active_labels = s_off[window];
    a.ctl->stop = 0;
    a.ctl->status = 0;
    for (int i = 0; i < 8; ++i) a.ctl->ctr[i] = 0;
  }
}

// Unpack every query's labels into its dist/hops arrays; status codes out.
__global__ void batch_epilogue_kernel(BatchArgs a) {
  extern __shared__ int s_off[];
  const int nq = a.hdr->nq;
  for (int i = threadIdx.x; i <= nq; i += blockDim.x) s_off[i] = a.loff[i];
  __syncthreads();
  const long long tid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const long long nth = (long long)gridDim.x * blockDim.x;
  const long long total = s_off[nq];
  for (long long i = tid; i < total; i += nth) {
    const int q = find_query(s_off, nq, (int)i);
    const QueryDesc& d = a.desc[q];
    const long long l = a.label[i];
    const int v = (int)(i - s_off[q]);
    const int dd = label_dist(l);
    d.dist[v] = dd;
    if (d.hops) d.hops[v] = (dd == kInf32) ? -1 : (int)label_hops(l);
  }
  const int gst = a.ctl->status;
  for (long long q = tid; q < nq; q += nth) {
    const int st = a.qstatus[q];
    int code = BFQ_OK;
    if (gst & (kStTimeout | kStQueue)) code = BFQ_ERR_TIMEOUT;
    else if (st & kStNegCycle) code = BFQ_NEG_CYCLE;
    else if (st & kStRange) code = BFQ_RANGE;
    a.qcode[q] = code;
  }
  if (tid == 0) a.ctl->last_status = (gst & (kStTimeout | kStQueue)) ? BFQ_ERR_TIMEOUT : 0;
}

int batch_ctas_per_sm() {
  int n = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, batch_persistent_kernel<true>, kBlock, 0) !=
      cudaSuccess)
    return 1;
  return n < 1 ? 1 : n;
}

int ceil_log2_ll(long long x) {
  int l = 0;
  while ((1LL << l) < x) ++l;
  return l;
}

}  // namespace
}  // namespace bfq

using namespace bfq;

struct bfq_batch {
  std::vector<bfq_graph_t> graphs;
  int maxq = 0;
  long long max_labels = 0;
  long long max_chunks = 0;
  bfq_tune tune{};
  BatchArgs args{};
  unsigned char* stage_host = nullptr;      // pinned
  unsigned char* stage_dev = nullptr;
  size_t stage_bytes = 0;
  int* qcode_host = nullptr;                // pinned
  int grid = 0;
  size_t dyn_smem = 0;
  cudaStream_t cap_stream = nullptr;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  cudaEvent_t ev0 = nullptr, ev1 = nullptr;
  long long bytes = 0;
  long long l2_bytes = 0;
  bool relax_min = false;                   // the captured persistent kernel's form
  std::vector<void*> allocs;

  int alloc(void** p, size_t n) {
    cudaError_t e = cudaMalloc(p, n ? n : 16);
    if (e != cudaSuccess) return cuda_fail(e, "cudaMalloc", __FILE__, __LINE__);
    allocs.push_back(*p);
    bytes += (long long)n;
    return BFQ_OK;
  }
  ~bfq_batch() {
    if (exec) cudaGraphExecDestroy(exec);
    if (graph) cudaGraphDestroy(graph);
    if (cap_stream) cudaStreamDestroy(cap_stream);
    if (ev0) cudaEventDestroy(ev0);
    if (ev1) cudaEventDestroy(ev1);
    for (void* p : allocs) cudaFree(p);
    if (stage_host) cudaFreeHost(stage_host);
    if (qcode_host) cudaFreeHost(qcode_host);
  }
};

// Graph internals the batch needs (defined in capi.cu).
namespace bfq {
struct GraphView {
  const int* row_ptr;
  const int2* adj;
  const int* hub_chunk0;
  const int4* chunk_tab;
  int V, n_chunks, hub_degree, chunk_edges;
};
int graph_view(bfq_graph_t g, GraphView* out);
}  // namespace bfq

static int b_invalid(const char* m) {
  set_error(m);
  return BFQ_ERR_INVALID;
}

static size_t stage_layout(int maxq, size_t* off_loff, size_t* off_coff, size_t* off_desc) {
  size_t o = sizeof(StageHeader);
  *off_loff = o;
  o += sizeof(int) * (maxq + 1);
  o = (o + 15) / 16 * 16;
  *off_coff = o;
  o += sizeof(int) * (maxq + 1);
  o = (o + 15) / 16 * 16;
  *off_desc = o;
  o += sizeof(QueryDesc) * maxq;
  return o;
}

// atomicMin relaxation while the label budget keeps the running queries'
// labels within half of L2.
static bool relax_min_for(const bfq_batch* b) {
  const int k = b->tune.batch_budget_klabels;
  const long long labels = k < 0 ? (1LL << 62) : k > 0 ? (long long)k << 10
                                                      : b->l2_bytes / 2 / (long long)sizeof(long long);
  return labels <= b->l2_bytes / 2 / (long long)sizeof(long long);
}

// Capture reset, init, persistent, epilogue and the two copies into one graph.
static int capture(bfq_batch* b) {
  BFQ_CUDA_TRY(cudaStreamBeginCapture(b->cap_stream, cudaStreamCaptureModeThreadLocal));
  cudaMemcpyAsync(b->stage_dev, b->stage_host, b->stage_bytes, cudaMemcpyHostToDevice,
                  b->cap_stream);
  const size_t smem_off = sizeof(int) * (b->maxq + 1);
  batch_reset_kernel<<<1024, 256, 0, b->cap_stream>>>(b->args);
  batch_init_kernel<<<2048, 256, smem_off, b->cap_stream>>>(b->args);
  b->relax_min = relax_min_for(b);
  if (b->relax_min)
    batch_persistent_kernel<true><<<b->grid, kBlock, b->dyn_smem, b->cap_stream>>>(b->args);
  else
    batch_persistent_kernel<false><<<b->grid, kBlock, b->dyn_smem, b->cap_stream>>>(b->args);
  batch_epilogue_kernel<<<2048, 256, smem_off, b->cap_stream>>>(b->args);
  cudaMemcpyAsync(b->qcode_host, b->args.qcode, sizeof(int) * b->maxq, cudaMemcpyDeviceToHost,
                  b->cap_stream);
  cudaError_t e = cudaStreamEndCapture(b->cap_stream, &b->graph);
  if (e != cudaSuccess) return cuda_fail(e, "cudaStreamEndCapture", __FILE__, __LINE__);
  BFQ_CUDA_TRY(cudaGraphInstantiate(&b->exec, b->graph, 0));
  return BFQ_OK;
}

extern "C" {

int bfq_batch_create(bfq_batch_t* out, const bfq_graph_t* graphs, int32_t ngraphs,
                     int32_t max_queries, int64_t max_total_vertices, const bfq_tune* tune) {
  if (!out) return b_invalid("bfq_batch_create: out is null");
  *out = nullptr;
  if (!graphs || ngraphs < 1) return b_invalid("bfq_batch_create: no graphs");
  if (max_queries < 1 || max_queries > 4096)
    return b_invalid("bfq_batch_create: max_queries must be in [1, 4096]");
  bfq_batch* b = new (std::nothrow) bfq_batch();
  if (!b) return b_invalid("bfq_batch_create: host allocation failed");
  bfq_tune_default(&b->tune);
  if (tune && (tune->cycle_walk_hops < 0 || tune->cycle_walk_hops == 1 ||
               tune->cycle_walk_hops > (1 << 30) || tune->batch_budget_klabels < -1)) {
    delete b;
    return b_invalid("bfq_batch_create: cycle_walk_hops or batch_budget_klabels out of range");
  }
  if (tune) {
    if (tune->share_div) b->tune.share_div = tune->share_div;
    if (tune->chunk_batch) b->tune.chunk_batch = tune->chunk_batch;
    if (tune->batch_items) b->tune.batch_items = tune->batch_items;
    if (tune->spin_limit) b->tune.spin_limit = tune->spin_limit;
    if (tune->time_limit_ms) b->tune.time_limit_ms = tune->time_limit_ms;
    if (tune->queues_per_cta) b->tune.queues_per_cta = tune->queues_per_cta;
    b->tune.test_phantom_items = tune->test_phantom_items;
    if (tune->cycle_walk_hops) b->tune.cycle_walk_hops = tune->cycle_walk_hops;
    b->tune.batch_budget_klabels = tune->batch_budget_klabels;
  }
  long long maxV = 0, maxC = 0;
  for (int i = 0; i < ngraphs; ++i) {
    GraphView gv;
    if (graph_view(graphs[i], &gv) != BFQ_OK) { delete b; return b_invalid("bfq_batch_create: bad graph handle"); }
    maxV = std::max<long long>(maxV, gv.V);
    maxC = std::max<long long>(maxC, gv.n_chunks);
    b->graphs.push_back(graphs[i]);
  }
  if (max_total_vertices <= 0) max_total_vertices = maxV * max_queries;
  if (max_total_vertices >= (1LL << 31))
    { delete b; return b_invalid("bfq_batch_create: max_total_vertices must be < 2^31"); }
  b->maxq = max_queries;
  b->max_labels = max_total_vertices;
  b->max_chunks = std::min<long long>(maxC * (long long)max_queries, (1LL << 31) - 1);

  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  int l2 = 0;
  cudaDeviceGetAttribute(&l2, cudaDevAttrL2CacheSize, dev);
  b->l2_bytes = l2;
  const size_t dyn = sizeof(int) * 2 * (max_queries + 1);
  b->dyn_smem = dyn;
  if (dyn > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(batch_persistent_kernel<true>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dyn);
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(batch_persistent_kernel<false>,
                               cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dyn);
    if (e != cudaSuccess) { delete b; return cuda_fail(e, "cudaFuncSetAttribute", __FILE__, __LINE__); }
  }
  int per_sm = 1;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, batch_persistent_kernel<true>, kBlock, dyn) !=
          cudaSuccess || per_sm < 1)
    per_sm = 1;
  b->grid = sms * per_sm;

  BatchArgs& a = b->args;
  a.maxq = max_queries;
  a.queues_per_cta = b->tune.queues_per_cta;
  const int Q = b->grid * a.queues_per_cta;
  a.qs.Q = Q;
  a.qs.cap_log2 = std::max(10, ceil_log2_ll((2 * max_total_vertices + Q - 1) / Q));
  a.cq.Q = b->grid;
  a.cq.cap_log2 = std::max(8, ceil_log2_ll((b->max_chunks + b->grid - 1) / b->grid));
  size_t o_loff, o_coff, o_desc;
  b->stage_bytes = stage_layout(max_queries, &o_loff, &o_coff, &o_desc);
  int rc = BFQ_OK;
#define B_TRY(x) do { rc = (x); if (rc != BFQ_OK) { delete b; return rc; } } while (0)
  B_TRY(b->alloc((void**)&b->stage_dev, b->stage_bytes));
  B_TRY(b->alloc((void**)&a.label, sizeof(long long) * (size_t)max_total_vertices));
  B_TRY(b->alloc((void**)&a.cyc, sizeof(long long) * (size_t)max_total_vertices));
  B_TRY(b->alloc((void**)&a.qs.meta, sizeof(QueueMeta) * Q));
  B_TRY(b->alloc((void**)&a.qs.slots, sizeof(unsigned long long) * ((size_t)Q << a.qs.cap_log2)));
  B_TRY(b->alloc((void**)&a.cq.meta, sizeof(QueueMeta) * a.cq.Q));
  B_TRY(b->alloc((void**)&a.cq.slots, sizeof(unsigned long long) * ((size_t)a.cq.Q << a.cq.cap_log2)));
  B_TRY(b->alloc((void**)&a.inflight, sizeof(int) * kCounterStride * max_queries));
  B_TRY(b->alloc((void**)&a.qstatus, sizeof(int) * max_queries));
  B_TRY(b->alloc((void**)&a.qcode, sizeof(int) * max_queries));
  B_TRY(b->alloc((void**)&a.ctl, sizeof(BatchCtl)));
#undef B_TRY
  a.hdr = (const StageHeader*)b->stage_dev;
  a.loff = (const int*)(b->stage_dev + o_loff);
  a.coff = (const int*)(b->stage_dev + o_coff);
  a.desc = (const QueryDesc*)(b->stage_dev + o_desc);
#define B_CUDA(x) do { cudaError_t e__ = (x); if (e__ != cudaSuccess) { int r__ = cuda_fail(e__, #x, __FILE__, __LINE__); delete b; return r__; } } while (0)
  B_CUDA(cudaMemset(a.cyc, 0xff, sizeof(long long) * (size_t)max_total_vertices));
  B_CUDA(cudaMemset(a.qs.meta, 0, sizeof(QueueMeta) * Q));
  B_CUDA(cudaMemset(a.qs.slots, 0, sizeof(unsigned long long) * ((size_t)Q << a.qs.cap_log2)));
  B_CUDA(cudaMemset(a.cq.meta, 0, sizeof(QueueMeta) * a.cq.Q));
  B_CUDA(cudaMemset(a.cq.slots, 0, sizeof(unsigned long long) * ((size_t)a.cq.Q << a.cq.cap_log2)));
  B_CUDA(cudaMemset(a.ctl, 0, sizeof(BatchCtl)));
  B_CUDA(cudaMallocHost((void**)&b->stage_host, b->stage_bytes));
  B_CUDA(cudaMallocHost((void**)&b->qcode_host, sizeof(int) * max_queries));
  std::memset(b->stage_host, 0, b->stage_bytes);
  B_CUDA(cudaStreamCreateWithFlags(&b->cap_stream, cudaStreamNonBlocking));
  B_CUDA(cudaEventCreate(&b->ev0));
  B_CUDA(cudaEventCreate(&b->ev1));
  B_CUDA(cudaDeviceSynchronize());
#undef B_CUDA
  rc = capture(b);
  if (rc != BFQ_OK) { delete b; return rc; }
  *out = b;
  return BFQ_OK;
}

int bfq_batch_destroy(bfq_batch_t b) {
  if (!b) return b_invalid("bfq_batch_destroy: null handle");
  cudaDeviceSynchronize();
  delete b;
  return BFQ_OK;
}

int64_t bfq_batch_device_bytes(bfq_batch_t b) { return b ? b->bytes : 0; }

int bfq_sssp_batch(bfq_batch_t b, int32_t nq, const int32_t* graph_id, const int32_t* src,
                   int32_t* const* dist, int32_t* const* hops, int32_t* status, void* stream) {
  if (!b) return b_invalid("bfq_sssp_batch: null handle");
  if (nq < 0 || nq > b->maxq) return b_invalid("bfq_sssp_batch: nq must be in [0, max_queries]");
  if (nq > 0 && (!graph_id || !src || !dist || !status))
    return b_invalid("bfq_sssp_batch: null argument");
  size_t o_loff, o_coff, o_desc;
  stage_layout(b->maxq, &o_loff, &o_coff, &o_desc);
  StageHeader* h = (StageHeader*)b->stage_host;
  int* loff = (int*)(b->stage_host + o_loff);
  int* coff = (int*)(b->stage_host + o_coff);
  QueryDesc* desc = (QueryDesc*)(b->stage_host + o_desc);
  long long lo = 0, co = 0;
  for (int q = 0; q < nq; ++q) {
    const int gi = graph_id[q];
    if (gi < 0 || gi >= (int)b->graphs.size()) return b_invalid("bfq_sssp_batch: graph id out of range");
    GraphView gv;
    graph_view(b->graphs[gi], &gv);
    if (src[q] < 0 || src[q] >= gv.V) return b_invalid("bfq_sssp_batch: source out of range");
    if (!dist[q]) return b_invalid("bfq_sssp_batch: null dist pointer");
    if (lo + gv.V > b->max_labels)
      return b_invalid("bfq_sssp_batch: the queries' vertices exceed max_total_vertices");
    QueryDesc& d = desc[q];
    d.row_ptr = gv.row_ptr;
    d.adj = gv.adj;
    d.hub_chunk0 = gv.hub_chunk0;
    d.chunk_tab = gv.chunk_tab;
    d.dist = dist[q];
    d.hops = hops ? hops[q] : nullptr;
    d.V = gv.V;
    d.src = src[q];
    d.hub_degree = gv.hub_degree;
    d.chunk_edges = gv.chunk_edges;
    d.label_off = (int)lo;
    d.chunk_off = (int)co;
    loff[q] = (int)lo;
    coff[q] = (int)co;
    lo += gv.V;
    co += gv.n_chunks;
  }
  if (co > b->max_chunks) return b_invalid("bfq_sssp_batch: too many hub chunks for this batch");
  loff[nq] = (int)lo;
  coff[nq] = (int)co;
  h->nq = nq;
  h->share_div = b->tune.share_div;
  h->chunk_batch = b->tune.chunk_batch;
  h->batch_items = b->tune.batch_items;
  h->phantom = b->tune.test_phantom_items;
  h->cyc_walk0 = b->tune.cycle_walk_hops;
  h->budget = b->tune.batch_budget_klabels < 0 ? (1LL << 62)
              : b->tune.batch_budget_klabels > 0 ? (long long)b->tune.batch_budget_klabels << 10
                                                 : b->l2_bytes / 2 / (long long)sizeof(long long);
  int window = 0;
  while (window < nq && (window == 0 || (long long)loff[window + 1] <= h->budget)) ++window;
  h->window = window;
  h->time_limit_ns = b->tune.time_limit_ms * 1000000LL;
  h->spin_limit = b->tune.spin_limit;
  cudaStream_t s = (cudaStream_t)stream;
  BFQ_CUDA_TRY(cudaEventRecord(b->ev0, s));
  BFQ_CUDA_TRY(cudaGraphLaunch(b->exec, s));
  BFQ_CUDA_TRY(cudaEventRecord(b->ev1, s));
  BFQ_CUDA_TRY(cudaStreamSynchronize(s));
  int rc = BFQ_OK;
  for (int q = 0; q < nq; ++q) {
    status[q] = b->qcode_host[q];
    if (status[q] == BFQ_ERR_TIMEOUT) rc = BFQ_ERR_TIMEOUT;
  }
  if (rc == BFQ_ERR_TIMEOUT) set_error("bfq_sssp_batch: a bounded device-side wait ran out");
  return rc;
}

int bfq_batch_get_stats(bfq_batch_t b, bfq_stats* out) {
  if (!b || !out) return b_invalid("bfq_batch_get_stats: null argument");
  std::memset(out, 0, sizeof(*out));
  BatchCtl c;
  BFQ_CUDA_TRY(cudaMemcpy(&c, b->args.ctl, sizeof(c), cudaMemcpyDeviceToHost));
  out->dequeued = (int64_t)c.ctr[kCtrDeq];
  out->relaxed = (int64_t)c.ctr[kCtrRel];
  out->updated = (int64_t)c.ctr[kCtrUpd];
  out->enqueued = (int64_t)c.ctr[kCtrEnq];
  out->steals = (int64_t)c.ctr[kCtrSteal];
  out->hub_chunks = (int64_t)c.ctr[kCtrChunk];
  out->idle_polls = (int64_t)c.ctr[kCtrIdle];
  out->grid = b->grid;
  out->block = kBlock;
  out->queues = b->args.qs.Q;
  out->queue_capacity = 1 << b->args.qs.cap_log2;
  float ms = 0.f;
  if (cudaEventElapsedTime(&ms, b->ev0, b->ev1) == cudaSuccess) out->kernel_ms = ms;
  cudaGetLastError();
  return BFQ_OK;
}

int bfq_batch_set_tune(bfq_batch_t b, const bfq_tune* t) {
  if (!b || !t) return b_invalid("bfq_batch_set_tune: null argument");
  if (t->share_div < 0 || t->chunk_batch < 0 || t->chunk_batch > 32 || t->batch_items < 0 ||
      t->batch_items > 32 || t->cycle_walk_hops < 0 || t->cycle_walk_hops == 1 ||
      t->cycle_walk_hops > (1 << 30) || t->batch_budget_klabels < -1)
    return b_invalid("bfq_batch_set_tune: parameter out of range");
  if (t->share_div) b->tune.share_div = t->share_div;
  if (t->chunk_batch) b->tune.chunk_batch = t->chunk_batch;
  if (t->batch_items) b->tune.batch_items = t->batch_items;
  if (t->time_limit_ms) b->tune.time_limit_ms = t->time_limit_ms;
  if (t->cycle_walk_hops) b->tune.cycle_walk_hops = t->cycle_walk_hops;
  b->tune.batch_budget_klabels = t->batch_budget_klabels;
  if (relax_min_for(b) != b->relax_min) {   // the captured kernel changes form
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->graph) cudaGraphDestroy(b->graph);
    b->exec = nullptr;
    b->graph = nullptr;
    return capture(b);
  }
  return BFQ_OK;
}

int bfq_batch_autotune(bfq_batch_t b, int32_t nq, const int32_t* graph_id, const int32_t* src,
                       int32_t* const* dist, int32_t* const* hops, bfq_tune* out, void* stream) {
  if (!b) return b_invalid("bfq_batch_autotune: null handle");
  static const int kShare[] = {1, 2, 4, 8};
  static const int kChunk[] = {2, 4, 8};
  static const int kItems[] = {16, 32};
  std::vector<int> st(std::max(1, (int)nq));
  const bfq_tune keep = b->tune;
  float best = -1.f;
  bfq_tune best_t = keep;
  for (int si : kShare)
    for (int ci : kChunk)
      for (int ii : kItems) {
        b->tune.share_div = si;
        b->tune.chunk_batch = ci;
        b->tune.batch_items = ii;
        float t_sum = 0.f;
        for (int rep = 0; rep < 2; ++rep) {
          int rc = bfq_sssp_batch(b, nq, graph_id, src, dist, hops, st.data(), stream);
          if (rc < 0) { b->tune = keep; return rc; }
          float ms = 0.f;
          cudaEventElapsedTime(&ms, b->ev0, b->ev1);
          if (rep == 1) t_sum = ms;
        }
        if (best < 0.f || t_sum < best) {
          best = t_sum;
          best_t = b->tune;
        }
      }
  b->tune = best_t;
  if (out) *out = best_t;
  return BFQ_OK;
}

}  // extern "C"
