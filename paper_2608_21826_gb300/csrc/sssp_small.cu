// Single-CTA query for small graphs (Algorithm 3 on one SM).  The labels, the
// recorded relaxation edges of the cycle accelerator and the vertex queue sit
// in shared memory, so each step of a deep, narrow search (a grid, a road
// network) costs shared-memory atomics instead of L2 round trips; the CSR
// stays in global memory and is read through L1.  The queue is one ring of
// vertex ids with a take ticket (head) and a fill ticket (tail): a warp
// reserves up to batch_items items with one compare-and-swap on head (the
// Broker Queue's warp-aggregated ensure step, Sec. III-A, at CTA scope),
// publishes its children with one fetch-add on tail, and every slot moves
// between empty and full with one atomic, so two tickets that meet on a
// slot can never take or fill it twice.  Termination, dedupe and the
// negative-cycle tests are those of the persistent kernel: an in-flight
// count, the in-queue flag in bit 0 of the label word, hops >= V, and
// walks of the recorded edges.
#include "bfq_internal.h"
#include "sssp_common.cuh"
#include "sssp_small.h"

namespace bfq {
namespace {

constexpr int kSmallChildBuf = 128;           // claimed children buffered per warp
constexpr unsigned kEmptySlot = 0xffffffffu;

struct SmallCtl {
  unsigned head;      // next ticket to take
  unsigned tail;      // next ticket to fill
  int inflight;       // items queued or being relaxed (termination at zero)
  int stop;           // 1: every warp leaves (cycle proved, or a wait ran out)
};

__device__ __forceinline__ int ld_volatile(const int* p) { return *(const volatile int*)p; }
__device__ __forceinline__ unsigned ld_volatile(const unsigned* p) {
  return *(const volatile unsigned*)p;
}
__device__ __forceinline__ long long ld_volatile(const long long* p) {
  return *(const volatile long long*)p;
}

__device__ __forceinline__ void small_raise(Control* ctl, SmallCtl* c, int bits) {
  atomicOr(&ctl->status, bits);
  *(volatile int*)&c->stop = 1;
}

// The cycle proof of prove_negative_cycle on the shared-memory records: a
// closed walk of recorded edges with negative total weight, through vertices
// that hold finite labels in this run, is a reachable negative cycle.
__device__ __noinline__ bool prove_cycle_shared(const long long* cyc, const long long* lab,
                                                int v, int V) {
  long long e = ld_volatile(cyc + v);
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
    e = ld_volatile(cyc + hare);
    hare = (int)(unsigned)e;
    ++lam;
    if (hare < 0 || hare >= V) return false;
  }
  long long sum = 0;
  int x = hare;
  for (int i = 0; i < lam; ++i) {
    if (label_dist(ld_volatile(lab + x)) == kInf32) return false;
    e = ld_volatile(cyc + x);
    const int y = (int)(unsigned)e;
    if (y < 0 || y >= V) return false;
    sum += (long long)(int)(e >> 32);
    x = y;
  }
  return x == hare && sum < 0;
}

// Publish the warp's buffered children and retire `retire` items in one
// update of the in-flight count, made before the children become visible.
// Returns false if a slot wait ran out (a wait also ends when the run is
// stopping, without failing: the results are unspecified then anyway).
__device__ __forceinline__ bool small_publish(const SsspArgs& a, SmallCtl* c, unsigned* ring,
                                              unsigned cap_mask, unsigned* buf, int& nbuf,
                                              int lane, WarpCounters& wc, int retire) {
  __syncwarp();
  if (lane == 0 && nbuf - retire != 0) atomicAdd(&c->inflight, nbuf - retire);
  bool ok = true;
  if (nbuf > 0) {
    // the children's labels (and this warp's earlier label atomics) are
    // ordered before the slots that name them
    __threadfence_block();
    unsigned p = 0;
    if (lane == 0) p = atomicAdd(&c->tail, (unsigned)nbuf);
    p = __shfl_sync(kFullMask, p, 0);
    for (int i = lane; i < nbuf; i += 32) {
      unsigned* sl = &ring[(p + (unsigned)i) & cap_mask];
      long long spins = 0;
      while (atomicCAS(sl, kEmptySlot, buf[i]) != kEmptySlot) {
        if (ld_volatile(&c->stop)) break;
        if (++spins > a.spin_limit) {
          ok = false;
          break;
        }
        __nanosleep(32);
      }
    }
    if (lane == 0) wc.enq += (unsigned)nbuf;
  }
  __syncwarp();
  nbuf = 0;
  return __all_sync(kFullMask, ok);
}

// Merged relaxation of the batch held by lanes [0, n): the same staged,
// lane-contiguous walk as the persistent kernel's, with one atomicMin on the
// shared-memory label per edge.  Returns false if a slot wait ran out.
__device__ __forceinline__ bool small_relax(const SsspArgs& a, long long* lab, long long* cyc,
                                            SmallCtl* c, unsigned* ring, unsigned cap_mask,
                                            int n, int beg, int deg, long long lb, int tail,
                                            int lane, WarpCounters& wc, unsigned* buf, int& nbuf,
                                            unsigned& walk_at, BatchStage* st) {
  constexpr int U = 2;
  const bool has = lane < n && deg > 0;
  const unsigned hm = __ballot_sync(kFullMask, has);
  if (!hm) return true;
  int total = 0;
  const int excl = warp_excl_scan(has ? deg : 0, lane, &total);
  wc.rel += (lane == 0) ? (unsigned)total : 0u;
  if (has) {
    const int r = __popc(hm & lanemask_lt());
    st->key0[r] = pack_label(label_dist(lb), label_hops(lb) + 1u);
    st->off[r] = beg - excl;
    st->tail[r] = tail;
  }
  __syncwarp();
  const unsigned V = (unsigned)a.V;
  for (int base = 0; base < total; base += 32 * U) {
    int2 cw[U];
    int own[U];
    long long key[U], cur[U];
    bool act[U];
#pragma unroll
    for (int g = 0; g < U; ++g) {
      act[g] = false;
      own[g] = 0;
      cw[g] = make_int2(0, 0);
      const int P = base + 32 * g;
      if (P < total) {                    // warp-uniform
        own[g] = staged_owner(has, excl, P);
        if (P + lane < total) {
          act[g] = true;
          cw[g] = __ldg(&a.adj[st->off[own[g]] + P + lane]);
        }
      }
    }
#pragma unroll
    for (int g = 0; g < U; ++g) {
      key[g] = 0;
      cur[g] = 0;
      if (act[g]) {
        const int cnd = edge_candidate(st->key0[own[g]], cw[g].y, &key[g]);
        if (cnd < 0) atomicOr(&a.ctl->status, kStRange);
        act[g] = cnd > 0;
        if (act[g]) cur[g] = atomicMin(&lab[cw[g].x], key[g] | kQueuedBit);
      }
    }
    bool enq[U];
#pragma unroll
    for (int g = 0; g < U; ++g) {
      enq[g] = false;
      if (act[g] && key[g] < label_key(cur[g])) {
        ++wc.upd;
        const unsigned nh = label_hops(key[g]);
        bool proven = nh >= V;            // a walk of >= V edges that still improved
        if (!proven && nh >= (a.cyc_walk0 >> 1)) {
          *(volatile long long*)(cyc + cw[g].x) = pack_edge(st->tail[own[g]], cw[g].y);
          if (nh >= walk_at) {
            if (prove_cycle_shared(cyc, lab, cw[g].x, a.V))
              proven = true;
            else
              walk_at = nh * 2;
          }
        }
        if (proven)
          small_raise(a.ctl, c, kStNegCycle);
        else
          enq[g] = !(cur[g] & kQueuedBit);
      }
    }
#pragma unroll
    for (int g = 0; g < U; ++g) {
      const unsigned m = __ballot_sync(kFullMask, enq[g]);
      if (m) {
        if (nbuf + __popc(m) > kSmallChildBuf) {
          if (!small_publish(a, c, ring, cap_mask, buf, nbuf, lane, wc, 0)) return false;
        }
        if (enq[g]) buf[nbuf + __popc(m & lanemask_lt())] = (unsigned)cw[g].x;
        nbuf += __popc(m);
      }
    }
  }
  __syncwarp();                         // stage free for the next batch
  return true;
}

// One CTA of BLOCK threads (1024, or 512: fewer warps contend for the ring
// on deep, narrow searches) runs the whole query; dynamic shared memory
// holds labels[V], recorded edges[V] and the ring (2^cap_log2 >= V slots).
// On exit the labels are written to a.label, for the epilogue and pred
// kernels.
template <int BLOCK>
__global__ void __launch_bounds__(BLOCK, 1) sssp_small_kernel(SsspArgs a, int cap_log2) {
  constexpr int kSmallBlock = BLOCK;
  constexpr int kSmallWarps = BLOCK / 32;
  extern __shared__ __align__(16) unsigned char s_dyn[];
  long long* lab = reinterpret_cast<long long*>(s_dyn);
  long long* cyc = lab + a.V;
  unsigned* ring = reinterpret_cast<unsigned*>(cyc + a.V);
  __shared__ SmallCtl c;
  __shared__ BatchStage s_stage[kSmallWarps];
  __shared__ unsigned s_child[kSmallWarps][kSmallChildBuf];
  const int lane = threadIdx.x & 31;
  const int wid = threadIdx.x >> 5;
  const unsigned cap_mask = (1u << cap_log2) - 1u;
  const int V = a.V;

  // A persistent run that ended early left items in the handle's global
  // sub-queues, and its init would clear them; this run does not use them
  // but will report its own status, so it empties them here (every
  // allocated sub-queue, as that init does), and the next persistent run
  // starts from clean queues whatever this one reports.
  if (a.ctl->last_status != 0) {
    const int q_all = a.q_alloc > 0 ? a.q_alloc : a.qs.Q;
    const int cq_all = a.cq_alloc > 0 ? a.cq_alloc : a.cq.Q;
    const long long nslots = (long long)q_all << a.qs.cap_log2;
    for (long long i = threadIdx.x; i < nslots; i += kSmallBlock) a.qs.slots[i] = 0ull;
    const long long ncslots = (long long)cq_all << a.cq.cap_log2;
    for (long long i = threadIdx.x; i < ncslots; i += kSmallBlock) a.cq.slots[i] = 0ull;
    for (int q = threadIdx.x; q < q_all; q += kSmallBlock) {
      a.qs.meta[q].count = 0;
      a.qs.meta[q].used = 0;
      a.qs.meta[q].head = 0;
      a.qs.meta[q].tail = 0;
    }
    for (int q = threadIdx.x; q < cq_all; q += kSmallBlock) {
      a.cq.meta[q].count = 0;
      a.cq.meta[q].used = 0;
      a.cq.meta[q].head = 0;
      a.cq.meta[q].tail = 0;
    }
  }
  for (int v = threadIdx.x; v < V; v += kSmallBlock) {
    lab[v] = (v == a.src) ? (pack_label(0, 0) | kQueuedBit) : kInfLabel;
    cyc[v] = pack_edge(-1, 0);            // no record: a walk from here fails
  }
  for (unsigned i = threadIdx.x; i <= cap_mask; i += kSmallBlock)
    ring[i] = (i == 0) ? (unsigned)a.src : kEmptySlot;
  if (threadIdx.x == 0) {
    c.head = 0;
    c.tail = 1;
    c.inflight = 1 + a.phantom;
    c.stop = 0;
    a.ctl->status = 0;
    a.ctl->stop = 0;
    a.ctl->inflight = 0;
    for (int i = 0; i < 8; ++i) a.ctl->ctr[i] = 0;
  }
  __syncthreads();

  WarpCounters wc;
  unsigned walk_at = a.cyc_walk0;
  const unsigned long long t_start = globaltimer_ns();
  const int share = a.share_div > 0 ? a.share_div : kSmallWarps;
  BatchStage* st = &s_stage[wid];
  unsigned* buf = s_child[wid];
  int nbuf = 0;
  int idle = 0;
  unsigned iter = 0;
  bool timed_out = false;
  for (;;) {
    // Every way out of the loop is decided by lane 0 and broadcast: lanes
    // can run apart after a sleep, and a lane that read the stop flag (or
    // the clock) differently would leave its warp short at the next
    // warp-wide operation.  Busy warps check the time limit too, so a run
    // that never runs dry still ends.
    int leave = 0;
    if (lane == 0) {
      if (ld_volatile(&c.stop))
        leave = 1;
      else if ((++iter & 255u) == 0 &&
               (long long)(globaltimer_ns() - t_start) > a.time_limit_ns)
        leave = 2;
    }
    leave = __shfl_sync(kFullMask, leave, 0);
    if (leave) {
      timed_out = leave == 2;
      break;
    }
    int got = 0;
    unsigned h = 0;
    if (lane == 0) {
      unsigned hh = ld_volatile(&c.head);
      for (;;) {
        const int avail = (int)(ld_volatile(&c.tail) - hh);
        if (avail <= 0) break;
        const int take = share_of(avail, a.batch_items, share);
        const unsigned old = atomicCAS(&c.head, hh, hh + (unsigned)take);
        if (old == hh) {
          got = take;
          h = hh;
          break;
        }
        hh = old;
      }
    }
    got = __shfl_sync(kFullMask, got, 0);
    h = __shfl_sync(kFullMask, h, 0);
    if (got == 0) {
      int done = 0;
      if (lane == 0) {
        if (ld_volatile(&c.inflight) == 0)
          done = 1;
        else if (((idle + 1) & 31) == 0 &&
                 (long long)(globaltimer_ns() - t_start) > a.time_limit_ns)
          done = 2;
      }
      done = __shfl_sync(kFullMask, done, 0);
      if (done) {
        timed_out = done == 2;
        break;
      }
      ++wc.idle;
      __nanosleep(min(32u << min(idle, 5), 1024u));
      ++idle;
      continue;
    }
    idle = 0;
    wc.deq += (lane == 0) ? (unsigned)got : 0u;
    unsigned item = 0;
    bool ok = true, stopped = false;
    if (lane < got) {
      unsigned* sl = &ring[(h + (unsigned)lane) & cap_mask];
      long long spins = 0;
      for (;;) {
        const unsigned x = atomicExch(sl, kEmptySlot);
        if (x != kEmptySlot) {
          item = x;
          break;
        }
        if (ld_volatile(&c.stop)) {
          stopped = true;
          break;
        }
        if (++spins > a.spin_limit) {
          ok = false;
          break;
        }
        __nanosleep(32);
      }
    }
    if (!__all_sync(kFullMask, ok)) {
      timed_out = true;
      break;
    }
    if (__any_sync(kFullMask, stopped)) break;
    // the slot is read before the label it names (the producer ordered the
    // label before the slot)
    __threadfence_block();
    int beg = 0, deg = 0, tail = 0;
    long long lb = 0;
    if (lane < got) {
      tail = (int)item;
      // clear the in-queue flag and read the label in one atomic: any later
      // improvement sees the flag clear and queues the vertex again
      lb = label_key((long long)atomicAnd((unsigned long long*)&lab[item],
                                          ~(unsigned long long)kQueuedBit));
      beg = __ldg(&a.row_ptr[item]);
      deg = __ldg(&a.row_ptr[item + 1]) - beg;
    }
    if (!small_relax(a, lab, cyc, &c, ring, cap_mask, got, beg, deg, lb, tail, lane, wc, buf,
                     nbuf, walk_at, st) ||
        !small_publish(a, &c, ring, cap_mask, buf, nbuf, lane, wc, got)) {
      timed_out = true;
      break;
    }
  }
  if (timed_out && lane == 0) small_raise(a.ctl, &c, kStTimeout);
  __syncthreads();
  for (int v = threadIdx.x; v < V; v += kSmallBlock) a.label[v] = lab[v];
  const unsigned long long upd_sum = warp_sum_u64(wc.upd);
  if (lane == 0) {
    if (wc.deq) atomicAdd(&a.ctl->ctr[kCtrDeq], (unsigned long long)wc.deq);
    if (wc.rel) atomicAdd(&a.ctl->ctr[kCtrRel], (unsigned long long)wc.rel);
    if (upd_sum) atomicAdd(&a.ctl->ctr[kCtrUpd], upd_sum);
    if (wc.enq) atomicAdd(&a.ctl->ctr[kCtrEnq], (unsigned long long)wc.enq);
    if (wc.idle) atomicAdd(&a.ctl->ctr[kCtrIdle], (unsigned long long)wc.idle);
  }
}

}  // namespace

// Dynamic shared memory of a small run over V vertices with a ring of
// 2^cap_log2 slots.
size_t sssp_small_smem(int V, int cap_log2) {
  return sizeof(long long) * 2 * (size_t)V + sizeof(unsigned) * ((size_t)1 << cap_log2);
}

// Largest dynamic shared memory the small kernel can use on the current
// device, the least over its two block sizes (0 when the attribute cannot
// be set).
template <int BLOCK>
static size_t small_smem_limit_of(int optin) {
  cudaFuncAttributes fa{};
  if (cudaFuncGetAttributes(&fa, sssp_small_kernel<BLOCK>) != cudaSuccess) return 0;
  if ((size_t)optin <= fa.sharedSizeBytes) return 0;
  const size_t dyn = (size_t)optin - fa.sharedSizeBytes;
  if (cudaFuncSetAttribute(sssp_small_kernel<BLOCK>,
                           cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dyn) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  return dyn;
}

size_t sssp_small_smem_limit() {
  int dev = 0, optin = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return 0;
  if (cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess)
    return 0;
  return std::min(small_smem_limit_of<1024>(optin), small_smem_limit_of<512>(optin));
}

cudaError_t launch_sssp_small_threads(const SsspArgs& a, int cap_log2, int threads,
                                      int32_t* status_dev, cudaEvent_t ev0, cudaEvent_t ev1,
                                      cudaStream_t s) {
  if (ev0) cudaEventRecord(ev0, s);
  const size_t smem = sssp_small_smem(a.V, cap_log2);
  if (threads == 512)
    sssp_small_kernel<512><<<1, 512, smem, s>>>(a, cap_log2);
  else
    sssp_small_kernel<1024><<<1, 1024, smem, s>>>(a, cap_log2);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  if (ev1) cudaEventRecord(ev1, s);
  return launch_sssp_epilogue(a, LaunchShape{(a.V + 255) / 256 < 1024 ? (a.V + 255) / 256 : 1024,
                                             256},
                              status_dev, nullptr, s);
}

cudaError_t launch_sssp_small(const SsspArgs& a, int cap_log2, int32_t* status_dev,
                              cudaEvent_t ev0, cudaEvent_t ev1, cudaStream_t s) {
  return launch_sssp_small_threads(a, cap_log2, 1024, status_dev, ev0, ev1, s);
}

}  // namespace bfq
