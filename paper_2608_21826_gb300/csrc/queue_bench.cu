// Standalone Broker Queue (Sec. III-A, Algorithm 1) and the workloads of
// Sec. IV: "EnqDeq" (all enqueues, then all dequeues) and "Mixed" (even
// blocks enqueue while odd blocks dequeue, in one launch).  Operation i is
// executed by thread i of a grid-stride loop, as in Algorithm 2's
// per-partition loops.
#include <cstring>
#include <new>
#include <vector>

#include "bfq_internal.h"

namespace bfq {
namespace {

struct BQArgs {
  BQState* st;                 // per-thread variants
  unsigned* tickets;           // [N]
  int* ring;                   // [N]
  long long N;
  QueueSet qs;                 // warp variant (Q = 1)
  int* err;
  int variant;
  long long spin_limit;
};

// ENQUEUE (Algorithm 1): ensure, else report FULL when the ring really holds
// N items (BQ) or at once (BWD); then PUT_DATA.
__device__ __forceinline__ long long bq_enqueue(const BQArgs& q, int item, bool bwd) {
  long long spins = 0;
  for (;;) {
    if (bq_ensure_enqueue(q.st, (int)q.N)) break;
    if (bwd) return -1;
    const long long t = (long long)ld_relaxed_u64(&q.st->tail);
    const long long h = (long long)ld_relaxed_u64(&q.st->head);
    if (t - h >= q.N) return -1;
    if (++spins > q.spin_limit) { atomicOr(q.err, kStTimeout); return -1; }
  }
  const unsigned long long pos = atomicAdd(&q.st->tail, 1ull);
  const long long slot = (long long)(pos % (unsigned long long)q.N);
  const unsigned lap = (unsigned)(pos / (unsigned long long)q.N);
  if (!bq_wait_ticket(&q.tickets[slot], 2u * lap, q.spin_limit)) {
    atomicOr(q.err, kStTimeout);
    return -1;
  }
  q.ring[slot] = item;
  st_release_u32(&q.tickets[slot], 2u * lap + 1u);
  return (long long)pos;
}

// DEQUEUE (Algorithm 1): ensure, else report EMPTY when no item is held
// (BQ) or at once (BWD); then READ_DATA, releasing the slot for the next lap.
__device__ __forceinline__ long long bq_dequeue(const BQArgs& q, int* item, bool bwd) {
  long long spins = 0;
  for (;;) {
    if (bq_ensure_dequeue(q.st)) break;
    if (bwd) return -1;
    const long long t = (long long)ld_relaxed_u64(&q.st->tail);
    const long long h = (long long)ld_relaxed_u64(&q.st->head);
    if (t - h <= 0) return -1;
    if (++spins > q.spin_limit) { atomicOr(q.err, kStTimeout); return -1; }
  }
  const unsigned long long pos = atomicAdd(&q.st->head, 1ull);
  const long long slot = (long long)(pos % (unsigned long long)q.N);
  const unsigned lap = (unsigned)(pos / (unsigned long long)q.N);
  if (!bq_wait_ticket(&q.tickets[slot], 2u * lap + 1u, q.spin_limit)) {
    atomicOr(q.err, kStTimeout);
    return -1;
  }
  *item = q.ring[slot];
  st_release_u32(&q.tickets[slot], 2u * (lap + 1u));
  return (long long)pos;
}

// Warp-aggregated forms: the active lanes of a warp form one reservation and
// one ticket range.  BFQ_QUEUE_BQ_WARP reserves on the exact broker count
// (compare-and-swap); BFQ_QUEUE_BWD_WARP (qs.split) makes one single-shot
// fetch-add on the count of its own side (see wq_reserve).
__device__ __forceinline__ long long wq_enqueue_lanes(const BQArgs& q, bool active, int item,
                                                      int lane) {
  const unsigned mask = __ballot_sync(kFullMask, active);
  if (!mask) return -1;
  const int k = __popc(mask);
  const int rank = __popc(mask & ((1u << lane) - 1u));
  unsigned long long pos = 0;
  int got = 0;
  if (lane == 0) got = wq_reserve(q.qs.meta, k, false, 1 << q.qs.cap_log2, &pos, -1, q.qs.split);
  got = __shfl_sync(kFullMask, got, 0);
  pos = __shfl_sync(kFullMask, pos, 0);
  long long r = -1;
  if (active && rank < got) {
    if (wq_put(q.qs.slots, q.qs.cap_log2, pos + rank, (unsigned)item, q.spin_limit))
      r = (long long)(pos + rank);
    else
      atomicOr(q.err, kStTimeout);
  }
  if (q.qs.split) {
    __syncwarp();
    if (lane == 0) wq_after_put(q.qs.meta, got, 1);
  }
  return r;
}

__device__ __forceinline__ long long wq_dequeue_lanes(const BQArgs& q, bool active, int* item,
                                                      int lane) {
  const unsigned mask = __ballot_sync(kFullMask, active);
  if (!mask) return -1;
  const int k = __popc(mask);
  const int rank = __popc(mask & ((1u << lane) - 1u));
  unsigned long long pos = 0;
  int got = 0;
  if (lane == 0) got = wq_reserve(q.qs.meta, k, true, 1 << q.qs.cap_log2, &pos, -1, q.qs.split);
  got = __shfl_sync(kFullMask, got, 0);
  pos = __shfl_sync(kFullMask, pos, 0);
  long long r = -1;
  if (active && rank < got) {
    unsigned it = 0;
    if (wq_take(q.qs.slots, q.qs.cap_log2, pos + rank, &it, q.spin_limit)) {
      *item = (int)it;
      r = (long long)(pos + rank);
    } else {
      atomicOr(q.err, kStTimeout);
    }
  }
  if (q.qs.split) {
    __syncwarp();
    if (lane == 0) wq_after_take(q.qs.meta, got, 1);
  }
  return r;
}

// One op per thread over [0, n); `first`/`count` select the blocks taking
// part (every block, or the even / odd ones for Mixed).
__device__ __forceinline__ void op_range(long long n, int part_block, int part_blocks,
                                         long long* i0, long long* stride) {
  *i0 = (long long)part_block * blockDim.x + threadIdx.x;
  *stride = (long long)part_blocks * blockDim.x;
}

__device__ void run_enqueues(const BQArgs& q, const int* items, long long n, long long* pos_out,
                             int part_block, int part_blocks) {
  long long i0, stride;
  op_range(n, part_block, part_blocks, &i0, &stride);
  if (q.variant == BFQ_QUEUE_BQ_WARP || q.variant == BFQ_QUEUE_BWD_WARP) {
    const int lane = threadIdx.x & 31;
    // whole warps iterate together so the warp collectives stay converged
    const long long wbase0 = i0 - lane;
    for (long long wb = wbase0; wb < n; wb += stride) {
      const long long i = wb + lane;
      const bool act = i < n;
      const long long p = wq_enqueue_lanes(q, act, act ? items[i] : 0, lane);
      if (act && pos_out) pos_out[i] = p;
    }
  } else {
    const bool bwd = q.variant == BFQ_QUEUE_BWD;
    for (long long i = i0; i < n; i += stride) {
      const long long p = bq_enqueue(q, items[i], bwd);
      if (pos_out) pos_out[i] = p;
    }
  }
}

__device__ void run_dequeues(const BQArgs& q, int* out, long long n, long long* pos_out,
                             int part_block, int part_blocks) {
  long long i0, stride;
  op_range(n, part_block, part_blocks, &i0, &stride);
  if (q.variant == BFQ_QUEUE_BQ_WARP || q.variant == BFQ_QUEUE_BWD_WARP) {
    const int lane = threadIdx.x & 31;
    const long long wbase0 = i0 - lane;
    for (long long wb = wbase0; wb < n; wb += stride) {
      const long long i = wb + lane;
      const bool act = i < n;
      int item = 0;
      const long long p = wq_dequeue_lanes(q, act, &item, lane);
      if (act) {
        if (p >= 0) out[i] = item;
        if (pos_out) pos_out[i] = p;
      }
    }
  } else {
    const bool bwd = q.variant == BFQ_QUEUE_BWD;
    for (long long i = i0; i < n; i += stride) {
      int item = 0;
      const long long p = bq_dequeue(q, &item, bwd);
      if (p >= 0) out[i] = item;
      if (pos_out) pos_out[i] = p;
    }
  }
}

__global__ void queue_enqueue_kernel(BQArgs q, const int* items, long long n, long long* pos_out) {
  run_enqueues(q, items, n, pos_out, blockIdx.x, gridDim.x);
}

__global__ void queue_dequeue_kernel(BQArgs q, int* out, long long n, long long* pos_out) {
  run_dequeues(q, out, n, pos_out, blockIdx.x, gridDim.x);
}

__global__ void queue_mixed_kernel(BQArgs q, const int* items, long long n_enq, long long* enq_pos,
                                   int* out, long long n_deq, long long* deq_pos) {
  const int even_blocks = (gridDim.x + 1) / 2, odd_blocks = gridDim.x / 2;
  if ((blockIdx.x & 1) == 0)
    run_enqueues(q, items, n_enq, enq_pos, blockIdx.x / 2, even_blocks);
  else
    run_dequeues(q, out, n_deq, deq_pos, blockIdx.x / 2, odd_blocks);
}

}  // namespace
}  // namespace bfq

using namespace bfq;

struct bfq_queue {
  int variant = 0;
  long long N = 0;
  BQArgs args{};
  std::vector<void*> allocs;
  int alloc(void** p, size_t n) {
    cudaError_t e = cudaMalloc(p, n ? n : 16);
    if (e != cudaSuccess) return cuda_fail(e, "cudaMalloc", __FILE__, __LINE__);
    allocs.push_back(*p);
    return BFQ_OK;
  }
  ~bfq_queue() {
    for (void* p : allocs) cudaFree(p);
  }
};

static int q_invalid(const char* m) {
  set_error(m);
  return BFQ_ERR_INVALID;
}

static int launch_ok(const char* what) {
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(e, what, __FILE__, __LINE__);
  return BFQ_OK;
}

// L2 atomic throughput: mode 0 = every thread adds to its own counter
// (distinct addresses), 1 = every thread adds to one counter and uses the old
// value (as a ticket), 2 = one lane per warp moves one counter by 32 with a
// compare-and-swap loop (the exact-count reservation of the warp-aggregated
// queue), counting 32 operations per success.  Totals land in ctr.
__global__ void atomic_bench_kernel(unsigned long long* ctr, long long n_ops, int mode,
                                    unsigned long long* sink) {
  const long long tid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const long long nth = (long long)gridDim.x * blockDim.x;
  unsigned long long acc = 0;
  if (mode == 0) {
    for (long long i = tid; i < n_ops; i += nth) acc += atomicAdd(&ctr[tid], 1ull);
  } else if (mode == 1) {
    for (long long i = tid; i < n_ops; i += nth) acc ^= atomicAdd(&ctr[0], 1ull);
  } else {
    const int lane = threadIdx.x & 31;
    const long long warp = tid >> 5, nw = nth >> 5;
    for (long long i = warp; i < n_ops / 32; i += nw) {
      if (lane == 0) {
        unsigned long long old = ld_relaxed_u64(&ctr[0]);
        for (;;) {
          const unsigned long long seen = atomicCAS(&ctr[0], old, old + 32ull);
          if (seen == old) break;
          old = seen;
        }
        acc += old;
      }
      __syncwarp();
    }
  }
  if (acc == 0x5eed5eed5eed5eedull) *sink = acc;   // keeps the results live
}

// The relaxation step's memory pattern alone (no queues, no decisions): a
// stream of (col, w) pairs read lane-contiguously, 8 bytes per edge, and one
// 64-bit atomicMin per edge at label[col], two edges per lane in flight as in
// the SSSP kernel's merged walk.  The number of labels the atomics lowered is
// summed into *lowered.
__global__ void relax_bench_fill_kernel(int2* edges, long long n_edges, int n_labels,
                                        long long* label) {
  const long long tid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const long long nth = (long long)gridDim.x * blockDim.x;
  for (long long i = tid; i < n_edges; i += nth) {
    unsigned long long h = (unsigned long long)i * 0x9e3779b97f4a7c15ull;
    h ^= h >> 29;
    h *= 0xbf58476d1ce4e5b9ull;
    h ^= h >> 32;
    edges[i] = make_int2((int)(h % (unsigned long long)n_labels), (int)((h >> 40) & 255u));
  }
  for (long long v = tid; v < n_labels; v += nth) label[v] = kInfLabel;
}

// FILTER: load the label first and issue the atomicMin only when the key is
// below it (the load-filtered relaxation form).
template <bool FILTER>
__global__ void relax_bench_kernel(const int2* __restrict__ edges, long long n_edges,
                                   long long* label, unsigned long long* lowered) {
  const long long nth = (long long)gridDim.x * blockDim.x;
  const long long tid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  unsigned long long low = 0;
  const long long base_key = pack_label(1000, 1);
  for (long long i = tid; i < n_edges; i += 2 * nth) {
    const int2 e0 = __ldg(&edges[i]);
    const bool two = i + nth < n_edges;
    const int2 e1 = two ? __ldg(&edges[i + nth]) : make_int2(0, 0);
    const long long k0 = base_key + (long long)((unsigned long long)(long long)e0.y << 32);
    const long long k1 = base_key + (long long)((unsigned long long)(long long)e1.y << 32);
    long long o0, o1;
    if (FILTER) {
      o0 = ld_relaxed_s64(&label[e0.x]);
      o1 = two ? ld_relaxed_s64(&label[e1.x]) : k1;
      if (k0 < label_key(o0)) o0 = atomicMin(&label[e0.x], k0 | kQueuedBit);
      if (two && k1 < label_key(o1)) o1 = atomicMin(&label[e1.x], k1 | kQueuedBit);
    } else {
      o0 = atomicMin(&label[e0.x], k0 | kQueuedBit);
      o1 = two ? atomicMin(&label[e1.x], k1 | kQueuedBit) : k1;
    }
    low += (k0 < label_key(o0)) + (two && k1 < label_key(o1));
  }
  low = __reduce_add_sync(kFullMask, (unsigned)low);
  if ((threadIdx.x & 31) == 0) atomicAdd(lowered, low);
}

extern "C" {

static int check_launch(int32_t grid, int32_t block, int64_t n);

int bfq_relax_bench(int32_t mode, int64_t n_edges, int32_t n_labels, int32_t grid,
                    int32_t block, double* ms_out, int64_t* lowered_out, void* stream) {
  if (mode < 0 || mode > 1) return q_invalid("bfq_relax_bench: mode must be 0 or 1");
  if (n_edges < 1 || n_labels < 1) return q_invalid("bfq_relax_bench: n_edges and n_labels must be >= 1");
  int rc = check_launch(grid, block, n_edges);
  if (rc) return rc;
  cudaStream_t s = (cudaStream_t)stream;
  int2* edges = nullptr;
  long long* label = nullptr;
  unsigned long long* low = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaError_t e = cudaMalloc((void**)&edges, sizeof(int2) * (size_t)n_edges);
  if (e == cudaSuccess) e = cudaMalloc((void**)&label, sizeof(long long) * (size_t)n_labels);
  if (e == cudaSuccess) e = cudaMalloc((void**)&low, sizeof(unsigned long long));
  if (e == cudaSuccess) e = cudaMemsetAsync(low, 0, sizeof(unsigned long long), s);
  if (e == cudaSuccess) {
    relax_bench_fill_kernel<<<2048, 256, 0, s>>>(edges, n_edges, n_labels, label);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  if (e == cudaSuccess) e = cudaEventRecord(e0, s);
  if (e == cudaSuccess) {
    if (mode)
      relax_bench_kernel<true><<<grid, block, 0, s>>>(edges, n_edges, label, low);
    else
      relax_bench_kernel<false><<<grid, block, 0, s>>>(edges, n_edges, label, low);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaEventRecord(e1, s);
  if (e == cudaSuccess) e = cudaEventSynchronize(e1);
  float ms = 0.f;
  if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
  unsigned long long lowered = 0;
  if (e == cudaSuccess) e = cudaMemcpy(&lowered, low, sizeof(lowered), cudaMemcpyDeviceToHost);
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  cudaFree(edges);
  cudaFree(label);
  cudaFree(low);
  if (e != cudaSuccess) return cuda_fail(e, "bfq_relax_bench", __FILE__, __LINE__);
  if (ms_out) *ms_out = ms;
  if (lowered_out) *lowered_out = (int64_t)lowered;
  return BFQ_OK;
}

int bfq_atomic_bench(int32_t mode, int64_t n_ops, int32_t grid, int32_t block,
                     double* ms_out, int64_t* total_out, void* stream) {
  if (mode < 0 || mode > 2) return q_invalid("bfq_atomic_bench: mode must be 0, 1 or 2");
  int rc = check_launch(grid, block, n_ops);
  if (rc) return rc;
  if (mode == 2 && n_ops % 32) return q_invalid("bfq_atomic_bench: mode 2 needs n_ops % 32 == 0");
  cudaStream_t s = (cudaStream_t)stream;
  const size_t nctr = (size_t)grid * (size_t)block + 1;
  unsigned long long* ctr = nullptr;
  BFQ_CUDA_TRY(cudaMalloc((void**)&ctr, sizeof(unsigned long long) * nctr));
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaError_t e = cudaMemsetAsync(ctr, 0, sizeof(unsigned long long) * nctr, s);
  if (e == cudaSuccess) e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  if (e == cudaSuccess) e = cudaEventRecord(e0, s);
  if (e == cudaSuccess) {
    atomic_bench_kernel<<<grid, block, 0, s>>>(ctr, n_ops, mode, ctr + nctr - 1);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaEventRecord(e1, s);
  if (e == cudaSuccess) e = cudaEventSynchronize(e1);
  float ms = 0.f;
  if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
  long long total = 0;
  if (e == cudaSuccess && total_out) {
    std::vector<unsigned long long> h(nctr - 1);
    e = cudaMemcpy(h.data(), ctr, sizeof(unsigned long long) * (nctr - 1), cudaMemcpyDeviceToHost);
    for (unsigned long long v : h) total += (long long)v;
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  cudaFree(ctr);
  if (e != cudaSuccess) return cuda_fail(e, "bfq_atomic_bench", __FILE__, __LINE__);
  if (ms_out) *ms_out = ms;
  if (total_out) *total_out = total;
  return BFQ_OK;
}

int bfq_queue_create(bfq_queue_t* out, int64_t capacity, int32_t variant) {
  if (!out) return q_invalid("bfq_queue_create: out is null");
  *out = nullptr;
  if (capacity < 1 || capacity > (1LL << 30))
    return q_invalid("bfq_queue_create: capacity must be in [1, 2^30]");
  if (variant < BFQ_QUEUE_BQ || variant > BFQ_QUEUE_BWD_WARP)
    return q_invalid("bfq_queue_create: unknown variant");
  bfq_queue* q = new (std::nothrow) bfq_queue();
  if (!q) return q_invalid("bfq_queue_create: host allocation failed");
  q->variant = variant;
  BQArgs& a = q->args;
  a.variant = variant;
  a.spin_limit = 1LL << 22;
  int rc = q->alloc((void**)&a.err, sizeof(int));
  if (!rc && (variant == BFQ_QUEUE_BQ_WARP || variant == BFQ_QUEUE_BWD_WARP)) {
    int l = 0;
    while ((1LL << l) < capacity) ++l;
    q->N = 1LL << l;
    a.N = q->N;
    a.qs.Q = 1;
    a.qs.cap_log2 = l;
    a.qs.split = variant == BFQ_QUEUE_BWD_WARP ? 1 : 0;
    rc = q->alloc((void**)&a.qs.meta, sizeof(QueueMeta));
    if (!rc) rc = q->alloc((void**)&a.qs.slots, sizeof(unsigned long long) * (size_t)q->N);
  } else if (!rc) {
    q->N = capacity;
    a.N = capacity;
    rc = q->alloc((void**)&a.st, sizeof(BQState));
    if (!rc) rc = q->alloc((void**)&a.tickets, sizeof(unsigned) * (size_t)capacity);
    if (!rc) rc = q->alloc((void**)&a.ring, sizeof(int) * (size_t)capacity);
  }
  if (rc) { delete q; return rc; }
  *out = q;
  return bfq_queue_reset(q, nullptr) == BFQ_OK ? (cudaDeviceSynchronize(), BFQ_OK) : BFQ_ERR_CUDA;
}

int bfq_queue_destroy(bfq_queue_t q) {
  if (!q) return q_invalid("bfq_queue_destroy: null handle");
  cudaDeviceSynchronize();
  delete q;
  return BFQ_OK;
}

int bfq_queue_reset(bfq_queue_t q, void* stream) {
  if (!q) return q_invalid("bfq_queue_reset: null handle");
  cudaStream_t s = (cudaStream_t)stream;
  BQArgs& a = q->args;
  BFQ_CUDA_TRY(cudaMemsetAsync(a.err, 0, sizeof(int), s));
  if (q->variant == BFQ_QUEUE_BQ_WARP || q->variant == BFQ_QUEUE_BWD_WARP) {
    BFQ_CUDA_TRY(cudaMemsetAsync(a.qs.meta, 0, sizeof(QueueMeta), s));
    BFQ_CUDA_TRY(cudaMemsetAsync(a.qs.slots, 0, sizeof(unsigned long long) * (size_t)q->N, s));
  } else {
    BFQ_CUDA_TRY(cudaMemsetAsync(a.st, 0, sizeof(BQState), s));
    BFQ_CUDA_TRY(cudaMemsetAsync(a.tickets, 0, sizeof(unsigned) * (size_t)q->N, s));
    BFQ_CUDA_TRY(cudaMemsetAsync(a.ring, 0, sizeof(int) * (size_t)q->N, s));
  }
  return BFQ_OK;
}

static int check_launch(int32_t grid, int32_t block, int64_t n) {
  if (grid < 1 || block < 32 || block > 1024 || block % 32) return q_invalid("bfq_queue: grid >= 1 and block a multiple of 32 in [32, 1024]");
  if (n < 0) return q_invalid("bfq_queue: negative op count");
  return BFQ_OK;
}

int bfq_queue_enqueue(bfq_queue_t q, const int32_t* items, int64_t n, int64_t* pos_out,
                      int32_t grid, int32_t block, void* stream) {
  if (!q || (n > 0 && !items)) return q_invalid("bfq_queue_enqueue: null argument");
  int rc = check_launch(grid, block, n);
  if (rc) return rc;
  if (n == 0) return BFQ_OK;
  queue_enqueue_kernel<<<grid, block, 0, (cudaStream_t)stream>>>(q->args, items, n,
                                                                 (long long*)pos_out);
  return launch_ok("queue_enqueue_kernel");
}

int bfq_queue_dequeue(bfq_queue_t q, int32_t* out, int64_t n, int64_t* pos_out, int32_t grid,
                      int32_t block, void* stream) {
  if (!q || (n > 0 && !out)) return q_invalid("bfq_queue_dequeue: null argument");
  int rc = check_launch(grid, block, n);
  if (rc) return rc;
  if (n == 0) return BFQ_OK;
  queue_dequeue_kernel<<<grid, block, 0, (cudaStream_t)stream>>>(q->args, out, n,
                                                                 (long long*)pos_out);
  return launch_ok("queue_dequeue_kernel");
}

int bfq_queue_mixed(bfq_queue_t q, const int32_t* items, int64_t n_enq, int64_t* enq_pos,
                    int32_t* out, int64_t n_deq, int64_t* deq_pos, int32_t grid, int32_t block,
                    void* stream) {
  if (!q || (n_enq > 0 && !items) || (n_deq > 0 && !out))
    return q_invalid("bfq_queue_mixed: null argument");
  if (grid < 2) return q_invalid("bfq_queue_mixed: grid must be >= 2");
  int rc = check_launch(grid, block, n_enq < n_deq ? n_enq : n_deq);
  if (rc) return rc;
  queue_mixed_kernel<<<grid, block, 0, (cudaStream_t)stream>>>(
      q->args, items, n_enq, (long long*)enq_pos, out, n_deq, (long long*)deq_pos);
  return launch_ok("queue_mixed_kernel");
}

int bfq_queue_state(bfq_queue_t q, int64_t* head, int64_t* tail, int64_t* count, void* stream) {
  if (!q) return q_invalid("bfq_queue_state: null handle");
  cudaStream_t s = (cudaStream_t)stream;
  BFQ_CUDA_TRY(cudaStreamSynchronize(s));
  int err = 0;
  long long h = 0, t = 0, c = 0;
  BFQ_CUDA_TRY(cudaMemcpy(&err, q->args.err, sizeof(int), cudaMemcpyDeviceToHost));
  if (q->variant == BFQ_QUEUE_BQ_WARP || q->variant == BFQ_QUEUE_BWD_WARP) {
    QueueMeta m;
    BFQ_CUDA_TRY(cudaMemcpy(&m, q->args.qs.meta, sizeof(m), cudaMemcpyDeviceToHost));
    h = (long long)m.head;
    t = (long long)m.tail;
    c = m.count;
  } else {
    BQState st;
    BFQ_CUDA_TRY(cudaMemcpy(&st, q->args.st, sizeof(st), cudaMemcpyDeviceToHost));
    h = (long long)st.head;
    t = (long long)st.tail;
    c = st.count;
  }
  if (head) *head = h;
  if (tail) *tail = t;
  if (count) *count = c;
  if (err) {
    set_error("bfq_queue: a bounded ticket wait ran out");
    return BFQ_ERR_TIMEOUT;
  }
  return BFQ_OK;
}

}  // extern "C"
