// Round-based Bellman-Ford (Algorithm 3's formulation on one GPU).
//
// Each round relaxes edges of the edge list in parallel and counts the
// successful label decreases (the change counter of Algorithm 3); the run
// ends after a round with no change.  A change in round V means a reachable
// negative cycle (labels are final after V - 1 rounds otherwise), and so does
// a label of V or more hops, which usually fires much earlier.  Labels are the
// same packed (dist, hops) words as the queue-driven kernel, lowered with
// compare-and-swap, so the fixed point is the same lexicographic minimum.
//
// GB300 mapping: one cooperative launch runs every round, separated by a
// grid-wide barrier (a monotone arrival counter, bounded spin), so there is
// no host round trip per round.  The edge list is cut into contiguous chunks
// of kChunk edges (CSR order, so tails are sorted); by default a round skips
// every chunk whose tail range holds no vertex changed in the previous round
// (a bitmap per round, three in rotation so clearing overlaps the next round)
// and, inside a chunk, every edge whose tail did not change.  This filter
// leaves the fixed point unchanged.  BFQ_ROUNDS_ALL_EDGES relaxes every edge
// of every round, as Algorithm 3 prints it.
#include "bfq_internal.h"
#include "sssp_common.cuh"

namespace bfq {
namespace {

constexpr int kRoundsBlock = 512;
constexpr int kChunkLog2 = 10;
constexpr long long kChunk = 1LL << kChunkLog2;
constexpr int kRoundGroups = 4;     // 32-edge steps of a chunk in flight per warp

// Device counters of one run (one 64-bit word each, own 128-byte line).
struct alignas(128) RoundsCtl {
  unsigned long long bar;            // grid-barrier arrivals
  unsigned long long pad0[15];
  unsigned long long changes[3];     // change counter of rounds r % 3
  unsigned long long pad1[13];
  int stat[3];                       // kSt* bits raised in rounds r % 3
  int pad2[29];
  unsigned long long rounds;         // rounds run
  unsigned long long relaxed;        // edges relaxed
  unsigned long long updated;        // sum of the change counters
  int status;                        // final kSt* bits
  int pad3[25];
};

struct RoundsArgs {
  const int2* adj;        // [E] (col, w)
  const int* tail;        // [E] tail of each edge
  const int2* chunk_rng;  // [n_chunks] first and last tail of each chunk
  long long* label;       // [V]
  unsigned* bits;         // [3 * words]
  RoundsCtl* ctl;
  long long E;
  long long words;
  long long n_chunks;
  long long max_rounds;   // V
  long long spin_limit;
  long long time_limit_ns;
  int V;
  int filter;             // 1: skip edges whose tail did not change
};

__global__ void rounds_tail_kernel(const int* __restrict__ row_ptr, int V, int* __restrict__ tail) {
  const int lane = threadIdx.x & 31;
  const long long warp = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const long long nw = ((long long)gridDim.x * blockDim.x) >> 5;
  for (long long v = warp; v < V; v += nw)
    for (int e = row_ptr[v] + lane; e < row_ptr[v + 1]; e += 32) tail[e] = (int)v;
}

__global__ void rounds_chunk_kernel(const int* __restrict__ tail, long long E, long long n_chunks,
                                    int2* __restrict__ rng) {
  for (long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x; c < n_chunks;
       c += (long long)gridDim.x * blockDim.x) {
    const long long e0 = c << kChunkLog2;
    const long long e1 = (e0 + kChunk < E ? e0 + kChunk : E) - 1;
    rng[c] = make_int2(tail[e0], tail[e1]);
  }
}

__global__ void rounds_init_kernel(long long* label, unsigned* bits, long long words, int V,
                                   int src, RoundsCtl* ctl) {
  const long long tid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const long long nth = (long long)gridDim.x * blockDim.x;
  for (long long v = tid; v < V; v += nth) label[v] = (v == src) ? pack_label(0, 0) : kInfLabel;
  for (long long i = tid; i < 3 * words; i += nth)
    bits[i] = (i == (src >> 5)) ? (1u << (src & 31)) : 0u;
  if (tid == 0) {
    ctl->bar = 0;
    for (int k = 0; k < 3; ++k) {
      ctl->changes[k] = 0;
      ctl->stat[k] = 0;
    }
    ctl->rounds = ctl->relaxed = ctl->updated = 0;
    ctl->status = 0;
  }
}

// Grid-wide barrier: the k-th barrier of the run completes once every block
// has arrived k times.  Returns false (in every thread of the block) when
// the wait ran out.
__device__ __forceinline__ bool grid_barrier(unsigned long long* bar, unsigned long long target,
                                             long long spin_limit) {
  __shared__ int s_ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    atomicAdd(bar, 1ull);
    long long polls = 0;
    int ok = 1;
    while (ld_acquire_u64(bar) < target) {
      if (++polls > spin_limit) {
        ok = 0;
        break;
      }
      __nanosleep(64);
    }
    __threadfence();
    s_ok = ok;
  }
  __syncthreads();
  return s_ok != 0;
}

__global__ void __launch_bounds__(kRoundsBlock) rounds_kernel(RoundsArgs a) {
  __shared__ unsigned long long s_sum[kRoundsBlock / 32];
  __shared__ int s_st;
  const int lane = threadIdx.x & 31;
  const int wib = threadIdx.x >> 5;
  const long long tid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const long long nth = (long long)gridDim.x * blockDim.x;
  const long long gw = tid >> 5;
  const long long nw = nth >> 5;
  RoundsCtl* c = a.ctl;
  const unsigned long long t0 = globaltimer_ns();
  unsigned long long relaxed = 0, updated = 0;
  long long r = 0;
  int final_st = 0;
  bool ran_out = false;
  for (; r < a.max_rounds; ++r) {
    const unsigned* cur = a.bits + (r % 3) * a.words;
    unsigned* nxt = a.bits + ((r + 1) % 3) * a.words;
    unsigned* clr = a.bits + ((r + 2) % 3) * a.words;
    // The previous round's input bitmap is free now: clear it for round r + 1.
    for (long long i = tid; i < a.words; i += nth) clr[i] = 0u;
    if (tid == 0) {
      c->changes[(r + 1) % 3] = 0;
      c->stat[(r + 1) % 3] = 0;
    }
    if (threadIdx.x == 0) s_st = 0;
    __syncthreads();
    unsigned long long ch = 0;
    int st = 0;
    for (long long k = gw; k < a.n_chunks; k += nw) {
      const long long e0 = k << kChunkLog2;
      const long long e1 = (e0 + kChunk < a.E) ? e0 + kChunk : a.E;
      if (a.filter) {
        const int2 rg = __ldg(a.chunk_rng + k);
        bool any = false;
        for (int wd = (rg.x >> 5) + lane; wd <= (rg.y >> 5); wd += 32) any |= cur[wd] != 0u;
        if (!__any_sync(kFullMask, any)) continue;
      }
      for (long long e = e0 + lane; e < e1; e += 32LL * kRoundGroups) {
        int u[kRoundGroups];
        bool act[kRoundGroups];
        int2 cw[kRoundGroups];
        long long key[kRoundGroups], old[kRoundGroups];
#pragma unroll
        for (int g = 0; g < kRoundGroups; ++g) {
          act[g] = e + 32LL * g < e1;
          u[g] = act[g] ? __ldg(a.tail + e + 32LL * g) : 0;
        }
#pragma unroll
        for (int g = 0; g < kRoundGroups; ++g)
          if (a.filter && act[g]) act[g] = (cur[u[g] >> 5] >> (u[g] & 31)) & 1u;
#pragma unroll
        for (int g = 0; g < kRoundGroups; ++g) {
          if (!act[g]) continue;
          ++relaxed;
          cw[g] = __ldg(a.adj + e + 32LL * g);
          key[g] = ld_relaxed_s64(a.label + u[g]);
        }
#pragma unroll
        for (int g = 0; g < kRoundGroups; ++g) {
          if (!act[g]) continue;
          const long long lu = key[g];
          const long long nd = (long long)label_dist(lu) + cw[g].y;
          if (label_dist(lu) == kInf32 || nd >= (long long)kInf32) {
            act[g] = false;
          } else if (nd <= -2147483648LL) {
            st |= kStRange;
            act[g] = false;
          } else {
            key[g] = pack_label((int)nd, label_hops(lu) + 1u);
            old[g] = ld_relaxed_s64(a.label + cw[g].x);
          }
        }
        // first compare-and-swap of every group back to back (they overlap)
        long long prev[kRoundGroups];
#pragma unroll
        for (int g = 0; g < kRoundGroups; ++g) {
          prev[g] = old[g];
          if (act[g] && key[g] < old[g])
            prev[g] = (long long)atomicCAS((unsigned long long*)(a.label + cw[g].x),
                                           (unsigned long long)old[g],
                                           (unsigned long long)key[g]);
          else
            act[g] = false;
        }
#pragma unroll
        for (int g = 0; g < kRoundGroups; ++g) {
          if (!act[g]) continue;
          if (prev[g] == old[g]) {
            ++ch;
            if (label_hops(key[g]) >= (unsigned)a.V) st |= kStNegCycle;
            atomicOr(nxt + (cw[g].x >> 5), 1u << (cw[g].x & 31));
            continue;
          }
          long long o = prev[g];
          while (key[g] < o) {
            const long long seen = (long long)atomicCAS((unsigned long long*)(a.label + cw[g].x),
                                                        (unsigned long long)o,
                                                        (unsigned long long)key[g]);
            if (seen == o) {
              ++ch;
              if (label_hops(key[g]) >= (unsigned)a.V) st |= kStNegCycle;
              atomicOr(nxt + (cw[g].x >> 5), 1u << (cw[g].x & 31));
              break;
            }
            o = seen;
          }
        }
      }
    }
    updated += ch;
    // block sums of this round's changes, then one atomic per block
    ch = warp_sum_u64(ch);
    if (st) atomicOr(&s_st, st);
    if (lane == 0) s_sum[wib] = ch;
    __syncthreads();
    if (threadIdx.x == 0) {
      unsigned long long b = 0;
      for (int i = 0; i < kRoundsBlock / 32; ++i) b += s_sum[i];
      if (b) atomicAdd(&c->changes[r % 3], b);
      int bst = s_st;
      if (globaltimer_ns() - t0 > (unsigned long long)a.time_limit_ns) bst |= kStTimeout;
      if (bst) atomicOr(&c->stat[r % 3], bst);
    }
    if (!grid_barrier(&c->bar, (unsigned long long)(r + 1) * gridDim.x, a.spin_limit)) {
      ran_out = true;
      final_st = kStTimeout;
      ++r;
      break;
    }
    const unsigned long long changes = ld_relaxed_u64(&c->changes[r % 3]);
    const int rst = ld_relaxed_s32(&c->stat[r % 3]);
    if (rst) {
      final_st = rst;
      ++r;
      break;
    }
    if (changes == 0) {
      ++r;
      break;
    }
    if (r + 1 == a.max_rounds) final_st = kStNegCycle;   // still changing in round V
  }
  relaxed = warp_sum_u64(relaxed);
  updated = warp_sum_u64(updated);
  if (lane == 0) {
    if (relaxed) atomicAdd(&c->relaxed, relaxed);
    if (updated) atomicAdd(&c->updated, updated);
  }
  if (tid == 0 || (ran_out && threadIdx.x == 0)) {
    atomicMax(&c->rounds, (unsigned long long)r);
    if (final_st) atomicOr(&c->status, final_st);
  }
}

__global__ void rounds_unpack_kernel(const long long* __restrict__ label, int V, int* dist,
                                     int* hops, int* pred) {
  for (long long v = (long long)blockIdx.x * blockDim.x + threadIdx.x; v < V;
       v += (long long)gridDim.x * blockDim.x) {
    const long long l = label[v];
    const int d = label_dist(l);
    dist[v] = d;
    if (hops) hops[v] = (d == kInf32) ? -1 : (int)label_hops(l);
    if (pred) pred[v] = -1;
  }
}

}  // namespace

RoundsState::~RoundsState() {
  if (tail) cudaFree(tail);
  if (chunk_rng) cudaFree(chunk_rng);
  if (bits) cudaFree(bits);
  if (ctl) cudaFree(ctl);
  if (host) cudaFreeHost(host);
  if (ev0) cudaEventDestroy(ev0);
  if (ev1) cudaEventDestroy(ev1);
}

long long rounds_device_bytes(int V, long long E) {
  const long long words = ((long long)V + 31) / 32;
  const long long n_chunks = (E + kChunk - 1) / kChunk;
  return 4 * E + 8 * n_chunks + 12 * words + (long long)sizeof(RoundsCtl);
}

int rounds_run(RoundsState& st, const int* row_ptr, const int2* adj, long long* label, int V,
               long long E, int src, int flags, int* dist, int* hops, int* pred,
               long long spin_limit, long long time_limit_ms, RoundsResult* res,
               cudaStream_t s) {
  const long long words = ((long long)V + 31) / 32;
  const long long n_chunks = (E + kChunk - 1) / kChunk;
  if (st.grid == 0) {   // first call: workspace and the per-edge tail array
    int dev = 0, sms = 0, per_sm = 0, coop = 0;
    BFQ_CUDA_TRY(cudaGetDevice(&dev));
    BFQ_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    BFQ_CUDA_TRY(cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev));
    if (!coop) {
      set_error("bfq_sssp_rounds: the device does not support cooperative launches");
      return BFQ_ERR_CUDA;
    }
    BFQ_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, rounds_kernel,
                                                               kRoundsBlock, 0));
    if (per_sm < 1) {
      set_error("bfq_sssp_rounds: the round kernel does not fit on an SM");
      return BFQ_ERR_CUDA;
    }
    if (!st.tail) BFQ_CUDA_TRY(cudaMalloc((void**)&st.tail, sizeof(int) * (size_t)(E > 0 ? E : 1)));
    if (!st.chunk_rng)
      BFQ_CUDA_TRY(cudaMalloc((void**)&st.chunk_rng,
                              sizeof(int2) * (size_t)(n_chunks > 0 ? n_chunks : 1)));
    if (!st.bits) BFQ_CUDA_TRY(cudaMalloc((void**)&st.bits, sizeof(unsigned) * (size_t)(3 * words)));
    if (!st.ctl) BFQ_CUDA_TRY(cudaMalloc(&st.ctl, sizeof(RoundsCtl)));
    if (!st.host) BFQ_CUDA_TRY(cudaMallocHost(&st.host, sizeof(RoundsCtl)));
    if (!st.ev0) BFQ_CUDA_TRY(cudaEventCreate(&st.ev0));
    if (!st.ev1) BFQ_CUDA_TRY(cudaEventCreate(&st.ev1));
    if (E > 0) {
      rounds_tail_kernel<<<1024, 256, 0, s>>>(row_ptr, V, st.tail);
      rounds_chunk_kernel<<<256, 256, 0, s>>>(st.tail, E, n_chunks, st.chunk_rng);
    }
    BFQ_CUDA_TRY(cudaGetLastError());
    st.grid = sms * per_sm;
  }
  RoundsCtl* ctl = (RoundsCtl*)st.ctl;
  rounds_init_kernel<<<1024, 256, 0, s>>>(label, st.bits, words, V, src, ctl);
  BFQ_CUDA_TRY(cudaGetLastError());
  RoundsArgs a{};
  a.adj = adj;
  a.tail = st.tail;
  a.chunk_rng = st.chunk_rng;
  a.label = label;
  a.bits = st.bits;
  a.ctl = ctl;
  a.E = E;
  a.words = words;
  a.n_chunks = n_chunks;
  a.max_rounds = V;
  a.spin_limit = spin_limit;
  a.time_limit_ns = time_limit_ms * 1000000LL;
  a.V = V;
  a.filter = (flags & BFQ_ROUNDS_ALL_EDGES) ? 0 : 1;
  void* params[] = {&a};
  BFQ_CUDA_TRY(cudaEventRecord(st.ev0, s));
  BFQ_CUDA_TRY(cudaLaunchCooperativeKernel((const void*)rounds_kernel, dim3(st.grid),
                                           dim3(kRoundsBlock), params, 0, s));
  BFQ_CUDA_TRY(cudaEventRecord(st.ev1, s));
  rounds_unpack_kernel<<<1024, 256, 0, s>>>(label, V, dist, hops, pred);
  BFQ_CUDA_TRY(cudaGetLastError());
  BFQ_CUDA_TRY(cudaMemcpyAsync(st.host, ctl, sizeof(RoundsCtl), cudaMemcpyDeviceToHost, s));
  BFQ_CUDA_TRY(cudaStreamSynchronize(s));
  const RoundsCtl* h = (const RoundsCtl*)st.host;
  int code = BFQ_OK;
  if (h->status & kStTimeout) code = BFQ_ERR_TIMEOUT;
  else if (h->status & kStNegCycle) code = BFQ_NEG_CYCLE;
  else if (h->status & kStRange) code = BFQ_RANGE;
  if (code == BFQ_OK && pred) {
    BFQ_CUDA_TRY(launch_pred_pass(row_ptr, adj, label, V, pred, s));
    BFQ_CUDA_TRY(cudaStreamSynchronize(s));
  }
  if (res) {
    res->rounds = (long long)h->rounds;
    res->relaxed = (long long)h->relaxed;
    res->updated = (long long)h->updated;
    float ms = 0.f;
    res->kernel_ms = (cudaEventElapsedTime(&ms, st.ev0, st.ev1) == cudaSuccess) ? ms : -1.f;
  }
  if (code == BFQ_ERR_TIMEOUT) set_error("bfq_sssp_rounds: a bounded device-side wait ran out");
  return code;
}

}  // namespace bfq
