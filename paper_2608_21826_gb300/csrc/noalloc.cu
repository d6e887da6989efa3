// bfq_sssp_noalloc: a single-source query that allocates no memory.
//
// Some callers cannot allocate device memory at the point where they need a
// query: code running while a CUDA stream is being captured into a graph
// (an allocation there breaks or invalidates the capture), programs that fix
// their whole memory budget at start-up (real-time services, plug-in hosts
// that forbid allocation after initialisation), or code running inside
// another framework's memory arena.  For them this entry point takes every
// byte of working memory from one fixed array in device global memory
// instead of from cudaMalloc.
//
// The array is file-scope and static, so every GPU that loads the library
// holds it (kNoAllocScratchBytes) until the process exits.  The caller still
// provides the graph and the outputs.  Limits: V <= kNoAllocMaxV, and the
// hub-splitting path is off (it needs per-graph tables).
#include <cstdint>
#include <mutex>

#include "bfq_internal.h"

namespace bfq {
namespace {

constexpr size_t kNoAllocScratchBytes = 16u << 20;      // 16 MiB per device
constexpr int kNoAllocMaxV = 1 << 19;                    // 524,288 vertices
constexpr int kNoAllocQueues = 256;
constexpr int kNoAllocMaxDevices = 64;

// The scratch array.  Host code must not use its name as an address (that is
// a host-side stand-in); the device address comes from cudaGetSymbolAddress.
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

std::mutex g_setup_mu;
void* g_scratch_dev[kNoAllocMaxDevices] = {};
long long g_l2_bytes[kNoAllocMaxDevices] = {};

// Byte offsets of the per-call working set inside the scratch array.
struct Layout {
  size_t ctl, bad, qmeta, qslots, cmeta, cslots, label, total;
  int cap_log2;
};

size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

Layout layout_for(int V) {
  Layout L{};
  long long per_q = (2LL * V + kNoAllocQueues - 1) / kNoAllocQueues;
  int l = 10;
  while ((1LL << l) < per_q) ++l;
  L.cap_log2 = l;
  size_t o = 0;
  L.ctl = o;    o = align_up(o + sizeof(Control), 256);
  L.bad = o;    o = align_up(o + sizeof(int), 256);
  L.qmeta = o;  o = align_up(o + sizeof(QueueMeta) * kNoAllocQueues, 256);
  L.qslots = o; o = align_up(o + sizeof(unsigned long long) * ((size_t)kNoAllocQueues << l), 256);
  L.cmeta = o;  o = align_up(o + sizeof(QueueMeta), 256);
  L.cslots = o; o = align_up(o + sizeof(unsigned long long) * 256, 256);
  L.label = o;  o = align_up(o + sizeof(long long) * (size_t)V, 256);
  L.total = o;
  return L;
}

// Zero the queues and control block of this call's working set (the
// array keeps whatever the previous call left), and check the CSR.
__global__ void noalloc_prepare_kernel(unsigned char* base, Layout L, const int* row_ptr,
                                       const int* adj, int V, long long E) {
  const long long tid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const long long nth = (long long)gridDim.x * blockDim.x;
  unsigned long long* z = (unsigned long long*)(base + L.ctl);
  const long long nz = (long long)(L.label - L.ctl) / 8;   // everything before the labels
  for (long long i = tid; i < nz; i += nth) {
    if ((size_t)(i * 8) >= L.bad && (size_t)(i * 8) < L.bad + 256) continue;   // the flag
    z[i] = 0ull;
  }
  int* bad = (int*)(base + L.bad);
  if (tid == 0 && (row_ptr[0] != 0 || (long long)row_ptr[V] != E)) atomicOr(bad, 1);
  for (long long v = tid; v < V; v += nth)
    if (row_ptr[v + 1] < row_ptr[v]) atomicOr(bad, 2);
  for (long long i = tid; i < E; i += nth) {
    const int c = adj[2 * i];
    if (c < 0 || c >= V) atomicOr(bad, 4);
  }
}

// Labels to (INF, -), the source to (0, 0) and queued, unless the CSR was
// rejected: then nothing is queued and the persistent kernel exits at once.
__global__ void noalloc_init_kernel(SsspArgs a, const int* bad) {
  const bool ok = *bad == 0;
  const long long tid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const long long nth = (long long)gridDim.x * blockDim.x;
  for (long long v = tid; v < a.V; v += nth)
    a.label[v] = (ok && v == a.src) ? (pack_label(0, 0) | kQueuedBit) : kInfLabel;
  if (tid == 0) {
    if (ok) {
      a.qs.slots[0] = (1ull << 32) | (unsigned)a.src;   // lap 0, full, at ticket 0
      a.qs.meta[0].tail = 1;
      a.qs.meta[0].count = 1;
    }
    a.ctl->inflight = ok ? 1 : 0;
    a.ctl->status = 0;
    a.ctl->stop = 0;
  }
}

// Device address of the scratch array on the current device and the
// device's L2 size, looked up once per device (with that device current).
int scratch_for_current_device(unsigned char** out, int* dev_out, long long* l2_out) {
  int dev = 0;
  BFQ_CUDA_TRY(cudaGetDevice(&dev));
  if (dev < 0 || dev >= kNoAllocMaxDevices) {
    set_error("bfq_sssp_noalloc: device index beyond the supported range");
    return BFQ_ERR_INVALID;
  }
  std::lock_guard<std::mutex> lk(g_setup_mu);
  if (!g_scratch_dev[dev]) {
    void* p = nullptr;
    BFQ_CUDA_TRY(cudaGetSymbolAddress(&p, g_noalloc_scratch));
    int l2 = 0;
    BFQ_CUDA_TRY(cudaDeviceGetAttribute(&l2, cudaDevAttrL2CacheSize, dev));
    g_l2_bytes[dev] = l2;
    g_scratch_dev[dev] = p;
  }
  *out = (unsigned char*)g_scratch_dev[dev];
  *dev_out = dev;
  *l2_out = g_l2_bytes[dev];
  return BFQ_OK;
}

}  // namespace
}  // namespace bfq

using namespace bfq;

extern "C" int bfq_sssp_noalloc(const int32_t* row_ptr, const int32_t* adj, int32_t V,
                                int64_t E, int32_t src, int32_t* dist, int32_t* hops,
                                int32_t* status_dev, void* stream) {
  if (!row_ptr || (E > 0 && !adj) || !dist || !status_dev) {
    set_error("bfq_sssp_noalloc: null pointer argument");
    return BFQ_ERR_INVALID;
  }
  if (((uintptr_t)adj & 7u) != 0) {
    set_error("bfq_sssp_noalloc: adj must be 8-byte aligned ((col, w) int32 pairs)");
    return BFQ_ERR_INVALID;
  }
  if (V < 1 || V > kNoAllocMaxV) {
    set_error("bfq_sssp_noalloc: V must be in [1, 524288] (the fixed 16 MiB scratch array)");
    return BFQ_ERR_INVALID;
  }
  if (E < 0 || E >= (1LL << 31)) {
    set_error("bfq_sssp_noalloc: E must be in [0, 2^31)");
    return BFQ_ERR_INVALID;
  }
  if (src < 0 || src >= V) {
    set_error("bfq_sssp_noalloc: source out of range");
    return BFQ_ERR_INVALID;
  }
  const Layout L = layout_for(V);
  if (L.total > kNoAllocScratchBytes) {
    set_error("bfq_sssp_noalloc: working set exceeds the 16 MiB scratch array");
    return BFQ_ERR_INVALID;
  }
  unsigned char* base = nullptr;
  int dev = 0;
  long long l2_bytes = 0;
  int rc = scratch_for_current_device(&base, &dev, &l2_bytes);
  if (rc != BFQ_OK) return rc;
  int sms = 0;
  BFQ_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  const LaunchShape run{sms * sssp_max_ctas_per_sm(256, 0), 256};
  const LaunchShape init{sms * 4, 256};
  cudaStream_t s = (cudaStream_t)stream;

  SsspArgs a{};
  a.row_ptr = row_ptr;
  a.adj = (const int2*)adj;
  a.label = (long long*)(base + L.label);
  a.cyc = nullptr;                 // cycle accelerator off: hops >= V decides alone
  a.qs = QueueSet{(QueueMeta*)(base + L.qmeta), (unsigned long long*)(base + L.qslots),
                  kNoAllocQueues, L.cap_log2};
  a.cq = QueueSet{(QueueMeta*)(base + L.cmeta), (unsigned long long*)(base + L.cslots), 1, 8};
  a.hub_chunk0 = nullptr;          // never read: no vertex exceeds hub_degree
  a.chunk_tab = nullptr;
  a.ctl = (Control*)(base + L.ctl);
  a.dist = dist;
  a.hops = hops;
  a.pred = nullptr;
  a.V = V;
  a.src = src;
  a.batch_items = 32;
  a.queues_per_cta = 1;
  a.share_div = 2;
  a.chunk_batch = 4;
  a.hub_degree = 0x7fffffff;
  a.chunk_edges = 256;
  a.spin_limit = 1LL << 22;
  a.time_limit_ns = 20000LL * 1000000LL;
  a.phantom = 0;
  // one atomicMin per relaxation while the labels fit in half of L2 (the
  // rule of the regular entry point; always so at the vertex limit on GB300)
  a.relax_min = (long long)sizeof(long long) * V <= l2_bytes / 2 ? 1 : 0;
  int* bad = (int*)(base + L.bad);

  BFQ_CUDA_TRY(cudaMemsetAsync(bad, 0, sizeof(int), s));
  noalloc_prepare_kernel<<<init.grid, init.block, 0, s>>>(base, L, row_ptr, adj, V, E);
  noalloc_init_kernel<<<init.grid, init.block, 0, s>>>(a, bad);
  BFQ_CUDA_TRY(cudaGetLastError());
  BFQ_CUDA_TRY(launch_sssp_persistent_only(a, run, s));
  BFQ_CUDA_TRY(launch_sssp_epilogue(a, init, status_dev, bad, s));
  return BFQ_OK;
}
