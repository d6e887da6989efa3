// C ABI: graph residency, single-query SSSP, statistics and errors.
#include <algorithm>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "bfq_internal.h"
#include "sssp_small.h"

namespace bfq {

namespace {
thread_local std::string g_last_error;
}

void set_error(const std::string& msg) { g_last_error = msg; }

int cuda_fail(cudaError_t e, const char* what, const char* file, int line) {
  char buf[512];
  std::snprintf(buf, sizeof(buf), "%s failed: %s (%s:%d)", what, cudaGetErrorString(e), file,
                line);
  set_error(buf);
  return e == cudaErrorMemoryAllocation ? BFQ_ERR_OOM : BFQ_ERR_CUDA;
}

static int invalid(const std::string& msg) {
  set_error(msg);
  return BFQ_ERR_INVALID;
}

static int ceil_log2(long long x) {
  int l = 0;
  while ((1LL << l) < x) ++l;
  return l;
}

}  // namespace bfq

using namespace bfq;

struct bfq_graph {
  int device = 0;
  int V = 0;
  long long E = 0;
  bfq_tune tune{};
  int* row_ptr = nullptr;
  int2* adj = nullptr;
  long long* label = nullptr;
  long long* cyc = nullptr;
  QueueSet qs{};
  QueueSet cq{};
  int* hub_chunk0 = nullptr;
  int4* chunk_tab = nullptr;
  int n_chunks = 0;
  Control* ctl = nullptr;
  int32_t* status_dev = nullptr;
  unsigned long long* scratch = nullptr;   // [2] reached-edge reduction
  int32_t* status_host = nullptr;          // pinned
  LaunchShape init_shape{};
  LaunchShape run_shape{};                     // the workspace's shape (narrow form)
  int sms = 0;
  int per_sm_wide = 0;                         // CTAs per SM of the wide form
  size_t small_smem_limit = 0;                 // dynamic shared memory of the small path
  LaunchShape last_shape{};                    // the last run's shape and
  int last_queues = 0;                         //   vertex sub-queues (stats)
  long long bytes = 0;
  cudaStream_t last_stream = nullptr;
  cudaEvent_t ev0 = nullptr, ev1 = nullptr;   // around the persistent kernel
  long long l2_bytes = 0;                      // device L2 size
  int l2_pct_applied = 0;                      // l2_persist_pct the window was made for
  size_t l2_limit_saved = 0;                   // persisting-L2 limit before the first window
  cudaAccessPolicyWindow l2win{};
  RoundsState rounds;                          // round-based path, made on first use
  std::vector<void*> allocs;

  int alloc(void** p, size_t n) {
    if (n == 0) n = 16;
    cudaError_t e = cudaMalloc(p, n);
    if (e != cudaSuccess) return cuda_fail(e, "cudaMalloc", __FILE__, __LINE__);
    allocs.push_back(*p);
    bytes += (long long)n;
    return BFQ_OK;
  }
  // Drop this handle's persisting lines and give the context its previous
  // persisting-L2 limit back.
  void release_l2() {
    if (l2_pct_applied == 0) return;
    cudaCtxResetPersistingL2Cache();
    cudaDeviceSetLimit(cudaLimitPersistingL2CacheSize, l2_limit_saved);
    l2_pct_applied = 0;
  }
  ~bfq_graph() {
    release_l2();
    for (void* p : allocs) cudaFree(p);
    if (status_host) cudaFreeHost(status_host);
    if (ev0) cudaEventDestroy(ev0);
    if (ev1) cudaEventDestroy(ev1);
  }
};

namespace bfq {
struct GraphView {
  const int* row_ptr;
  const int2* adj;
  const int* hub_chunk0;
  const int4* chunk_tab;
  int V, n_chunks, hub_degree, chunk_edges;
};
int graph_view(bfq_graph_t g, GraphView* out) {
  if (!g || !out) return BFQ_ERR_INVALID;
  out->row_ptr = g->row_ptr;
  out->adj = g->adj;
  out->hub_chunk0 = g->hub_chunk0;
  out->chunk_tab = g->chunk_tab;
  out->V = g->V;
  out->n_chunks = g->n_chunks;
  out->hub_degree = g->tune.hub_degree;
  out->chunk_edges = g->tune.chunk_edges;
  return BFQ_OK;
}
}  // namespace bfq

extern "C" {

const char* bfq_last_error(void) { return g_last_error.c_str(); }

int32_t bfq_version(void) { return 10000; }

int bfq_tune_default(bfq_tune* t) {
  if (!t) return invalid("bfq_tune_default: null pointer");
  std::memset(t, 0, sizeof(*t));
  t->threads_per_cta = 256;
  t->ctas_per_sm = 0;          // 0: as many as fit (occupancy)
  t->queues_per_cta = 1;
  t->batch_items = 32;
  t->hub_degree = 512;
  t->chunk_edges = 256;
  t->spin_limit = 1LL << 22;
  t->time_limit_ms = 20000;
  t->l2_persist_pct = 0;
  t->share_div = 2;
  t->chunk_batch = 4;
  t->cycle_walk_hops = 64;
  return BFQ_OK;
}

static int fill_tune(const bfq_tune* in, bfq_tune* out) {
  bfq_tune_default(out);
  if (!in) return BFQ_OK;
  if (in->threads_per_cta) out->threads_per_cta = in->threads_per_cta;
  if (in->ctas_per_sm) out->ctas_per_sm = in->ctas_per_sm;
  if (in->queues_per_cta) out->queues_per_cta = in->queues_per_cta;
  if (in->batch_items) out->batch_items = in->batch_items;
  if (in->hub_degree) out->hub_degree = in->hub_degree;
  if (in->chunk_edges) out->chunk_edges = in->chunk_edges;
  if (in->spin_limit) out->spin_limit = in->spin_limit;
  if (in->time_limit_ms) out->time_limit_ms = in->time_limit_ms;
  if (in->l2_persist_pct) out->l2_persist_pct = in->l2_persist_pct;
  out->test_phantom_items = in->test_phantom_items;
  if (in->share_div) out->share_div = in->share_div;
  if (in->chunk_batch) out->chunk_batch = in->chunk_batch;
  out->neg_cycle_mode = in->neg_cycle_mode;
  if (in->cycle_walk_hops) out->cycle_walk_hops = in->cycle_walk_hops;
  out->relax_atomic = in->relax_atomic;
  out->kernel_ctas = in->kernel_ctas;
  out->queue_form = in->queue_form;
  out->small_path = in->small_path;
  out->small_threads = in->small_threads;
  if (out->threads_per_cta != 256)
    return invalid("bfq_tune: threads_per_cta must be 256 (the shared-memory layout of the kernels)");
  if (out->queues_per_cta < 1 || out->queues_per_cta > 8)
    return invalid("bfq_tune: queues_per_cta must be in [1, 8]");
  if (out->batch_items < 1 || out->batch_items > 32)
    return invalid("bfq_tune: batch_items must be in [1, 32]");
  if (out->chunk_edges < 32 || out->chunk_edges % 32)
    return invalid("bfq_tune: chunk_edges must be a positive multiple of 32");
  if (out->hub_degree < out->chunk_edges)
    return invalid("bfq_tune: hub_degree must be >= chunk_edges");
  if (out->spin_limit < 1 || out->time_limit_ms < 1 || out->ctas_per_sm < 0 ||
      out->l2_persist_pct < 0 || out->l2_persist_pct > 100 || out->test_phantom_items < 0 ||
      out->share_div < 0 || out->chunk_batch < 1 || out->chunk_batch > 32 ||
      (out->neg_cycle_mode != BFQ_NEG_CYCLE_STOP && out->neg_cycle_mode != BFQ_NEG_CYCLE_MARK) ||
      out->cycle_walk_hops < 2 || out->cycle_walk_hops > (1 << 30) ||
      out->relax_atomic < BFQ_RELAX_AUTO || out->relax_atomic > BFQ_RELAX_FILTERED ||
      (out->kernel_ctas != 0 && out->kernel_ctas != 3 && out->kernel_ctas != 4) ||
      out->queue_form < BFQ_QUEUE_FORM_AUTO || out->queue_form > BFQ_QUEUE_FORM_SINGLE_SHOT ||
      out->small_path < BFQ_SMALL_PATH_AUTO || out->small_path > BFQ_SMALL_PATH_OFF ||
      (out->small_threads != 0 && out->small_threads != 512 && out->small_threads != 1024))
    return invalid("bfq_tune: bad limits");
  return BFQ_OK;
}

int bfq_graph_create(bfq_graph_t* out, int32_t V, int64_t E, const int32_t* row_ptr,
                     const int32_t* col, const int32_t* w, int on_device, const bfq_tune* tune,
                     void* stream) {
  if (!out) return invalid("bfq_graph_create: out is null");
  *out = nullptr;
  if (V < 1) return invalid("bfq_graph_create: V must be >= 1");
  if (E < 0 || E >= (1LL << 31)) return invalid("bfq_graph_create: E must be in [0, 2^31)");
  if (!row_ptr || (E > 0 && (!col || !w))) return invalid("bfq_graph_create: null CSR array");
  cudaStream_t s = (cudaStream_t)stream;
  bfq_graph* g = new (std::nothrow) bfq_graph();
  if (!g) return invalid("bfq_graph_create: host allocation failed");
  int rc = fill_tune(tune, &g->tune);
  if (rc) { delete g; return rc; }
  g->V = V;
  g->E = E;
  cudaGetDevice(&g->device);

  // host copy of row_ptr (validation on the host when the CSR is host-side,
  // hub chunk table in both cases)
  std::vector<int> rp(V + 1);
#define G_TRY(x)                                        \
  do {                                                  \
    int rc__ = (x);                                     \
    if (rc__ != BFQ_OK) { delete g; return rc__; }      \
  } while (0)
#define G_CUDA(x)                                                              \
  do {                                                                         \
    cudaError_t e__ = (x);                                                     \
    if (e__ != cudaSuccess) { int rc__ = cuda_fail(e__, #x, __FILE__, __LINE__); delete g; return rc__; } \
  } while (0)
  if (on_device) {
    G_CUDA(cudaMemcpyAsync(rp.data(), row_ptr, sizeof(int) * (V + 1), cudaMemcpyDeviceToHost, s));
    G_CUDA(cudaStreamSynchronize(s));
  } else {
    std::memcpy(rp.data(), row_ptr, sizeof(int) * (V + 1));
  }
  if (rp[0] != 0 || (long long)rp[V] != E) { delete g; return invalid("bfq_graph_create: row_ptr[0] must be 0 and row_ptr[V] == E"); }
  for (int v = 0; v < V; ++v)
    if (rp[v + 1] < rp[v]) { delete g; return invalid("bfq_graph_create: row_ptr not monotone"); }
  if (!on_device) {
    for (long long i = 0; i < E; ++i)
      if (col[i] < 0 || col[i] >= V) { delete g; return invalid("bfq_graph_create: col out of range"); }
  }

  // graph arrays
  G_TRY(g->alloc((void**)&g->row_ptr, sizeof(int) * (V + 1)));
  G_TRY(g->alloc((void**)&g->adj, sizeof(int2) * (size_t)E));
  G_CUDA(cudaMemcpyAsync(g->row_ptr, rp.data(), sizeof(int) * (V + 1), cudaMemcpyHostToDevice, s));
  if (E > 0) {
    if (on_device) {
      int* bad = nullptr;
      G_CUDA(cudaMalloc((void**)&bad, sizeof(int)));
      cudaError_t e1 = cudaMemsetAsync(bad, 0, sizeof(int), s);
      if (e1 == cudaSuccess) e1 = launch_validate_csr(g->row_ptr, col, V, E, bad, s);
      if (e1 == cudaSuccess) e1 = launch_pack_adj(col, w, g->adj, E, s);
      int hbad = 0;
      if (e1 == cudaSuccess) e1 = cudaMemcpyAsync(&hbad, bad, sizeof(int), cudaMemcpyDeviceToHost, s);
      if (e1 == cudaSuccess) e1 = cudaStreamSynchronize(s);
      cudaFree(bad);
      G_CUDA(e1);
      if (hbad) { delete g; return invalid("bfq_graph_create: col out of range"); }
    } else {
      std::vector<int2> packed((size_t)E);
      for (long long i = 0; i < E; ++i) packed[i] = make_int2(col[i], w[i]);
      G_CUDA(cudaMemcpyAsync(g->adj, packed.data(), sizeof(int2) * (size_t)E,
                             cudaMemcpyHostToDevice, s));
      G_CUDA(cudaStreamSynchronize(s));
    }
  }

  // hub chunk table: vertices of degree > hub_degree, chunk_edges per chunk
  const int hub = g->tune.hub_degree, ce = g->tune.chunk_edges;
  std::vector<int> chunk0(V, -1);
  std::vector<int4> tab;
  for (int v = 0; v < V; ++v) {
    const int d = rp[v + 1] - rp[v];
    if (d > hub) {
      chunk0[v] = (int)tab.size();
      for (int b = rp[v]; b < rp[v + 1]; b += ce)
        tab.push_back(make_int4(v, b, std::min(b + ce, rp[v + 1]), 0));
    }
  }
  g->n_chunks = (int)tab.size();
  G_TRY(g->alloc((void**)&g->hub_chunk0, sizeof(int) * V));
  G_TRY(g->alloc((void**)&g->chunk_tab, sizeof(int4) * std::max<size_t>(1, tab.size())));
  G_CUDA(cudaMemcpyAsync(g->hub_chunk0, chunk0.data(), sizeof(int) * V, cudaMemcpyHostToDevice, s));
  if (!tab.empty())
    G_CUDA(cudaMemcpyAsync(g->chunk_tab, tab.data(), sizeof(int4) * tab.size(),
                           cudaMemcpyHostToDevice, s));

  // launch shape
  int sms = 0;
  G_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, g->device));
  int l2 = 0;
  G_CUDA(cudaDeviceGetAttribute(&l2, cudaDevAttrL2CacheSize, g->device));
  g->l2_bytes = l2;
  const int block = g->tune.threads_per_cta;
  int per_sm = sssp_max_ctas_per_sm(block, 0);
  if (g->tune.ctas_per_sm > 0) per_sm = std::min(per_sm, g->tune.ctas_per_sm);
  g->run_shape = {sms * per_sm, block};
  g->sms = sms;
  // the wide form fits fewer CTAs: it runs on a prefix of the sub-queues
  g->per_sm_wide = std::min(per_sm, sssp_max_ctas_per_sm(block, 1));
  g->init_shape = {sms * 4, 256};
  g->small_smem_limit = sssp_small_smem_limit();

  // workspace: labels (with in-queue flags), vertex and chunk sub-queues
  const int Q = g->run_shape.grid * g->tune.queues_per_cta;
  const long long per_q = (2LL * V + Q - 1) / Q;
  int cap_log2 = std::max(10, ceil_log2(per_q));
  g->qs.Q = Q;
  g->qs.cap_log2 = cap_log2;
  const int Qc = g->n_chunks > 0 ? g->run_shape.grid : 1;
  const long long per_qc = (4LL * g->n_chunks + Qc - 1) / Qc;
  g->cq.Q = Qc;
  g->cq.cap_log2 = std::max(8, ceil_log2(std::max(1LL, per_qc)));
  G_TRY(g->alloc((void**)&g->label, sizeof(long long) * (size_t)V));
  G_TRY(g->alloc((void**)&g->cyc, sizeof(long long) * (size_t)V));
  G_TRY(g->alloc((void**)&g->qs.meta, sizeof(QueueMeta) * Q));
  G_TRY(g->alloc((void**)&g->qs.slots, sizeof(unsigned long long) * ((size_t)Q << cap_log2)));
  G_TRY(g->alloc((void**)&g->cq.meta, sizeof(QueueMeta) * Qc));
  G_TRY(g->alloc((void**)&g->cq.slots,
                 sizeof(unsigned long long) * ((size_t)Qc << g->cq.cap_log2)));
  G_TRY(g->alloc((void**)&g->ctl, sizeof(Control)));
  G_TRY(g->alloc((void**)&g->status_dev, sizeof(int32_t)));
  G_TRY(g->alloc((void**)&g->scratch, 2 * sizeof(unsigned long long)));
  G_CUDA(cudaMemsetAsync(g->cyc, 0xff, sizeof(long long) * (size_t)V, s));   // tail -1: none
  G_CUDA(cudaMemsetAsync(g->qs.meta, 0, sizeof(QueueMeta) * Q, s));
  G_CUDA(cudaMemsetAsync(g->qs.slots, 0, sizeof(unsigned long long) * ((size_t)Q << cap_log2), s));
  G_CUDA(cudaMemsetAsync(g->cq.meta, 0, sizeof(QueueMeta) * Qc, s));
  G_CUDA(cudaMemsetAsync(g->cq.slots, 0,
                         sizeof(unsigned long long) * ((size_t)Qc << g->cq.cap_log2), s));
  G_CUDA(cudaMemsetAsync(g->ctl, 0, sizeof(Control), s));
  G_CUDA(cudaMallocHost((void**)&g->status_host, sizeof(int32_t)));
  G_CUDA(cudaEventCreate(&g->ev0));
  G_CUDA(cudaEventCreate(&g->ev1));
  G_CUDA(cudaStreamSynchronize(s));
#undef G_TRY
#undef G_CUDA
  *out = g;
  return BFQ_OK;
}

int bfq_graph_destroy(bfq_graph_t g) {
  if (!g) return invalid("bfq_graph_destroy: null handle");
  cudaDeviceSynchronize();
  delete g;
  return BFQ_OK;
}

int64_t bfq_graph_device_bytes(bfq_graph_t g) { return g ? g->bytes : 0; }

// Register form of the persistent kernel: 80 registers (3 CTAs per SM) by
// default below an average out-degree of 8, where queue operations take a
// larger share of each warp step.
static int wide_form(bfq_graph_t g, const bfq_tune& t) {
  return t.kernel_ctas == 3 ? 1 : t.kernel_ctas == 4 ? 0 : g->E < 8LL * g->V ? 1 : 0;
}

// Relaxation form of the persistent kernel (SsspArgs::relax_min: 0 CAS,
// 1 atomicMin, 2 filtered atomicMin).  AUTO: atomicMin while the label array
// fits in half of L2; filtered instead on large graphs (2^21 vertices or
// more) of average out-degree 8 or more, where most relaxations fail and L2
// atomic throughput, not the extra round trip of a lowering relaxation,
// sets the pace (measured on R-MAT: atomicMin 20% faster at 2^18 vertices,
// even at 2^20, filtered 7% faster at 2^21 and 2^22); filtered once the
// labels outgrow half of L2, where every atomicMin would dirty a line that
// L2 cannot keep (measured against load + compare-and-swap: 6-9% faster on
// R-MAT 23, level on a 4096^2 road-like grid).
static const int32_t kRelaxTuneOf[3] = {BFQ_RELAX_CAS, BFQ_RELAX_MIN, BFQ_RELAX_FILTERED};
static int relax_form(bfq_graph_t g, int32_t relax_atomic) {
  switch (relax_atomic) {
    case BFQ_RELAX_CAS: return 0;
    case BFQ_RELAX_MIN: return 1;
    case BFQ_RELAX_FILTERED: return 2;
    default: break;
  }
  if ((long long)sizeof(long long) * g->V > g->l2_bytes / 2) return 2;
  return (g->V >= (1 << 21) && g->E >= 8LL * g->V) ? 2 : 1;
}

static SsspArgs make_args(bfq_graph_t g, int32_t src, int32_t* dist, int32_t* hops,
                          int32_t* pred) {
  SsspArgs a{};
  a.row_ptr = g->row_ptr;
  a.adj = g->adj;
  a.label = g->label;
  a.cyc = g->cyc;
  a.qs = g->qs;
  a.cq = g->cq;
  a.hub_chunk0 = g->hub_chunk0;
  a.chunk_tab = g->chunk_tab;
  a.ctl = g->ctl;
  a.dist = dist;
  a.hops = hops;
  a.pred = pred;
  a.V = g->V;
  a.src = src;
  a.batch_items = g->tune.batch_items;
  a.queues_per_cta = g->tune.queues_per_cta;
  a.share_div = g->tune.share_div;
  a.chunk_batch = g->tune.chunk_batch;
  a.hub_degree = g->tune.hub_degree;
  a.chunk_edges = g->tune.chunk_edges;
  a.spin_limit = g->tune.spin_limit;
  a.time_limit_ns = g->tune.time_limit_ms * 1000000LL;
  a.phantom = g->tune.test_phantom_items;
  a.mark_neg_inf = g->tune.neg_cycle_mode == BFQ_NEG_CYCLE_MARK ? 1 : 0;
  a.cyc_walk0 = (unsigned)g->tune.cycle_walk_hops;
  a.relax_min = relax_form(g, g->tune.relax_atomic);
  a.wide = wide_form(g, g->tune);
  a.q_alloc = g->qs.Q;
  a.cq_alloc = g->cq.Q;
  a.qs.split = a.cq.split = g->tune.queue_form == BFQ_QUEUE_FORM_SINGLE_SHOT ? 1 : 0;
  if (a.wide) {
    // a smaller grid on a prefix of the sub-queues (the init kernel resets
    // all of them after any run that did not end cleanly)
    a.qs.Q = g->sms * g->per_sm_wide * g->tune.queues_per_cta;
    if (g->n_chunks > 0) a.cq.Q = g->sms * g->per_sm_wide;
  }
  return a;
}

static LaunchShape shape_for(bfq_graph_t g, const SsspArgs& a) {
  return a.wide ? LaunchShape{g->sms * g->per_sm_wide, g->run_shape.block} : g->run_shape;
}

// L2 persistence for the label array (Sec. IV's L2 set-aside sweep): set
// aside l2_persist_pct percent of the device's maximum persisting L2 for this
// context and describe a window over the labels, attached to the persistent
// launch.  The set-aside is a limit of the calling process's context; the
// previous limit comes back when the share returns to 0 or the handle goes.
static int apply_l2_window(bfq_graph_t g) {
  const int pct = g->tune.l2_persist_pct;
  if (g->l2_pct_applied == pct) return BFQ_OK;
  int max_persist = 0, max_window = 0;
  BFQ_CUDA_TRY(cudaDeviceGetAttribute(&max_persist, cudaDevAttrMaxPersistingL2CacheSize,
                                      g->device));
  BFQ_CUDA_TRY(cudaDeviceGetAttribute(&max_window, cudaDevAttrMaxAccessPolicyWindowSize,
                                      g->device));
  if (max_persist <= 0 || max_window <= 0)
    return invalid("bfq_sssp: the device offers no persisting L2 (l2_persist_pct must be 0)");
  if (g->l2_pct_applied == 0)
    BFQ_CUDA_TRY(cudaDeviceGetLimit(&g->l2_limit_saved, cudaLimitPersistingL2CacheSize));
  const size_t setaside = (size_t)max_persist * (size_t)pct / 100;
  BFQ_CUDA_TRY(cudaDeviceSetLimit(cudaLimitPersistingL2CacheSize, setaside));
  const size_t bytes = std::min(sizeof(long long) * (size_t)g->V, (size_t)max_window);
  g->l2win = cudaAccessPolicyWindow{};
  g->l2win.base_ptr = g->label;
  g->l2win.num_bytes = bytes;
  g->l2win.hitRatio = std::min(1.0f, (float)setaside / (float)bytes);
  g->l2win.hitProp = cudaAccessPropertyPersisting;
  g->l2win.missProp = cudaAccessPropertyStreaming;
  g->l2_pct_applied = pct;
  return BFQ_OK;
}

// Ring of the small path: a power of two >= V (at most V vertices are queued
// at once), at least one warp's worth.
static int small_cap_log2(int V) { return std::max(5, ceil_log2(V)); }

// Whether a query runs on the single-CTA path: asked for or AUTO, it fits
// in shared memory, and cycles stop the run.  AUTO: up to 32K edges, where
// one SM keeps up with the work and the search's depth, not its width, sets
// the time (measured against the persistent kernel: the 64x64 grid 0.46
// against 0.82 ms, a 64x64 road-like grid 0.15 against 0.22 ms, and 9 of
// the batched mix's 10 graphs up to 32K edges 30-50% faster, the tenth 7%
// slower; above that the single SM falls behind, e.g. 8K vertices and
// 40K-80K edges 15-50% slower).
static bool small_path_fits(bfq_graph_t g, const bfq_tune& t) {
  return t.neg_cycle_mode != BFQ_NEG_CYCLE_MARK &&
         sssp_small_smem(g->V, small_cap_log2(g->V)) <= g->small_smem_limit;
}
static bool use_small_path(bfq_graph_t g, const bfq_tune& t) {
  if (t.small_path == BFQ_SMALL_PATH_OFF || !small_path_fits(g, t)) return false;
  if (t.small_path == BFQ_SMALL_PATH_ON) return true;
  return g->E <= 32768;
}

int bfq_sssp_async(bfq_graph_t g, int32_t src, int32_t* dist, int32_t* hops, int32_t* pred,
                   int32_t* status_dev, void* stream) {
  if (!g) return invalid("bfq_sssp: null graph handle");
  if (src < 0 || src >= g->V) return invalid("bfq_sssp: source out of range");
  if (!dist) return invalid("bfq_sssp: dist is null");
  cudaStream_t s = (cudaStream_t)stream;
  g->last_stream = s;
  if (use_small_path(g, g->tune)) {
    SsspArgs a = make_args(g, src, dist, hops, pred);
    const int threads = g->tune.small_threads == 512 ? 512 : 1024;
    g->last_shape = LaunchShape{1, threads};
    g->last_queues = 1;
    BFQ_CUDA_TRY(launch_sssp_small_threads(a, small_cap_log2(g->V), threads, status_dev, g->ev0,
                                           g->ev1, s));
    if (pred) BFQ_CUDA_TRY(launch_sssp_pred(a, s));
    return BFQ_OK;
  }
  const cudaAccessPolicyWindow* win = nullptr;
  if (g->tune.l2_persist_pct > 0) {
    const int rc = apply_l2_window(g);
    if (rc != BFQ_OK) return rc;
    win = &g->l2win;
  } else {
    g->release_l2();
  }
  SsspArgs a = make_args(g, src, dist, hops, pred);
  g->last_shape = shape_for(g, a);
  g->last_queues = a.qs.Q;
  BFQ_CUDA_TRY(launch_sssp(a, g->init_shape, g->last_shape, status_dev, g->ev0, g->ev1, s, win));
  return BFQ_OK;
}

int bfq_sssp(bfq_graph_t g, int32_t src, int32_t* dist, int32_t* hops, int32_t* pred,
             void* stream) {
  int rc = bfq_sssp_async(g, src, dist, hops, pred, g ? g->status_dev : nullptr, stream);
  if (rc != BFQ_OK) return rc;
  cudaStream_t s = (cudaStream_t)stream;
  BFQ_CUDA_TRY(cudaMemcpyAsync(g->status_host, g->status_dev, sizeof(int32_t),
                               cudaMemcpyDeviceToHost, s));
  BFQ_CUDA_TRY(cudaStreamSynchronize(s));
  // the query is over: turn its persisting lines back into normal ones, so
  // that the set-aside holds no stale labels for other work
  if (g->l2_pct_applied > 0) cudaCtxResetPersistingL2Cache();
  const int st = *g->status_host;
  if (st == BFQ_ERR_TIMEOUT) set_error("bfq_sssp: a bounded device-side wait ran out");
  return st;
}

int bfq_sssp_rounds(bfq_graph_t g, int32_t src, int32_t flags, int32_t* dist, int32_t* hops,
                    int32_t* pred, bfq_rounds_stats* stats, void* stream) {
  if (!g) return invalid("bfq_sssp_rounds: null graph handle");
  if (src < 0 || src >= g->V) return invalid("bfq_sssp_rounds: source out of range");
  if (!dist) return invalid("bfq_sssp_rounds: dist is null");
  if (flags & ~BFQ_ROUNDS_ALL_EDGES) return invalid("bfq_sssp_rounds: unknown flag");
  cudaStream_t s = (cudaStream_t)stream;
  const bool fresh = g->rounds.grid == 0;
  RoundsResult r{};
  const int rc = rounds_run(g->rounds, g->row_ptr, g->adj, g->label, g->V, g->E, src, flags, dist,
                            hops, pred, g->tune.spin_limit, g->tune.time_limit_ms, &r, s);
  if (fresh && g->rounds.grid != 0) g->bytes += rounds_device_bytes(g->V, g->E);
  if (rc < 0 && rc != BFQ_ERR_TIMEOUT) return rc;
  if (stats) {
    std::memset(stats, 0, sizeof(*stats));
    stats->rounds = r.rounds;
    stats->relaxed = r.relaxed;
    stats->updated = r.updated;
    stats->kernel_ms = r.kernel_ms;
  }
  return rc;
}

int bfq_graph_get_tune(bfq_graph_t g, bfq_tune* out) {
  if (!g || !out) return invalid("bfq_graph_get_tune: null argument");
  *out = g->tune;
  return BFQ_OK;
}

int bfq_graph_set_tune(bfq_graph_t g, const bfq_tune* t) {
  if (!g || !t) return invalid("bfq_graph_set_tune: null argument");
  bfq_tune n{};
  const int rc = fill_tune(t, &n);
  if (rc != BFQ_OK) return rc;
  const bfq_tune& o = g->tune;
  if (n.threads_per_cta != o.threads_per_cta || n.queues_per_cta != o.queues_per_cta ||
      n.hub_degree != o.hub_degree || n.chunk_edges != o.chunk_edges ||
      (t->ctas_per_sm != 0 && t->ctas_per_sm != o.ctas_per_sm))
    return invalid("bfq_graph_set_tune: threads_per_cta, ctas_per_sm, queues_per_cta, "
                   "hub_degree and chunk_edges are fixed when the graph is created");
  n.ctas_per_sm = o.ctas_per_sm;
  g->tune = n;
  if (n.l2_persist_pct == 0) g->release_l2();
  return BFQ_OK;
}

int bfq_get_stats(bfq_graph_t g, bfq_stats* out) {
  if (!g || !out) return invalid("bfq_get_stats: null argument");
  std::memset(out, 0, sizeof(*out));
  cudaStream_t s = g->last_stream;
  BFQ_CUDA_TRY(cudaStreamSynchronize(s));
  Control c;
  BFQ_CUDA_TRY(cudaMemcpy(&c, g->ctl, sizeof(Control), cudaMemcpyDeviceToHost));
  BFQ_CUDA_TRY(launch_reached_edges(g->row_ptr, g->label, g->V, g->scratch, s));
  unsigned long long red[2] = {0, 0};
  BFQ_CUDA_TRY(cudaMemcpyAsync(red, g->scratch, sizeof(red), cudaMemcpyDeviceToHost, s));
  BFQ_CUDA_TRY(cudaStreamSynchronize(s));
  out->dequeued = (int64_t)c.ctr[kCtrDeq];
  out->relaxed = (int64_t)c.ctr[kCtrRel];
  out->updated = (int64_t)c.ctr[kCtrUpd];
  out->enqueued = (int64_t)c.ctr[kCtrEnq];
  out->steals = (int64_t)c.ctr[kCtrSteal];
  out->hub_chunks = (int64_t)c.ctr[kCtrChunk];
  out->idle_polls = (int64_t)c.ctr[kCtrIdle];
  out->m_reached = (int64_t)red[0];
  out->reached = (int64_t)red[1];
  out->V = g->V;
  out->E = g->E;
  const LaunchShape sh = g->last_shape.grid ? g->last_shape : g->run_shape;
  out->grid = sh.grid;
  out->block = sh.block;
  out->queues = g->last_queues ? g->last_queues : g->qs.Q;
  out->queue_capacity = 1 << g->qs.cap_log2;
  float ms = 0.f;
  if (cudaEventElapsedTime(&ms, g->ev0, g->ev1) == cudaSuccess) out->kernel_ms = ms;
  cudaGetLastError();   // no run yet: events never recorded
  return BFQ_OK;
}

int bfq_autotune(bfq_graph_t g, const int32_t* srcs, int32_t n, bfq_tune* out, void* stream) {
  if (!g || !srcs || n < 1) return invalid("bfq_autotune: null argument or no sources");
  for (int i = 0; i < n; ++i)
    if (srcs[i] < 0 || srcs[i] >= g->V) return invalid("bfq_autotune: source out of range");
  static const int kShare[] = {1, 2, 4, 8};
  static const int kChunk[] = {2, 4, 8};
  static const int kItems[] = {16, 32};
  cudaStream_t s = (cudaStream_t)stream;
  int* dist = nullptr;
  BFQ_CUDA_TRY(cudaMalloc((void**)&dist, sizeof(int) * (size_t)g->V));
  const bfq_tune keep = g->tune;
  bfq_tune best_t = keep;
  int rc = BFQ_OK;
  // device time of `passes` timed passes over the sources on g->tune, after
  // one untimed pass
  auto time_it = [&](int passes) {
    float total = 0.f;
    for (int rep = 0; rep <= passes && rc == BFQ_OK; ++rep) {
      for (int i = 0; i < n && rc == BFQ_OK; ++i) {
        int st = bfq_sssp(g, srcs[i], dist, nullptr, nullptr, stream);
        if (st < 0) rc = st;
        float ms = 0.f;
        if (rep > 0 && cudaEventElapsedTime(&ms, g->ev0, g->ev1) == cudaSuccess) total += ms;
      }
    }
    return total;
  };
  // every candidate once; the asynchronous order makes single passes vary
  // by a few percent, so the best few are timed again over more passes
  std::vector<std::pair<float, bfq_tune>> cand;
  for (int si : kShare)
    for (int ci : kChunk)
      for (int ii : kItems) {
        if (rc != BFQ_OK) break;
        g->tune.share_div = si;
        g->tune.chunk_batch = ci;
        g->tune.batch_items = ii;
        const float t = time_it(1);
        cand.emplace_back(t, g->tune);
      }
  if (rc == BFQ_OK) {
    std::stable_sort(cand.begin(), cand.end(),
                     [](const std::pair<float, bfq_tune>& x,
                        const std::pair<float, bfq_tune>& y) { return x.first < y.first; });
    constexpr int kFinalists = 4, kPasses = 4;
    float best = -1.f;
    for (int k = 0; k < kFinalists && k < (int)cand.size() && rc == BFQ_OK; ++k) {
      g->tune = cand[k].second;
      const float t = time_it(kPasses);
      if (rc == BFQ_OK && (best < 0.f || t < best)) {
        best = t;
        best_t = g->tune;
      }
    }
    // then, one at a time at the best parameters so far: the other register
    // form, the other queue reservation form, and an L2 set-aside for the
    // labels (Sec. IV's L2 sweep) of half and three quarters
    auto try_one = [&](bfq_tune cand) {
      if (rc != BFQ_OK) return;
      g->tune = cand;
      const float t = time_it(kPasses);
      if (rc == BFQ_OK && t < best) {
        best = t;
        best_t = cand;
      }
    };
    {
      bfq_tune c = best_t;
      c.kernel_ctas = wide_form(g, best_t) ? 4 : 3;
      try_one(c);
    }
    {
      bfq_tune c = best_t;
      c.queue_form = best_t.queue_form == BFQ_QUEUE_FORM_SINGLE_SHOT ? BFQ_QUEUE_FORM_EXACT
                                                                     : BFQ_QUEUE_FORM_SINGLE_SHOT;
      try_one(c);
    }
    {
      // the other relaxation forms (atomicMin pays while the labels stay in
      // L2, the filtered form where most relaxations fail; near the rules'
      // edges any may win)
      const bfq_tune base = best_t;
      const int now = relax_form(g, base.relax_atomic);
      for (int f = 0; f < 3; ++f)
        if (f != now) {
          bfq_tune c = base;
          c.relax_atomic = kRelaxTuneOf[f];
          try_one(c);
        }
    }
    int max_persist = 0;
    cudaDeviceGetAttribute(&max_persist, cudaDevAttrMaxPersistingL2CacheSize, g->device);
    cudaGetLastError();
    if (max_persist > 0) {
      // with every relaxation form: a set-aside that keeps the labels from
      // being evicted by the adjacency stream can make atomicMin pay where
      // it lost without one (labels near half of L2)
      const bfq_tune base = best_t;
      for (int pct : {50, 75})
        for (int f = 0; f < 3; ++f) {
          bfq_tune c = base;
          c.l2_persist_pct = pct;
          c.relax_atomic = kRelaxTuneOf[f];
          try_one(c);
        }
    }
    if (small_path_fits(g, best_t)) {
      // the other path: one CTA with the search state in shared memory, or
      // the persistent kernel; then the single CTA's other size
      {
        bfq_tune c = best_t;
        c.small_path = use_small_path(g, best_t) ? BFQ_SMALL_PATH_OFF : BFQ_SMALL_PATH_ON;
        try_one(c);
      }
      if (use_small_path(g, best_t)) {
        bfq_tune c = best_t;
        c.small_threads = best_t.small_threads == 512 ? 1024 : 512;
        try_one(c);
      }
    }
  }
  cudaStreamSynchronize(s);
  cudaFree(dist);
  g->tune = (rc == BFQ_OK) ? best_t : keep;
  if (g->tune.l2_persist_pct == 0) g->release_l2();
  if (out && rc == BFQ_OK) *out = best_t;
  return rc;
}

}  // extern "C"
