// Host-side internals shared by the library's translation units.
#pragma once

#include <cstdint>
#include <string>

#include <cuda_runtime.h>

#include "../../include/bfq.h"
#include "bfq_device.cuh"

namespace bfq {

// Per-run control block in device memory; each hot field on its own line.
struct alignas(128) Control {
  int inflight;                 // items enqueued and not yet fully processed
  int pad0[31];
  int status;                   // kSt* bits of the current run
  int pad1[31];
  int stop;                     // set once a run must end early
  int pad2[31];
  unsigned long long ctr[8];    // summed warp counters, see CtrIndex
  unsigned long long pad3[8];
  int last_status;              // status code of the previous run (0 = clean)
  int pad4[31];
};

enum CtrIndex { kCtrDeq = 0, kCtrRel, kCtrUpd, kCtrEnq, kCtrSteal, kCtrChunk, kCtrIdle, kCtrSpare };

struct SsspArgs {
  const int* row_ptr;           // [V+1]
  const int2* adj;              // [E] (col, w)
  long long* label;             // [V] packed (dist, hops, in-queue flag)
  long long* cyc;               // [V] recorded relaxation edges (tail, w), or null
  QueueSet qs;                  // vertex sub-queues
  QueueSet cq;                  // hub edge-chunk sub-queues
  const int* hub_chunk0;        // [V] first chunk-table entry of a hub (read for hubs only)
  const int4* chunk_tab;        // {u, beg, end, 0} per hub chunk
  Control* ctl;
  int* dist;                    // [V] output
  int* hops;                    // [V] output or null
  int* pred;                    // [V] output or null (initialised to -1 here)
  int V;
  int src;
  int batch_items;
  int queues_per_cta;
  int share_div;                // a warp takes ceil(count / share_div) items (0: warps per queue)
  int chunk_batch;              // hub chunks a warp takes at once
  int hub_degree;
  int chunk_edges;
  long long spin_limit;
  long long time_limit_ns;
  int phantom;                  // test hook: unbacked in-flight items
  int mark_neg_inf;             // 1: resolve negative cycles to minus infinity
  unsigned cyc_walk0;           // first cycle-walk threshold (hops); records from half
  int relax_min;                // 0: CAS, 1: one atomicMin, 2: load then atomicMin
  int wide;                     // 1: the 80-register build (3 CTAs per SM), else 64
  int q_alloc;                  // sub-queues allocated (qs.Q of them serve this run;
  int cq_alloc;                 //   a reset clears all); 0: as many as qs.Q / cq.Q
};

struct LaunchShape {
  int grid;
  int block;
};

// Thread-local last-error message (bfq_last_error).
void set_error(const std::string& msg);
int cuda_fail(cudaError_t e, const char* what, const char* file, int line);

#define BFQ_CUDA_TRY(call)                                                     \
  do {                                                                         \
    cudaError_t e__ = (call);                                                  \
    if (e__ != cudaSuccess) return ::bfq::cuda_fail(e__, #call, __FILE__, __LINE__); \
  } while (0)

// Kernels launchers (sssp.cu)
int sssp_max_ctas_per_sm(int block, int wide);
// init, persistent run (bracketed by ev0/ev1 when given), epilogue, pred.
// l2win (nullable): L2 access-policy window attached to the persistent launch.
cudaError_t launch_sssp(const SsspArgs& a, LaunchShape init_shape, LaunchShape run_shape,
                        int32_t* status_dev, cudaEvent_t ev0, cudaEvent_t ev1,
                        cudaStream_t s, const cudaAccessPolicyWindow* l2win = nullptr);
cudaError_t launch_reached_edges(const int* row_ptr, const long long* label, int V,
                                 unsigned long long* out2, cudaStream_t s);
cudaError_t launch_pack_adj(const int* col, const int* w, int2* adj, long long E, cudaStream_t s);
cudaError_t launch_validate_csr(const int* row_ptr, const int* col, int V, long long E,
                                int* bad, cudaStream_t s);
cudaError_t launch_queue_reset(QueueSet qs, cudaStream_t s);
// The persistent relaxation kernel alone (no init, epilogue or pred pass).
cudaError_t launch_sssp_persistent_only(const SsspArgs& a, LaunchShape run_shape,
                                        cudaStream_t s);
// The epilogue alone: unpack labels to dist/hops (pred to -1) and write the
// status code; `bad` (nullable, device) forces BFQ_ERR_INVALID when non-zero.
cudaError_t launch_sssp_epilogue(const SsspArgs& a, LaunchShape shape, int32_t* status_dev,
                                 const int* bad, cudaStream_t s);

// Single-CTA query for small graphs (sssp_small.cu): dynamic shared memory
// of a run over V vertices with a ring of 2^cap_log2 slots, the most the
// device allows (sets the kernel attribute; 0 if unavailable), and the run
// (kernel bracketed by ev0/ev1 when given, then the epilogue).
size_t sssp_small_smem(int V, int cap_log2);
size_t sssp_small_smem_limit();
cudaError_t launch_sssp_small(const SsspArgs& a, int cap_log2, int32_t* status_dev,
                              cudaEvent_t ev0, cudaEvent_t ev1, cudaStream_t s);

// The run's predecessor pass (a.pred), after its epilogue: skipped, leaving
// -1, when the run did not end clean.
cudaError_t launch_sssp_pred(const SsspArgs& a, cudaStream_t s);

// Predecessor pass alone over final labels (pred must hold -1 beforehand).
cudaError_t launch_pred_pass(const int* row_ptr, const int2* adj, const long long* label, int V,
                             int* pred, cudaStream_t s);

// Round-based relaxation (rounds.cu).  Workspace made on first use.
struct RoundsState {
  int* tail = nullptr;          // [E] tail vertex of each edge
  int2* chunk_rng = nullptr;    // first and last tail of each edge chunk
  unsigned* bits = nullptr;     // three changed-vertex bitmaps
  void* ctl = nullptr;          // device counters
  void* host = nullptr;         // pinned copy of the counters
  cudaEvent_t ev0 = nullptr, ev1 = nullptr;
  int grid = 0;
  RoundsState() = default;
  RoundsState(const RoundsState&) = delete;
  RoundsState& operator=(const RoundsState&) = delete;
  ~RoundsState();
};
struct RoundsResult {
  long long rounds;
  long long relaxed;
  long long updated;
  float kernel_ms;
};
long long rounds_device_bytes(int V, long long E);
// Runs one query and synchronises `s`; returns a BFQ_* status code.
int rounds_run(RoundsState& st, const int* row_ptr, const int2* adj, long long* label, int V,
               long long E, int src, int flags, int* dist, int* hops, int* pred,
               long long spin_limit, long long time_limit_ms, RoundsResult* res,
               cudaStream_t s);

}  // namespace bfq
