/*
 * bfq.h -- C ABI of a single-GPU (GB300, sm_103a) queue-driven Bellman-Ford
 * SSSP library.
 *
 * The method is the one of "A Concurrent Queue System for Multi-GPU Platforms:
 * Application to Bellman-Ford SSSP": active vertices flow through a Broker
 * Queue (Sec. III-A, Algorithm 1) -- a ring buffer with head/tail ticket
 * counters, per-slot tickets and a broker count reserved before a ticket is
 * taken -- and each dequeued vertex relaxes its out-edges (Sec. III-C,
 * Algorithm 3).  The paper's per-GPU queue partitions (Sec. III-B,
 * Algorithm 2) become per-CTA sub-queues with work stealing on one GPU.
 *
 * Conventions for every entry point
 *   - Return value: >= 0 is a status (BFQ_OK, BFQ_NEG_CYCLE, ...), < 0 an
 *     error.  bfq_last_error() returns a message for the last error raised
 *     by the calling host thread.
 *   - "device pointer" arguments are caller-owned CUDA device memory (for
 *     instance torch tensors); the library never frees them.  "host pointer"
 *     arguments are ordinary host memory.
 *   - `stream` is a cudaStream_t passed as void*; NULL is the legacy default
 *     stream.  Work is enqueued on it; functions documented as synchronising
 *     wait for it.
 *   - A handle (graph, queue, batch, server) is not thread-safe: calls on one
 *     handle must be serialised by the caller, and GPU work issued through one
 *     handle on different streams must not overlap.
 *   - Graph data: CSR with int32 row_ptr[V+1], col[E], w[E]; 0 <= col < V;
 *     row_ptr non-decreasing from 0 to E.  Parallel edges and self-loops are
 *     allowed.
 *   - Distances are int32.  INT32_MAX (2147483647) means "no path".  A
 *     candidate distance >= INT32_MAX is discarded; a candidate <= INT32_MIN
 *     stops the run with status BFQ_RANGE.  hops[v] is the edge count of the
 *     least (dist, hops) label (the least-weight path with the fewest edges),
 *     -1 when unreachable.
 *   - Negative cycles (Algorithm 3 reports "detection of negative cycles"):
 *     status BFQ_NEG_CYCLE iff a negative-weight cycle is reachable from the
 *     source; dist/hops/pred contents are then unspecified.  Detection is
 *     exact: without such a cycle every accepted label is a simple path, so an
 *     accepted label with hops >= V proves one.  If V * max(0, -min weight)
 *     >= 2^31 and such a cycle exists, BFQ_RANGE may be returned instead.
 *   - Every device-side wait is bounded; a run that exceeds its bounds ends
 *     with BFQ_ERR_TIMEOUT and leaves the CUDA context usable.
 */
#ifndef BFQ_H
#define BFQ_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status and error codes ------------------------------------------- */
enum {
  BFQ_OK = 0,            /* finished, results valid                         */
  BFQ_NEG_CYCLE = 1,     /* a negative cycle is reachable from the source   */
  BFQ_FULL = 2,          /* queue: enqueue refused, ring holds N items      */
  BFQ_EMPTY = 3,         /* queue: dequeue refused, ring holds no item      */
  BFQ_RANGE = 4,         /* a distance fell below the int32 range           */
  BFQ_PENDING = 5,       /* server: request not finished yet                */
  BFQ_ERR_INVALID = -1,  /* bad argument or malformed graph                 */
  BFQ_ERR_OOM = -2,      /* device or host allocation failed                */
  BFQ_ERR_TIMEOUT = -3,  /* a bounded device-side wait ran out              */
  BFQ_ERR_CUDA = -4,     /* a CUDA call failed                              */
  BFQ_ERR_BUDGET = -5    /* server: request can never fit the memory budget */
};

/* Queue variants (Sec. III-A). */
enum {
  BFQ_QUEUE_BQ = 0,      /* Broker Queue, one operation per thread (Alg. 1)  */
  BFQ_QUEUE_BWD = 1,     /* Broker Work Distributor: ensure tried once        */
  BFQ_QUEUE_BQ_WARP = 2, /* Broker Queue, warp-aggregated: one exact-count
                            reservation (compare-and-swap) and one ticket
                            range per warp; the SSSP worklist's default form */
  BFQ_QUEUE_BWD_WARP = 3 /* Broker Work Distributor, warp-aggregated: one
                            single-shot fetch-add reservation (no retry) on
                            one of two counters, then one ticket range; the
                            SSSP worklist's BFQ_QUEUE_FORM_SINGLE_SHOT     */
};

typedef struct bfq_graph* bfq_graph_t;
typedef struct bfq_queue* bfq_queue_t;
typedef struct bfq_batch* bfq_batch_t;
typedef struct bfq_server* bfq_server_t;

/* Launch and queue parameters of the persistent SSSP kernel.  Zero in any
 * field selects the library default for it (bfq_tune_default). */
typedef struct bfq_tune {
  int32_t ctas_per_sm;      /* persistent CTAs per SM                        */
  int32_t threads_per_cta;  /* multiple of 32, <= 1024                       */
  int32_t queues_per_cta;   /* sub-queues per CTA (>= 1)                     */
  int32_t batch_items;      /* max vertices a warp dequeues at once (<= 32)  */
  int32_t hub_degree;       /* out-degree above which a vertex is split into
                               edge chunks shared by many warps             */
  int32_t chunk_edges;      /* edges per hub chunk (multiple of 32)          */
  int64_t spin_limit;       /* max polls of one ticket slot                  */
  int64_t time_limit_ms;    /* max wall time of one run on the device        */
  int32_t l2_persist_pct;   /* 0..100: share of the L2 set-aside asked for the
                               label array (access-policy window); 0 = off  */
  int32_t test_phantom_items; /* test hook, 0 in normal use: in-flight items
                               that no queued item backs, so a run can only
                               end through time_limit_ms (BFQ_ERR_TIMEOUT) */
  int32_t share_div;        /* a warp dequeues ceil(count / share_div) items
                               of a sub-queue holding count (<= batch_items);
                               0 = the number of warps serving it           */
  int32_t chunk_batch;      /* hub chunks a warp dequeues at once (1..32)    */
  int32_t neg_cycle_mode;   /* BFQ_NEG_CYCLE_STOP or BFQ_NEG_CYCLE_MARK, for
                               bfq_sssp / bfq_sssp_async (see there)         */
  int32_t cycle_walk_hops;  /* negative-cycle accelerator: a label of this
                               many hops makes its lane walk the recorded
                               relaxation edges behind it looking for a
                               negative cycle; a failed walk raises that
                               lane's threshold to twice the label's hops;
                               edges are recorded from half of it.  2..2^30,
                               0 = default (64).
                               Only speed depends on it: hops >= V stays the
                               exact test.                                   */
  int32_t relax_atomic;     /* how bfq_sssp lowers a label: BFQ_RELAX_AUTO,
                               BFQ_RELAX_MIN (one atomicMin per edge: fastest
                               while the label array sits in L2, but every
                               atomic dirties its line), BFQ_RELAX_FILTERED
                               (load, then atomicMin only when lower: fewer
                               atomics where most relaxations fail) or
                               BFQ_RELAX_CAS (load, then compare-and-swap
                               only when lower).  AUTO takes MIN when 8 V <=
                               half of L2, except FILTERED there for V >=
                               2^21 and E >= 8 V, and FILTERED when 8 V is
                               above half of L2.
                               Results are the same in every form.           */
  int32_t batch_budget_klabels; /* batched queries: labels (in units of 1024)
                               of the queries running at once.  Queries start
                               in order while the running ones fit, so their
                               labels stay in L2; one always runs.  The server
                               admits requests below its large-request size
                               by the same budget.  0 = half of L2 (8-byte
                               labels); -1 = no budget                      */
  int32_t kernel_ctas;      /* register form of bfq_sssp's persistent kernel:
                               4 = built for 4 CTAs per SM (64 registers per
                               thread), 3 = built for 3 (80 registers: fewer
                               spills, fewer warps; it runs on a smaller
                               grid, never above ctas_per_sm).  0 = auto: 3
                               when E < 8 V, else 4.  Results are the same
                               either way; bfq_autotune tries both.         */
  int32_t queue_form;       /* reservations on bfq_sssp's sub-queues:
                               BFQ_QUEUE_FORM_AUTO, BFQ_QUEUE_FORM_EXACT (the
                               Broker Queue's exact count, moved by
                               compare-and-swap) or BFQ_QUEUE_FORM_SINGLE_SHOT
                               (the Broker Work Distributor's ensure-once: one
                               fetch-add on one of two counters, no retry).
                               Results are the same either way.             */
  int32_t small_path;       /* BFQ_SMALL_PATH_AUTO, _ON or _OFF: run bfq_sssp /
                               bfq_sssp_async on one CTA whose shared memory
                               holds the labels, the recorded relaxation
                               edges and the vertex queue (the same queue-
                               driven algorithm at CTA scope; the CSR is read
                               from global memory).  Only when they fit
                               (16 B per vertex plus the queue ring: about
                               8,000 vertices on GB300) and neg_cycle_mode is
                               STOP; otherwise the persistent kernel runs.
                               AUTO takes it for graphs of at most 32,768
                               edges (that fit).
                               Results are the same either way.             */
  int32_t small_threads;    /* threads of that CTA: 1024 (0 = default) or 512
                               (fewer warps contending for the queue ring:
                               faster on deep, narrow searches such as grids,
                               slower on denser graphs); bfq_autotune tries
                               both.                                        */
} bfq_tune;

/* What a single query (bfq_sssp, bfq_sssp_async) does once it has proved a
 * reachable negative cycle.  STOP (the paper's behaviour, Sec. III-C: report
 * only) ends the run at once; dist/hops are then unspecified.  MARK keeps
 * relaxing and resolves the cycles: every vertex that a reachable negative
 * cycle reaches gets dist INT32_MIN ("minus infinity") and hops -2, every
 * other vertex its exact (dist, hops) label and, when asked, a predecessor
 * (pred -1 on minus-infinity vertices); the status is BFQ_NEG_CYCLE when any
 * vertex is minus infinity.  The result is unique when V * max|w| < 2^31;
 * beyond that a falling label may leave the int32 range before its cycle is
 * proved, and the run reports BFQ_RANGE instead.  The batched, serving,
 * round-based and allocation-free entry points always STOP. */
#define BFQ_NEG_CYCLE_STOP 0
#define BFQ_NEG_CYCLE_MARK 1

/* bfq_tune.queue_form (Sec. III-A: BQ retries its ensure step until the
 * count is final, BWD tries it once).  AUTO is EXACT. */
#define BFQ_QUEUE_FORM_AUTO 0
#define BFQ_QUEUE_FORM_EXACT 1
#define BFQ_QUEUE_FORM_SINGLE_SHOT 2

/* bfq_tune.small_path */
#define BFQ_SMALL_PATH_AUTO 0
#define BFQ_SMALL_PATH_ON 1
#define BFQ_SMALL_PATH_OFF 2

/* bfq_tune.relax_atomic */
#define BFQ_RELAX_AUTO 0
#define BFQ_RELAX_MIN 1
#define BFQ_RELAX_CAS 2
#define BFQ_RELAX_FILTERED 3

/* Counters of the last finished run on a graph handle (summed over warps). */
typedef struct bfq_stats {
  int64_t dequeued;       /* items taken from sub-queues (vertices + chunks)  */
  int64_t relaxed;        /* edges scanned                                   */
  int64_t updated;        /* successful label decreases                      */
  int64_t enqueued;       /* vertices enqueued (bitmap test-and-set won)     */
  int64_t steals;         /* dequeues from a sub-queue other than home       */
  int64_t hub_chunks;     /* hub edge chunks processed                       */
  int64_t m_reached;      /* edges whose tail is reachable (GTEPS numerator) */
  int64_t reached;        /* reachable vertices                              */
  int64_t V, E;
  int32_t grid, block, queues, queue_capacity;
  double kernel_ms;       /* duration of the persistent relaxation kernel,
                             from CUDA events recorded around its launch on
                             the caller's stream                            */
  int64_t idle_polls;     /* polls by warps that found no work               */
  int64_t reserved[4];
} bfq_stats;

/* ---- errors ------------------------------------------------------------ */
/* Message of the last error raised on this host thread ("" if none). */
const char* bfq_last_error(void);
/* Library ABI version (major*10000 + minor*100 + patch). */
int32_t bfq_version(void);

/* ---- tuning ------------------------------------------------------------- */
/* Fill *t with the defaults for the current device.  Returns BFQ_OK. */
int bfq_tune_default(bfq_tune* t);

/* ---- graphs (graph residency, Sec. III-C: graph data moved to GPU memory) */
/* Copy a CSR graph into library-owned device memory (interleaved
 * (col, w) pairs, 8 B per edge) and allocate its per-run workspace (labels,
 * in-queue bitmap, sub-queues).  row_ptr/col/w are host pointers when
 * on_device == 0, device pointers otherwise (read on `stream`).  The graph
 * is validated (monotone row_ptr, 0 <= col < V); BFQ_ERR_INVALID otherwise.
 * Synchronises `stream`.  tune may be NULL (defaults). */
int bfq_graph_create(bfq_graph_t* out, int32_t V, int64_t E,
                     const int32_t* row_ptr, const int32_t* col,
                     const int32_t* w, int on_device, const bfq_tune* tune,
                     void* stream);
int bfq_graph_destroy(bfq_graph_t g);
/* Device memory the handle holds, in bytes (graph + workspace). */
int64_t bfq_graph_device_bytes(bfq_graph_t g);

/* ---- single-source shortest paths (Algorithm 3 on one GPU) --------------- */
/* One query from `src`.  dist (int32[V], device) receives distances; hops
 * and pred (int32[V], device, each nullable) receive edge counts and a
 * predecessor tree (pred[src] = -1, -1 when unreachable; any tight
 * predecessor u with hops[u] + 1 == hops[v]).  Synchronises `stream` and
 * returns BFQ_OK, BFQ_NEG_CYCLE, BFQ_RANGE or an error. */
int bfq_sssp(bfq_graph_t g, int32_t src, int32_t* dist, int32_t* hops,
             int32_t* pred, void* stream);
/* Same, without synchronising: the status code (int32) is written to
 * status_dev (device pointer) when the run finishes on `stream`.  Returns
 * BFQ_OK once the work is enqueued, or an argument error. */
int bfq_sssp_async(bfq_graph_t g, int32_t src, int32_t* dist, int32_t* hops,
                   int32_t* pred, int32_t* status_dev, void* stream);
/* Counters of the last run on g (synchronises the device). */
int bfq_get_stats(bfq_graph_t g, bfq_stats* out);

/* One query that allocates nothing (the paper has no counterpart; this is a
 * library facility).  It is meant for callers that cannot allocate device
 * memory when they need a query: code running while a stream is captured
 * into a CUDA graph (an allocation there breaks the capture), programs that
 * fix their memory budget at start-up, or code living inside another
 * framework's memory arena.  All working memory (labels, in-queue bitmap,
 * sub-queues, control block) comes from one static 16 MiB array in device
 * memory that every GPU loading this library holds until the process exits.
 *   row_ptr: int32[V+1], adj: int32[2E] interleaved (col, w) pairs, 8-byte
 *   aligned; dist: int32[V]; hops: int32[V] or NULL; status_dev: one int32.
 *   All are caller-owned device pointers.
 * Limits: 1 <= V <= 524288 and 0 <= E < 2^31; larger graphs are rejected
 * with BFQ_ERR_INVALID and a message.  Hub splitting is off on this path.
 * Asynchronous on `stream`: returns BFQ_OK once enqueued; the run's status
 * (BFQ_OK, BFQ_NEG_CYCLE, BFQ_RANGE, BFQ_ERR_TIMEOUT, or BFQ_ERR_INVALID if
 * the CSR fails the device-side check) is written to *status_dev.
 * There is no pred output and no graph handle: the CSR is read in place, and
 * negative cycles are always reported by stopping (BFQ_NEG_CYCLE_STOP).
 * The first call on a device looks up the array's device address
 * (cudaGetSymbolAddress) and the device's L2 size with that device current,
 * and keeps both for the life of the process (a cudaDeviceReset is not
 * supported afterwards); make that first call before any stream capture.
 * Every call reuses the same array and clears the parts it needs, so calls
 * whose GPU work overlaps (on two streams, or from two threads) race and
 * must be serialised by the caller. */
int bfq_sssp_noalloc(const int32_t* row_ptr, const int32_t* adj, int32_t V,
                     int64_t E, int32_t src, int32_t* dist, int32_t* hops,
                     int32_t* status_dev, void* stream);
/* ---- round-based Bellman-Ford (Algorithm 3's formulation, Sec. III-C) ---
 * Algorithm 3 relaxes the edge list in synchronous rounds, counts the label
 * decreases of each round in a change counter, stops after a round with no
 * change, and reports a negative cycle when round V still changes a label.
 * bfq_sssp_rounds runs that formulation on one GPU, on the same graph handle
 * and with the same packed (dist, hops) labels as bfq_sssp, so dist, hops and
 * pred are identical to bfq_sssp's for every graph without a reachable
 * negative cycle.  A label of V or more hops also proves a negative cycle and
 * usually ends such runs long before round V.  By default a round relaxes
 * only the edges whose tail changed in the previous round (the fixed point
 * is the same); BFQ_ROUNDS_ALL_EDGES relaxes every edge every round, as the
 * algorithm prints it.  The first call on a handle adds 4 B per edge plus
 * 12 B per 32 vertices of workspace (counted by bfq_graph_device_bytes).
 * Runs as one cooperative launch; synchronises `stream`.
 *   dist: int32[V] device (required); hops, pred: int32[V] device or NULL;
 *   stats: host struct or NULL.
 * Returns BFQ_OK, BFQ_NEG_CYCLE, BFQ_RANGE, BFQ_ERR_TIMEOUT (a grid barrier
 * waited longer than spin_limit polls, or the run longer than time_limit_ms)
 * or an argument/CUDA error.  After BFQ_NEG_CYCLE, BFQ_RANGE or a timeout
 * dist/hops hold the labels reached and pred is all -1. */
#define BFQ_ROUNDS_ALL_EDGES 1

typedef struct bfq_rounds_stats {
  int64_t rounds;     /* rounds run, the last one included                  */
  int64_t relaxed;    /* edges relaxed over all rounds                      */
  int64_t updated;    /* label decreases: the sum of the change counters    */
  double kernel_ms;   /* device time of the round kernel (CUDA events)      */
  int64_t reserved[4];
} bfq_rounds_stats;

int bfq_sssp_rounds(bfq_graph_t g, int32_t src, int32_t flags, int32_t* dist,
                    int32_t* hops, int32_t* pred, bfq_rounds_stats* stats,
                    void* stream);

/* Run-time parameters of a graph handle.  set_tune validates like
 * bfq_graph_create (zero fields take the defaults) and rejects a change of
 * the parameters that size the workspace (threads_per_cta, ctas_per_sm,
 * queues_per_cta, hub_degree, chunk_edges) with BFQ_ERR_INVALID; the others
 * take effect at the next query.  A non-zero l2_persist_pct sets aside that
 * share of the device's maximum persisting L2 for the calling context
 * (cudaLimitPersistingL2CacheSize) and attaches an access-policy window over
 * the label array to the persistent launch.  Setting it back to 0, or
 * destroying the handle, drops the persisting lines and restores the
 * context's previous persisting-L2 limit (the set-aside takes L2 capacity
 * from every other kernel of the process while it is held).  With a non-zero
 * share, bfq_sssp (the synchronous call) turns the persisting lines back into
 * normal ones once its query is over (cudaCtxResetPersistingL2Cache, which
 * acts on the whole context); bfq_sssp_async leaves them, so that queries in
 * a row on one handle keep their labels in L2. */
int bfq_graph_get_tune(bfq_graph_t g, bfq_tune* out);
int bfq_graph_set_tune(bfq_graph_t g, const bfq_tune* t);


/* Pick the run-time parameters (share_div, chunk_batch, batch_items, then
 * kernel_ctas, queue_form, relax_atomic, l2_persist_pct and small_path) that
 * make the queries from srcs[0..n) (host array) fastest on g, keep them on
 * the handle and copy them to *out (nullable).  Times a fixed grid of
 * candidates in the handle's register form over one pass of the sources
 * each, the best four again over four passes, then, one at a time at the
 * best so far, the other register form, the other queue form, the other
 * relaxation forms, an L2 set-aside of 50 and 75 percent for the labels with
 * each relaxation form, and, where the graph fits, the other of the
 * single-CTA and persistent paths (CUDA events, each pass after an untimed
 * one); allocates one int32[V] scratch array for the duration.
 * Synchronises `stream`. */
int bfq_autotune(bfq_graph_t g, const int32_t* srcs, int32_t n, bfq_tune* out, void* stream);

/* ---- batched queries: many sources over many resident graphs in one
 * persistent launch, replayed from a captured CUDA graph ------------------ */
/* graphs: host array of ngraphs handles (they must outlive the batch).
 * max_queries <= 4096 queries per call; max_total_vertices bounds the sum of
 * V over one call's queries (<= 0: max V x max_queries) and sizes the label
 * pool and sub-queues.  tune may be NULL. */
int bfq_batch_create(bfq_batch_t* out, const bfq_graph_t* graphs, int32_t ngraphs,
                     int32_t max_queries, int64_t max_total_vertices,
                     const bfq_tune* tune);
int bfq_batch_destroy(bfq_batch_t b);
int64_t bfq_batch_device_bytes(bfq_batch_t b);
/* Run nq queries (graph_id[q], src[q]: host arrays) in one launch.  dist and
 * hops are host arrays of nq device pointers (int32[V_q] each; hops may be
 * NULL or hold NULLs).  status (host, int32[nq]) receives each query's
 * status (BFQ_OK, BFQ_NEG_CYCLE, BFQ_RANGE, BFQ_ERR_TIMEOUT).  A query with a
 * negative cycle stops alone; the others finish.  Synchronises `stream`;
 * returns BFQ_OK, BFQ_ERR_TIMEOUT if the launch ran out of time, or an
 * argument error (nq > max_queries, vertices beyond max_total_vertices). */
int bfq_sssp_batch(bfq_batch_t b, int32_t nq, const int32_t* graph_id,
                   const int32_t* src, int32_t* const* dist, int32_t* const* hops,
                   int32_t* status, void* stream);
/* Counters of the last batch launch (kernel_ms = whole captured run). */
int bfq_batch_get_stats(bfq_batch_t b, bfq_stats* out);
/* Set the run-time parameters (share_div, chunk_batch, batch_items,
 * time_limit_ms; zero fields are left unchanged). */
int bfq_batch_set_tune(bfq_batch_t b, const bfq_tune* t);
/* Autotuner: runs the given query set under a grid of run-time parameters,
 * keeps the fastest on the handle and copies it to *out (nullable). */
int bfq_batch_autotune(bfq_batch_t b, int32_t nq, const int32_t* graph_id,
                       const int32_t* src, int32_t* const* dist,
                       int32_t* const* hops, bfq_tune* out, void* stream);

/* ---- serving: continuous batching on a resident kernel ------------------- */
/* A server keeps the graphs (host array of handles that must outlive it)
 * resident and runs requests on one resident persistent kernel.  Requests
 * are admitted in arrival order when one of max_slots (<= 2048) query slots
 * is free and the label pool -- hbm_budget_bytes / 32 labels, each label
 * taking 8 B, 8 B of recorded relaxation edge and 16 B of sub-queue
 * capacity -- has a contiguous run for the
 * graph's V labels; admitted requests join the queries already running on the
 * device.  One exception to arrival order: a request whose labels exceed a
 * quarter of the device's L2 (V >= L2 bytes / 32; such a query keeps the GPU
 * busy alone, and two of them evict each other's labels) runs only while no
 * other such request runs, and smaller requests behind it may be admitted
 * while it waits.  Such a large request (also any request over half of the
 * label budget below) runs alone through the single-query kernel on its
 * graph's handle: the resident kernel stops between batches, the query
 * runs, and the resident kernel resumes with its queued work.  It runs with
 * the handle's own run-time parameters (bfq_graph_set_tune).  So while a
 * server runs, no other query may use a served graph's handle.  The other
 * requests are admitted while their labels fit tune->batch_budget_klabels
 * (default: half of L2), so the labels being relaxed stay in L2; one always
 * runs.  A host thread drives admission and completion.  tune may be NULL. */
int bfq_server_create(bfq_server_t* out, const bfq_graph_t* graphs, int32_t ngraphs,
                      int64_t hbm_budget_bytes, int32_t max_slots, const bfq_tune* tune);
/* Queue a request (thread-safe).  dist / hops: caller-owned device arrays of
 * the graph's V int32 (either may be NULL).  The server writes them from its
 * own stream, unordered with the caller's streams: they must hold no pending
 * work of the caller at submission and stay valid until the request
 * completes.  *req_id receives the request's id.  BFQ_ERR_BUDGET if the
 * graph can never fit the budget. */
int bfq_server_submit(bfq_server_t sv, int32_t graph_id, int32_t src, int32_t* dist,
                      int32_t* hops, int64_t* req_id);
/* BFQ_PENDING while the request runs or waits, else BFQ_OK with *status the
 * request's status and the host steady-clock times (ns) of submission and of
 * completion as seen by the server thread. */
int bfq_server_poll(bfq_server_t sv, int64_t req_id, int32_t* status,
                    int64_t* t_submit_ns, int64_t* t_done_ns);
/* Wait up to timeout_ms for a request; BFQ_PENDING if it is still running. */
int bfq_server_wait(bfq_server_t sv, int64_t req_id, int64_t timeout_ms, int32_t* status);
/* Requests completed, kernel launches so far, most requests admitted at once. */
int bfq_server_stats(bfq_server_t sv, int64_t* completed, int64_t* launches,
                     int64_t* peak_active);
/* Monitoring snapshot, out[0..min(n,10)): requests waiting, requests
 * admitted, free slots, largest free label run, kernel launches, requests
 * completed, kernel running (0/1), CUDA error that stopped the server (0 =
 * none), first failed device range check (0 = none) and its value. */
int bfq_server_state(bfq_server_t sv, int64_t* out, int32_t n);
/* Finish admitted requests, stop the kernel and free everything. */
int bfq_server_destroy(bfq_server_t sv);

/* ---- standalone Broker Queue (Sec. III-A, Algorithm 1; Sec. IV workloads) */
/* A ring of `capacity` int32 items (rounded up to a power of two for the
 * warp variant), variant = BFQ_QUEUE_*. */
int bfq_queue_create(bfq_queue_t* q, int64_t capacity, int32_t variant);
int bfq_queue_destroy(bfq_queue_t q);
/* Reset head, tail, count and tickets to zero (INITIALIZE). */
int bfq_queue_reset(bfq_queue_t q, void* stream);
/* n ENQUEUE operations of items[i] (device), op i by thread i of a
 * grid-stride loop over grid x block threads.  pos_out (int64[n], device,
 * nullable) receives the ring position (tail ticket) of each successful op
 * or -1 for BFQ_FULL.  Asynchronous. */
int bfq_queue_enqueue(bfq_queue_t q, const int32_t* items, int64_t n,
                      int64_t* pos_out, int32_t grid, int32_t block,
                      void* stream);
/* n DEQUEUE operations; out[i] (device) receives the item of op i, pos_out
 * (nullable) its head ticket or -1 for BFQ_EMPTY.  Asynchronous. */
int bfq_queue_dequeue(bfq_queue_t q, int32_t* out, int64_t n,
                      int64_t* pos_out, int32_t grid, int32_t block,
                      void* stream);
/* The paper's "Global Mixed" workload: in one launch, even blocks perform
 * n_enq ENQUEUEs of items[] and odd blocks n_deq DEQUEUEs into out[];
 * enq_pos/deq_pos as above (nullable).  grid >= 2.  Asynchronous. */
int bfq_queue_mixed(bfq_queue_t q, const int32_t* items, int64_t n_enq,
                    int64_t* enq_pos, int32_t* out, int64_t n_deq,
                    int64_t* deq_pos, int32_t grid, int32_t block,
                    void* stream);
/* L2 atomic throughput on this device (the measured denominator of the
 * queue benchmark; the paper has no counterpart): n_ops atomics by grid x
 * block threads.  mode 0: each thread adds to its own 8-byte counter
 * (distinct addresses); 1: every thread adds to one counter and uses the
 * returned value (a ticket); 2: one lane per warp moves one counter by 32
 * with a compare-and-swap loop (n_ops a multiple of 32, counted as 32 per
 * success).  *ms_out (nullable) receives the CUDA-event time of the launch
 * and *total_out (nullable) the sum of the counters (== n_ops).  Allocates
 * and frees its counters; synchronises `stream`. */
int bfq_atomic_bench(int32_t mode, int64_t n_ops, int32_t grid, int32_t block,
                     double* ms_out, int64_t* total_out, void* stream);

/* The relaxation step's memory pattern alone, as the measured bound of the
 * SSSP kernels' relax phase (the paper has no counterpart): n_edges (col, w)
 * pairs, generated on the device, are read lane-contiguously (8 B per edge,
 * two per lane in flight) and each relaxes a random one of n_labels labels
 * (starting at infinity) with a key of 256 possible distances, with no queue
 * work.  mode 0: one 64-bit atomicMin per edge; 1: a load of the label, then
 * the atomicMin only when the key is below it (the BFQ_RELAX_FILTERED form).
 * grid x block threads; *ms_out (nullable) receives the CUDA-event time of
 * the relax launch (generation untimed) and *lowered_out (nullable) the
 * number of edges that lowered a label.  Allocates 8 B per edge and per
 * label for the call; synchronises `stream`.  BFQ_ERR_INVALID for a mode
 * other than 0 or 1, n_edges or n_labels < 1, or a bad launch shape. */
int bfq_relax_bench(int32_t mode, int64_t n_edges, int32_t n_labels, int32_t grid,
                    int32_t block, double* ms_out, int64_t* lowered_out, void* stream);

/* Read head, tail and count (host pointers, each nullable) and the queue's
 * error word; synchronises `stream`.  Returns BFQ_OK or BFQ_ERR_TIMEOUT if a
 * ticket wait of an earlier launch ran out. */
int bfq_queue_state(bfq_queue_t q, int64_t* head, int64_t* tail,
                    int64_t* count, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* BFQ_H */
