/*
 * Oracle for queue-driven Bellman-Ford SSSP -- TEST INFRASTRUCTURE ONLY.
 *
 * Plain, slow, sequential C that states what the GPU path must compute.  It
 * shares no code, header, table or constant with the CUDA library: only the
 * tests, the smoke check and the CPU-baseline leg of the benchmark may load it.
 *
 * Problem (paper Sec. II-D and Sec. III-C, Algorithm 3 inputs/outputs): for a
 * directed graph with int32 edge weights, which may be negative, and a source s,
 * compute d[v] = the least weight of an s->v path, and report whether a cycle of
 * negative weight can be reached from s.
 *
 * Representation (readings of points the paper leaves open):
 *   - Graph in CSR form: row_ptr[V+1], col[E], w[E] (int32).
 *   - A label is the pair (dist, hops) ordered lexicographically; hops is the
 *     number of edges of the path that produced dist.  For each vertex the
 *     lexicographic minimum is unique when no negative cycle is reachable: the
 *     least weight and, among least-weight paths, the fewest edges.
 *   - Unreachable: dist = INT32_MAX, hops = -1.
 *   - Candidates are formed in int64.  A candidate >= INT32_MAX is discarded
 *     (cannot be stored; "infinity").  A candidate <= INT32_MIN cannot be
 *     stored either and stops the run with status RANGE.
 *   - Negative cycle: without a reachable negative cycle every accepted label
 *     is a simple path (a walk around a cycle of weight >= 0 is never
 *     lexicographically smaller than the label it started from), so hops stays
 *     <= V-1.  Accepting a label with hops >= V therefore proves a reachable
 *     negative cycle, and with one the labels never settle, so such a label is
 *     eventually accepted.  This replaces the per-round change count of
 *     Algorithm 3 and does not depend on the order of relaxations.
 *
 * Status codes (own copy, by value): 0 OK, 1 NEG_CYCLE, 4 RANGE.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_OK 0
#define ORC_NEG_CYCLE 1
#define ORC_RANGE 4
#define ORC_ERR_INVALID (-1)
#define ORC_ERR_OOM (-2)

#define ORC_INF32 ((int64_t)2147483647)
#define ORC_MIN32 ((int64_t)(-2147483647 - 1))

/* lexicographic (d1,h1) < (d2,h2) */
static int lex_less(int64_t d1, int64_t h1, int64_t d2, int64_t h2) {
  return d1 < d2 || (d1 == d2 && h1 < h2);
}

static int check_csr(int32_t V, const int32_t* row_ptr, const int32_t* col,
                     int32_t src) {
  if (V < 1 || src < 0 || src >= V || row_ptr[0] != 0) return 0;
  for (int32_t v = 0; v < V; ++v)
    if (row_ptr[v + 1] < row_ptr[v]) return 0;
  for (int64_t e = 0; e < row_ptr[V]; ++e)
    if (col[e] < 0 || col[e] >= V) return 0;
  return 1;
}

/*
 * FIFO label-correcting Bellman-Ford (Bellman-Ford-Moore, the FIFO-queue form
 * of Bellman-Ford named in Sec. II-D): a vertex whose label drops is appended
 * to a FIFO queue unless it is already in it; a dequeued vertex relaxes all its
 * out-edges (the relaxation test of PARALLEL_RELAX_EDGES in Algorithm 3, applied
 * to the lexicographic label).
 *
 * Outputs dist[V], hops[V]; *n_relax (nullable) receives the number of edges
 * scanned.  Returns a status or a negative error.
 */
int oracle_spfa(int32_t V, const int32_t* row_ptr, const int32_t* col,
                const int32_t* w, int32_t src, int32_t* dist, int32_t* hops,
                int64_t* n_relax) {
  if (!check_csr(V, row_ptr, col, src)) return ORC_ERR_INVALID;
  int64_t* d = (int64_t*)malloc(sizeof(int64_t) * (size_t)V);
  int64_t* h = (int64_t*)malloc(sizeof(int64_t) * (size_t)V);
  int32_t* fifo = (int32_t*)malloc(sizeof(int32_t) * (size_t)V); /* circular */
  char* inq = (char*)calloc((size_t)V, 1);
  if (!d || !h || !fifo || !inq) {
    free(d); free(h); free(fifo); free(inq);
    return ORC_ERR_OOM;
  }
  for (int32_t v = 0; v < V; ++v) { d[v] = ORC_INF32; h[v] = -1; }
  d[src] = 0;
  h[src] = 0;
  /* at most V vertices are queued at once (the in-queue flag) */
  int64_t qhead = 0, qlen = 0;
  fifo[0] = src;
  qlen = 1;
  inq[src] = 1;
  int status = ORC_OK;
  int64_t scanned = 0;
  while (qlen > 0 && status == ORC_OK) {
    int32_t u = fifo[qhead];
    qhead = (qhead + 1) % V;
    --qlen;
    inq[u] = 0;
    int64_t du = d[u], hu = h[u];
    for (int32_t e = row_ptr[u]; e < row_ptr[u + 1]; ++e) {
      ++scanned;
      int32_t v = col[e];
      int64_t nd = du + (int64_t)w[e];
      int64_t nh = hu + 1;
      if (nd >= ORC_INF32) continue;           /* not storable: infinity */
      if (!lex_less(nd, nh, d[v], h[v])) continue;
      if (nd <= ORC_MIN32) { status = ORC_RANGE; break; }
      d[v] = nd;
      h[v] = nh;
      if (nh >= V) { status = ORC_NEG_CYCLE; break; }
      if (!inq[v]) {
        inq[v] = 1;
        fifo[(qhead + qlen) % V] = v;
        ++qlen;
      }
    }
  }
  for (int32_t v = 0; v < V; ++v) {
    dist[v] = (int32_t)(d[v] >= ORC_INF32 ? ORC_INF32 : d[v]);
    hops[v] = (int32_t)h[v];
  }
  if (n_relax) *n_relax = scanned;
  free(d); free(h); free(fifo); free(inq);
  return status;
}

/*
 * The same FIFO label-correcting Bellman-Ford, with a faster exact test for a
 * reachable negative cycle: the parent-graph search (Tarjan's observation, in
 * the "amortized search" form studied by Cherkassky and Goldberg, "Negative-
 * cycle detection algorithms", Math. Programming 85, 1999).  It is here so
 * that the status of queries on graphs of a million vertices with a planted
 * negative cycle can be decided in seconds; oracle_spfa needs about V/|C|
 * passes around a cycle C before a label reaches V hops.
 *
 *   - Every accepted label records its parent p[v] = u and the weight pw[v]
 *     of the edge (u, v) that produced it.
 *   - After every V accepted labels, the parent graph (one out-pointer per
 *     vertex) is searched for a cycle by walking the pointers from every
 *     vertex, marking each walk with its own number.
 *   - A cycle of the parent graph has negative weight.  For each parent edge,
 *     label(v) >= label(p[v]) + (pw[v], 1) holds from the moment it is set
 *     (later relaxations only lower label(p[v])), strictly for the edge set
 *     last; summed around the cycle in the ordered group Z^2 (lexicographic
 *     order) this gives (sum pw, length) < (0, 0), and as length > 0 the
 *     weight sum is negative.  Its vertices hold labels, so it is reachable.
 *     The code adds the weights up and checks the sign all the same; a
 *     non-negative sum would be a bug and returns ORC_ERR_INTERNAL.
 *   - Conversely, with a reachable negative cycle the labels never settle, so
 *     either the parent graph closes a cycle or a label reaches V hops (the
 *     test of oracle_spfa, kept as the fallback), whichever comes first.
 * Without a reachable negative cycle the parent graph is a tree and nothing
 * changes: dist, hops, the order of relaxations and *n_relax are those of
 * oracle_spfa.  *cycle_vertex (nullable) receives a vertex of the cycle found
 * by the search, or -1 (no cycle, or the hops test fired first).
 */
#define ORC_ERR_INTERNAL (-3)

static int64_t parent_graph_cycle(int32_t V, const int32_t* p, int64_t* mark,
                                  int64_t* walk) {
  /* returns a vertex on a cycle of the parent graph, or -1 */
  for (int32_t v = 0; v < V; ++v) mark[v] = 0;
  for (int32_t v = 0; v < V; ++v) {
    if (mark[v] != 0) continue;
    ++*walk;
    int32_t x = v;
    while (x >= 0 && mark[x] == 0) {
      mark[x] = *walk;
      x = p[x];
    }
    if (x >= 0 && mark[x] == *walk) return x;
  }
  return -1;
}

int oracle_spfa_cycle_search(int32_t V, const int32_t* row_ptr, const int32_t* col,
                             const int32_t* w, int32_t src, int32_t* dist,
                             int32_t* hops, int64_t* n_relax, int32_t* cycle_vertex) {
  if (!check_csr(V, row_ptr, col, src)) return ORC_ERR_INVALID;
  int64_t* d = (int64_t*)malloc(sizeof(int64_t) * (size_t)V);
  int64_t* h = (int64_t*)malloc(sizeof(int64_t) * (size_t)V);
  int32_t* fifo = (int32_t*)malloc(sizeof(int32_t) * (size_t)V);
  char* inq = (char*)calloc((size_t)V, 1);
  int32_t* p = (int32_t*)malloc(sizeof(int32_t) * (size_t)V);
  int64_t* pw = (int64_t*)malloc(sizeof(int64_t) * (size_t)V);
  int64_t* mark = (int64_t*)malloc(sizeof(int64_t) * (size_t)V);
  if (!d || !h || !fifo || !inq || !p || !pw || !mark) {
    free(d); free(h); free(fifo); free(inq); free(p); free(pw); free(mark);
    return ORC_ERR_OOM;
  }
  for (int32_t v = 0; v < V; ++v) { d[v] = ORC_INF32; h[v] = -1; p[v] = -1; pw[v] = 0; }
  d[src] = 0;
  h[src] = 0;
  int64_t qhead = 0, qlen = 1;
  fifo[0] = src;
  inq[src] = 1;
  int status = ORC_OK;
  int64_t scanned = 0, since_search = 0, walk = 0;
  int32_t found = -1;
  while (qlen > 0 && status == ORC_OK) {
    int32_t u = fifo[qhead];
    qhead = (qhead + 1) % V;
    --qlen;
    inq[u] = 0;
    int64_t du = d[u], hu = h[u];
    for (int32_t e = row_ptr[u]; e < row_ptr[u + 1]; ++e) {
      ++scanned;
      int32_t v = col[e];
      int64_t nd = du + (int64_t)w[e];
      int64_t nh = hu + 1;
      if (nd >= ORC_INF32) continue;
      if (!lex_less(nd, nh, d[v], h[v])) continue;
      if (nd <= ORC_MIN32) { status = ORC_RANGE; break; }
      d[v] = nd;
      h[v] = nh;
      p[v] = u;
      pw[v] = w[e];
      if (nh >= V) { status = ORC_NEG_CYCLE; break; }
      if (!inq[v]) {
        inq[v] = 1;
        fifo[(qhead + qlen) % V] = v;
        ++qlen;
      }
      if (++since_search >= V) {
        since_search = 0;
        int64_t c = parent_graph_cycle(V, p, mark, &walk);
        if (c >= 0) {
          int64_t sum = 0;
          int32_t x = (int32_t)c;
          do { sum += pw[x]; x = p[x]; } while (x != (int32_t)c);
          if (sum >= 0) { status = ORC_ERR_INTERNAL; break; }
          found = (int32_t)c;
          status = ORC_NEG_CYCLE;
          break;
        }
      }
    }
  }
  for (int32_t v = 0; v < V; ++v) {
    dist[v] = (int32_t)(d[v] >= ORC_INF32 ? ORC_INF32 : d[v]);
    hops[v] = (int32_t)h[v];
  }
  if (n_relax) *n_relax = scanned;
  if (cycle_vertex) *cycle_vertex = found;
  free(d); free(h); free(fifo); free(inq); free(p); free(pw); free(mark);
  return status;
}

/*
 * Distances with negative cycles resolved.  The paper stops at reporting that
 * a negative cycle is reachable; this states the usual refinement of that
 * answer, which the library offers as an option: d(v) = -infinity exactly
 * when some vertex of a negative cycle reachable from s reaches v (walks to v
 * are then unboundedly short); every other reachable v keeps its
 * lexicographic (dist, hops) label, all of whose walks avoid the -infinity
 * vertices.  Steps:
 *   1. Bellman-Ford rounds from s in int64, each round reading the previous
 *      round's distances (Jacobi form), V-1 rounds at most, stopping early
 *      after a round without change.  After round k every d[v] is the least
 *      weight over s->v walks of at most k edges.
 *   2. One further round: the head of every edge (u, v) with u reached and
 *      d[u] + w < d[v] is marked.  Each reachable negative cycle has such an
 *      edge (the inequalities cannot all fail around a cycle of negative
 *      weight), and a marked head is reachable from a negative cycle (without
 *      one, d[u] and d[v] are final after V-1 rounds and the test fails).
 *   3. Every vertex reachable from a marked vertex is -infinity.
 *   4. oracle_spfa on the graph without the -infinity vertices' edges gives
 *      the other labels (status OK or RANGE there).
 * Output: dist INT32_MIN and hops -2 on -infinity vertices, dist INT32_MAX
 * and hops -1 on unreachable ones.  Status NEG_CYCLE when a vertex is
 * -infinity, else the status of step 4.
 */
int oracle_spfa_neg_inf(int32_t V, const int32_t* row_ptr, const int32_t* col,
                        const int32_t* w, int32_t src, int32_t* dist, int32_t* hops) {
  if (!check_csr(V, row_ptr, col, src)) return ORC_ERR_INVALID;
  const int64_t E = row_ptr[V];
  const int64_t INF64 = INT64_MAX;
  int64_t* d = (int64_t*)malloc(sizeof(int64_t) * (size_t)V);
  int64_t* dn = (int64_t*)malloc(sizeof(int64_t) * (size_t)V);
  char* ninf = (char*)calloc((size_t)V, 1);
  int32_t* stack = (int32_t*)malloc(sizeof(int32_t) * (size_t)V);
  int32_t* rp2 = (int32_t*)malloc(sizeof(int32_t) * ((size_t)V + 1));
  int32_t* col2 = (int32_t*)malloc(sizeof(int32_t) * (size_t)(E > 0 ? E : 1));
  int32_t* w2 = (int32_t*)malloc(sizeof(int32_t) * (size_t)(E > 0 ? E : 1));
  if (!d || !dn || !ninf || !stack || !rp2 || !col2 || !w2) {
    free(d); free(dn); free(ninf); free(stack); free(rp2); free(col2); free(w2);
    return ORC_ERR_OOM;
  }
  /* 1. Jacobi Bellman-Ford rounds */
  for (int32_t v = 0; v < V; ++v) d[v] = INF64;
  d[src] = 0;
  int changed = 1;
  for (int64_t round = 1; round <= (int64_t)V - 1 && changed; ++round) {
    changed = 0;
    memcpy(dn, d, sizeof(int64_t) * (size_t)V);
    for (int32_t u = 0; u < V; ++u) {
      if (d[u] == INF64) continue;
      for (int32_t e = row_ptr[u]; e < row_ptr[u + 1]; ++e) {
        const int64_t nd = d[u] + (int64_t)w[e];
        if (nd < dn[col[e]]) { dn[col[e]] = nd; changed = 1; }
      }
    }
    memcpy(d, dn, sizeof(int64_t) * (size_t)V);
  }
  /* 2. heads of edges still relaxable; 3. everything they reach */
  int64_t top = 0;
  if (changed) {
    for (int32_t u = 0; u < V; ++u) {
      if (d[u] == INF64) continue;
      for (int32_t e = row_ptr[u]; e < row_ptr[u + 1]; ++e) {
        const int32_t v = col[e];
        if (d[u] + (int64_t)w[e] < d[v] && !ninf[v]) { ninf[v] = 1; stack[top++] = v; }
      }
    }
  }
  while (top > 0) {
    const int32_t u = stack[--top];
    for (int32_t e = row_ptr[u]; e < row_ptr[u + 1]; ++e) {
      const int32_t v = col[e];
      if (!ninf[v]) { ninf[v] = 1; stack[top++] = v; }
    }
  }
  /* 4. labels of the rest on the graph without the -infinity vertices' edges */
  int64_t k = 0;
  int any = 0;
  rp2[0] = 0;
  for (int32_t u = 0; u < V; ++u) {
    any |= ninf[u];
    if (!ninf[u])
      for (int32_t e = row_ptr[u]; e < row_ptr[u + 1]; ++e)
        if (!ninf[col[e]]) { col2[k] = col[e]; w2[k] = w[e]; ++k; }
    rp2[u + 1] = (int32_t)k;
  }
  int status = oracle_spfa(V, rp2, col2, w2, src, dist, hops, NULL);
  for (int32_t v = 0; v < V; ++v)
    if (ninf[v]) { dist[v] = (int32_t)ORC_MIN32; hops[v] = -2; }
  if (status >= 0 && any) status = ORC_NEG_CYCLE;
  free(d); free(dn); free(ninf); free(stack); free(rp2); free(col2); free(w2);
  return status;
}

/*
 * Dijkstra with a binary heap on lexicographic (dist, hops) keys.  Requires
 * every weight >= 0.  Used to pin the SPFA oracle through the potential
 * transform: if w'(u,v) = w(u,v) + p(u) - p(v) then every s->v path changes
 * weight by exactly p(s) - p(v), so d'(v) = d(v) + p(s) - p(v) and the hop
 * count of the optimal label is unchanged.
 */
typedef struct { int64_t d, h; int32_t v; } heap_item;

static void heap_push(heap_item* a, int64_t* n, heap_item x) {
  int64_t i = (*n)++;
  a[i] = x;
  while (i > 0) {
    int64_t p = (i - 1) / 2;
    if (!lex_less(a[i].d, a[i].h, a[p].d, a[p].h)) break;
    heap_item t = a[i]; a[i] = a[p]; a[p] = t;
    i = p;
  }
}

static heap_item heap_pop(heap_item* a, int64_t* n) {
  heap_item top = a[0];
  a[0] = a[--(*n)];
  int64_t i = 0;
  for (;;) {
    int64_t l = 2 * i + 1, r = l + 1, m = i;
    if (l < *n && lex_less(a[l].d, a[l].h, a[m].d, a[m].h)) m = l;
    if (r < *n && lex_less(a[r].d, a[r].h, a[m].d, a[m].h)) m = r;
    if (m == i) break;
    heap_item t = a[i]; a[i] = a[m]; a[m] = t;
    i = m;
  }
  return top;
}

int oracle_dijkstra(int32_t V, const int32_t* row_ptr, const int32_t* col,
                    const int32_t* w, int32_t src, int32_t* dist,
                    int32_t* hops) {
  if (!check_csr(V, row_ptr, col, src)) return ORC_ERR_INVALID;
  int64_t E = row_ptr[V];
  for (int64_t e = 0; e < E; ++e)
    if (w[e] < 0) return ORC_ERR_INVALID;
  int64_t* d = (int64_t*)malloc(sizeof(int64_t) * (size_t)V);
  int64_t* h = (int64_t*)malloc(sizeof(int64_t) * (size_t)V);
  char* done = (char*)calloc((size_t)V, 1);
  heap_item* heap = (heap_item*)malloc(sizeof(heap_item) * (size_t)(E + 1));
  if (!d || !h || !done || !heap) {
    free(d); free(h); free(done); free(heap);
    return ORC_ERR_OOM;
  }
  for (int32_t v = 0; v < V; ++v) { d[v] = ORC_INF32; h[v] = -1; }
  d[src] = 0;
  h[src] = 0;
  int64_t n = 0;
  heap_item s0 = {0, 0, src};
  heap_push(heap, &n, s0);
  while (n > 0) {
    heap_item it = heap_pop(heap, &n);
    int32_t u = it.v;
    if (done[u]) continue;
    done[u] = 1;
    for (int32_t e = row_ptr[u]; e < row_ptr[u + 1]; ++e) {
      int32_t v = col[e];
      int64_t nd = d[u] + (int64_t)w[e];
      int64_t nh = h[u] + 1;
      if (nd >= ORC_INF32 || done[v]) continue;
      if (lex_less(nd, nh, d[v], h[v])) {
        d[v] = nd;
        h[v] = nh;
        heap_item x = {nd, nh, v};
        heap_push(heap, &n, x);
      }
    }
  }
  for (int32_t v = 0; v < V; ++v) {
    dist[v] = (int32_t)d[v];
    hops[v] = (int32_t)h[v];
  }
  free(d); free(h); free(done); free(heap);
  return ORC_OK;
}

/*
 * Floyd-Warshall over the lexicographic (dist, hops) pairs, for small V (the
 * all-pairs dense form; distinct algorithm from the label-correcting oracle).
 * Values are clamped at -2^60 so that repeated passes around a negative cycle
 * cannot overflow; the clamp keeps every sign.  A negative cycle is reachable
 * from src iff some k with D[src][k] finite has D[k][k] < 0.
 *
 * dist/hops receive row src; returns OK or NEG_CYCLE.  Weights are assumed
 * small enough that no path weight reaches INT32_MAX (tests keep them so).
 */
int oracle_fw(int32_t V, const int32_t* row_ptr, const int32_t* col,
              const int32_t* w, int32_t src, int32_t* dist, int32_t* hops) {
  if (!check_csr(V, row_ptr, col, src) || V > 512) return ORC_ERR_INVALID;
  const int64_t INF = INT64_MAX / 4;
  const int64_t FLOOR = -((int64_t)1 << 60);
  size_t n = (size_t)V * (size_t)V;
  int64_t* D = (int64_t*)malloc(sizeof(int64_t) * n);
  int64_t* H = (int64_t*)malloc(sizeof(int64_t) * n);
  if (!D || !H) { free(D); free(H); return ORC_ERR_OOM; }
  for (size_t i = 0; i < n; ++i) { D[i] = INF; H[i] = 0; }
  for (int32_t i = 0; i < V; ++i) { D[(size_t)i * V + i] = 0; H[(size_t)i * V + i] = 0; }
  for (int32_t u = 0; u < V; ++u)
    for (int32_t e = row_ptr[u]; e < row_ptr[u + 1]; ++e) {
      size_t ij = (size_t)u * V + col[e];
      if (lex_less(w[e], 1, D[ij], H[ij])) { D[ij] = w[e]; H[ij] = 1; }
    }
  for (int32_t k = 0; k < V; ++k)
    for (int32_t i = 0; i < V; ++i) {
      size_t ik = (size_t)i * V + k;
      if (D[ik] >= INF) continue;
      for (int32_t j = 0; j < V; ++j) {
        size_t kj = (size_t)k * V + j, ij = (size_t)i * V + j;
        if (D[kj] >= INF) continue;
        int64_t nd = D[ik] + D[kj], nh = H[ik] + H[kj];
        if (nd < FLOOR) nd = FLOOR;
        if (nh > ((int64_t)1 << 40)) nh = (int64_t)1 << 40;
        if (lex_less(nd, nh, D[ij], H[ij])) { D[ij] = nd; H[ij] = nh; }
      }
    }
  int status = ORC_OK;
  for (int32_t k = 0; k < V; ++k)
    if (D[(size_t)src * V + k] < INF && D[(size_t)k * V + k] < 0) status = ORC_NEG_CYCLE;
  for (int32_t v = 0; v < V; ++v) {
    size_t sv = (size_t)src * V + v;
    dist[v] = D[sv] >= INF ? (int32_t)ORC_INF32 : (int32_t)D[sv];
    hops[v] = D[sv] >= INF ? -1 : (int32_t)H[sv];
  }
  free(D); free(H);
  return status;
}

/*
 * Predecessor-tree invariant (the predecessor choice is not unique under ties,
 * so it is checked, not compared): for every reachable v != src, (pred[v], v)
 * must be an edge with dist[v] == dist[pred[v]] + w; pred[src] == -1 and
 * pred[v] == -1 for unreachable v; following pred from any reachable v reaches
 * src within V steps.  Returns 1 if all hold, else 0.
 */
int oracle_check_pred(int32_t V, const int32_t* row_ptr, const int32_t* col,
                      const int32_t* w, int32_t src, const int32_t* dist,
                      const int32_t* pred) {
  if (!check_csr(V, row_ptr, col, src)) return 0;
  if (pred[src] != -1 || dist[src] != 0) return 0;
  for (int32_t v = 0; v < V; ++v) {
    if (v == src) continue;
    if (dist[v] == (int32_t)ORC_INF32) { if (pred[v] != -1) return 0; continue; }
    int32_t u = pred[v];
    if (u < 0 || u >= V || dist[u] == (int32_t)ORC_INF32) return 0;
    int tight = 0;
    for (int32_t e = row_ptr[u]; e < row_ptr[u + 1] && !tight; ++e)
      if (col[e] == v && (int64_t)dist[u] + w[e] == (int64_t)dist[v]) tight = 1;
    if (!tight) return 0;
  }
  /* acyclic: every chain ends at src within V steps */
  for (int32_t v = 0; v < V; ++v) {
    if (dist[v] == (int32_t)ORC_INF32) continue;
    int32_t x = v;
    int64_t steps = 0;
    while (x != src && steps <= V) { x = pred[x]; ++steps; }
    if (x != src) return 0;
  }
  return 1;
}

/*
 * Number of directed edges whose tail is reachable from the source
 * (dist < INT32_MAX): the numerator of traversed-edges-per-second.
 */
int64_t oracle_reached_edges(int32_t V, const int32_t* row_ptr,
                             const int32_t* dist) {
  int64_t m = 0;
  for (int32_t v = 0; v < V; ++v)
    if (dist[v] != (int32_t)ORC_INF32) m += row_ptr[v + 1] - row_ptr[v];
  return m;
}
