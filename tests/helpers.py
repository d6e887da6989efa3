"""Shared test helpers: golden-fixture parsing and small brute-force checks."""
from __future__ import annotations

import concurrent.futures as cf
import functools
import glob
import itertools
import os

import numpy as np

from paper_2608_21826_gb300 import synth

GOLDEN_DIR = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")
INF = 2147483647


NEG_INF = -2147483648


def _ints(tokens):
    return [INF if t == "INF" else NEG_INF if t == "NEGINF" else int(t) for t in tokens]


def load_golden(path):
    """Parse one fixture into (Graph, expected dict)."""
    lines = [ln.split("#")[0].strip() for ln in open(path)]
    lines = [ln for ln in lines if ln]
    V, src = map(int, lines[0].split())
    assert lines[1] == "edges"
    edges, exp = [], {}
    for ln in lines[2:]:
        tok = ln.split()
        if tok[0] in ("dist", "hops", "status"):
            exp[tok[0]] = _ints(tok[1:])
        else:
            edges.append(tuple(int(t) for t in tok))
    u = np.array([e[0] for e in edges], np.int64)
    v = np.array([e[1] for e in edges], np.int64)
    w = np.array([e[2] for e in edges], np.int64)
    row_ptr, col, order = synth.csr_from_edges(V, u, v, dedupe=False,
                                               drop_self_loops=False, return_order=True)
    g = synth.Graph(os.path.basename(path), row_ptr, col, w[order].astype(np.int32),
                    np.array([src], np.int32))
    exp["status"] = exp["status"][0]
    return g, exp


def golden_files():
    return sorted(glob.glob(os.path.join(GOLDEN_DIR, "*.txt")))


def golden_neg_inf_files():
    return sorted(glob.glob(os.path.join(GOLDEN_DIR, "neg_inf", "*.txt")))


def brute_force(g, src):
    """Enumerate simple paths (tiny V only).  Returns (has_neg_cycle, dist, hops)
    with dist/hops the lexicographic minimum over simple s->v paths and
    has_neg_cycle true iff a simple cycle of negative weight is reachable."""
    V = g.V
    adj = {u: [] for u in range(V)}
    for u in range(V):
        for e in range(g.row_ptr[u], g.row_ptr[u + 1]):
            adj[u].append((int(g.col[e]), int(g.w[e])))
    best = {src: (0, 0)}
    reach = {src}

    def dfs(u, d, h, on_path):
        for v, w in adj[u]:
            if v in on_path:
                continue
            nd, nh = d + w, h + 1
            reach.add(v)
            if v not in best or (nd, nh) < best[v]:
                best[v] = (nd, nh)
            on_path.add(v)
            dfs(v, nd, nh, on_path)
            on_path.discard(v)

    dfs(src, 0, 0, {src})
    neg = False
    # simple cycles through each reachable start vertex c: DFS back to c
    def cyc(c, u, d, on_path):
        nonlocal neg
        for v, w in adj[u]:
            if v == c and d + w < 0:
                neg = True
            if v != c and v not in on_path and v > c:
                on_path.add(v)
                cyc(c, v, d + w, on_path)
                on_path.discard(v)
    for c in sorted(reach):
        cyc(c, c, 0, {c})
    dist = np.full(V, INF, np.int64)
    hops = np.full(V, -1, np.int64)
    for v, (d, h) in best.items():
        dist[v], hops[v] = d, h
    return neg, dist, hops


def subgraph_without(g, drop):
    """The same vertices with every edge that touches a vertex in `drop`
    removed (CSR order kept)."""
    drop = np.asarray(drop, bool)
    rp = [0]
    col, w = [], []
    for u in range(g.V):
        for e in range(g.row_ptr[u], g.row_ptr[u + 1]):
            v = int(g.col[e])
            if not drop[u] and not drop[v]:
                col.append(v)
                w.append(int(g.w[e]))
        rp.append(len(col))
    return synth.Graph(g.name + "-sub", np.array(rp, np.int32), np.array(col, np.int32),
                       np.array(w, np.int32), g.sources)


def brute_force_neg_inf(g, src):
    """Distances with negative cycles resolved, by enumeration (tiny V only):
    every simple cycle of negative weight through a vertex reachable from
    src marks its vertices; everything they reach is -inf; the other labels
    are the lexicographic minimum over simple paths avoiding the -inf
    vertices.  Returns (any_neg_inf, dist, hops) with (INT32_MIN, -2) on
    -inf vertices."""
    V = g.V
    adj = {u: [] for u in range(V)}
    for u in range(V):
        for e in range(g.row_ptr[u], g.row_ptr[u + 1]):
            adj[u].append((int(g.col[e]), int(g.w[e])))
    reach = bfs_levels(g, src) >= 0
    seeds = set()

    def cyc(c, u, d, path):
        for v, w in adj[u]:
            if v == c and d + w < 0:
                seeds.update(path)
            if v != c and v not in path and v > c:
                cyc(c, v, d + w, path + [v])
    for c in range(V):
        if reach[c]:
            cyc(c, c, 0, [c])
    ninf = np.zeros(V, bool)
    stack = list(seeds)
    for s in stack:
        ninf[s] = True
    while stack:
        u = stack.pop()
        for v, _ in adj[u]:
            if not ninf[v]:
                ninf[v] = True
                stack.append(v)
    _, dist, hops = brute_force(subgraph_without(g, ninf), src)
    dist[ninf] = NEG_INF
    hops[ninf] = -2
    return bool(ninf.any()), dist, hops


def bfs_levels(g, src):
    V = g.V
    lev = np.full(V, -1, np.int64)
    lev[src] = 0
    front = [src]
    while front:
        nxt = []
        for u in front:
            for e in range(g.row_ptr[u], g.row_ptr[u + 1]):
                v = int(g.col[e])
                if lev[v] < 0:
                    lev[v] = lev[u] + 1
                    nxt.append(v)
        front = nxt
    return lev


def shifted_expectation(dist_base, hops_base, p, s):
    """d'(v) = d(v) + p(s) - p(v) for reachable v (potential transform)."""
    p = p.astype(np.int64)
    d = dist_base.astype(np.int64)
    out = np.where(d == INF, INF, d + p[s] - p)
    return out, hops_base


@functools.lru_cache(maxsize=1)
def batched_workload():
    """The full batched mix (64 graphs, 512 queries), generated once per
    test process."""
    return synth.workload_batched()


def oracle_many(jobs, threads=None):
    """Run oracle.spfa_cycle_search on many (graph, src) jobs in threads (the
    oracle is C called through ctypes, which releases the GIL; no processes
    are forked).  Returns a list of (status, dist, hops) in job order."""
    import oracle

    def one(job):
        g, s = job
        st, d, h, _, _ = oracle.spfa_cycle_search(g.row_ptr, g.col, g.w, int(s))
        return st, d, h

    with cf.ThreadPoolExecutor(max_workers=threads or min(16, os.cpu_count() or 4)) as ex:
        return list(ex.map(one, jobs))
