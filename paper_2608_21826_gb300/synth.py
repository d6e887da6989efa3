"""Seeded synthetic graph generators (inputs only).

These build the workloads: grids, road-like grids with dropped edges and
shortcuts, R-MAT power-law graphs, potential-shifted weights that create
negative edges without negative cycles, planted negative cycles, and the
batched mix.  Everything draws from ``numpy.random.Generator(PCG64(seed))``
so a seed gives the same graph on every host.  Nothing here computes shortest
paths: both the CUDA path and the oracle receive these arrays as inputs.

The paper evaluates on SuiteSparse matrices (Sec. IV, Table I); these seeded
graphs stand in for them.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

INF32 = 2147483647


def rng_for(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


@dataclasses.dataclass
class Graph:
    """CSR graph: row_ptr int32[V+1], col int32[E], w int32[E].

    ``base_w``/``potential`` are kept when the weights were made by the
    potential shift w = base_w + p[u] - p[v] with base_w >= 0 (else None).
    ``sources`` are the query sources the workload prescribes."""
    name: str
    row_ptr: np.ndarray
    col: np.ndarray
    w: np.ndarray
    sources: np.ndarray
    base_w: np.ndarray | None = None
    potential: np.ndarray | None = None
    cycle: np.ndarray | None = None      # vertices of a planted negative cycle

    @property
    def V(self) -> int:
        return len(self.row_ptr) - 1

    @property
    def E(self) -> int:
        return len(self.col)

    def tails(self) -> np.ndarray:
        """Source vertex of every edge (int32[E])."""
        deg = np.diff(self.row_ptr)
        return np.repeat(np.arange(self.V, dtype=np.int32), deg)


def csr_from_edges(V: int, u: np.ndarray, v: np.ndarray, dedupe: bool = True,
                   drop_self_loops: bool = True, return_order: bool = False):
    """Sort directed edges by (u, v); optionally drop self-loops and repeats
    (the first occurrence of a repeated edge is kept).  Returns
    (row_ptr, col, order) where ``order`` indexes the kept input edges, or is
    None unless ``return_order``."""
    if V >= 2**31:
        raise ValueError("vertex count exceeds int32")
    u = np.asarray(u)
    v = np.asarray(v)
    key = (u.astype(np.uint64) << np.uint64(32)) | v.astype(np.uint64)
    idx = np.nonzero(u != v)[0] if drop_self_loops else None
    if idx is not None:
        key = key[idx]
    order = None
    if return_order:
        srt = np.argsort(key, kind="stable")
        key = key[srt]
        order = srt if idx is None else idx[srt]
    else:
        key = np.sort(key)
    if dedupe and key.size:
        first = np.empty(key.size, dtype=bool)
        first[0] = True
        np.not_equal(key[1:], key[:-1], out=first[1:])
        key = key[first]
        if order is not None:
            order = order[first]
    uu = (key >> np.uint64(32)).astype(np.int64)
    row_ptr = np.zeros(V + 1, dtype=np.int64)
    np.cumsum(np.bincount(uu, minlength=V), out=row_ptr[1:])
    if row_ptr[-1] >= 2**31:
        raise ValueError("edge count exceeds int32 CSR")
    col = (key & np.uint64(0xFFFFFFFF)).astype(np.int32)
    return row_ptr.astype(np.int32), col, order


def potential_shift(row_ptr: np.ndarray, col: np.ndarray, base_w: np.ndarray,
                    p: np.ndarray) -> np.ndarray:
    """w'(u,v) = w(u,v) + p(u) - p(v), in int64 then checked into int32."""
    V = len(row_ptr) - 1
    u = np.repeat(np.arange(V, dtype=np.int64), np.diff(row_ptr))
    w = base_w.astype(np.int64) + p[u].astype(np.int64) - p[col].astype(np.int64)
    if w.size and (w.min() < -(2**31) or w.max() >= 2**31):
        raise ValueError("shifted weight outside int32")
    return w.astype(np.int32)


def _finish(name, V, u, v, rng, wmax, pmax, n_sources, wmin=1, src_fixed=None,
            dedupe=True):
    row_ptr, col, _ = csr_from_edges(V, u, v, dedupe=dedupe)
    E = len(col)
    base_w = rng.integers(wmin, wmax, size=E, endpoint=True, dtype=np.int32)
    p = rng.integers(0, pmax, size=V, endpoint=True, dtype=np.int32)
    w = potential_shift(row_ptr, col, base_w, p)
    if src_fixed is not None:
        sources = np.asarray(src_fixed, dtype=np.int32)
    else:
        deg = np.diff(row_ptr)
        cand = np.nonzero(deg > 0)[0]
        if len(cand) == 0:
            cand = np.arange(V)
        sources = np.sort(rng.choice(cand, size=min(n_sources, len(cand)),
                                     replace=False)).astype(np.int32)
    return Graph(name, row_ptr, col, w, sources, base_w=base_w, potential=p)


def _grid_undirected(rows: int, cols: int):
    r, c = np.meshgrid(np.arange(rows), np.arange(cols), indexing="ij")
    vid = (r * cols + c).astype(np.int64)
    hu, hv = vid[:, :-1].ravel(), vid[:, 1:].ravel()
    vu, vv = vid[:-1, :].ravel(), vid[1:, :].ravel()
    return np.concatenate([hu, vu]), np.concatenate([hv, vv])


def grid_graph(rows: int = 64, cols: int = 64, seed: int = 1, wmax: int = 100,
               pmax: int = 50, src: int = 0) -> Graph:
    """4-neighbour grid, both directions, base w ~ U[1,wmax], p ~ U[0,pmax]."""
    rng = rng_for(seed)
    a, b = _grid_undirected(rows, cols)
    u = np.concatenate([a, b])
    v = np.concatenate([b, a])
    return _finish(f"grid{rows}x{cols}", rows * cols, u, v, rng, wmax, pmax, 1,
                   src_fixed=[src])


def road_graph(n: int = 1024, seed: int = 2, drop: float = 0.10,
               shortcut_frac: float = 0.01, wmax: int = 1000, pmax: int = 500,
               n_sources: int = 8) -> Graph:
    """n x n grid with a fraction ``drop`` of undirected edges removed and
    round(shortcut_frac * V) random undirected long-range shortcuts added;
    both directions kept, duplicates removed."""
    rng = rng_for(seed)
    V = n * n
    a, b = _grid_undirected(n, n)
    m = len(a)
    keep = rng.permutation(m)[: int(round((1.0 - drop) * m))]
    a, b = a[keep], b[keep]
    ns = int(round(shortcut_frac * V))
    sa = rng.integers(0, V, size=ns, dtype=np.int64)
    sb = rng.integers(0, V, size=ns, dtype=np.int64)
    a = np.concatenate([a, sa])
    b = np.concatenate([b, sb])
    u = np.concatenate([a, b])
    v = np.concatenate([b, a])
    g = _finish(f"road{n}x{n}", V, u, v, rng, wmax, pmax, 0)
    g.sources = np.sort(rng.choice(V, size=n_sources, replace=False)).astype(np.int32)
    return g


def _pair_table(abcd):
    """Map a 16-bit uniform to the joint outcome of two R-MAT levels: the 16
    (quadrant, quadrant) pairs get consecutive runs of the 65536 codes in
    proportion to their probabilities.  Entry = (u bits << 2) | v bits."""
    probs = np.asarray(abcd, dtype=np.float64)
    ubit = np.array([0, 0, 1, 1])
    vbit = np.array([0, 1, 0, 1])
    joint = np.outer(probs, probs).ravel()            # (first, second) level
    bounds = np.rint(np.cumsum(joint) * 65536.0).astype(np.int64)
    bounds[-1] = 65536
    code = np.searchsorted(bounds, np.arange(65536), side="right")
    q1, q2 = code // 4, code % 4
    ub = (ubit[q1] << 1) | ubit[q2]
    vb = (vbit[q1] << 1) | vbit[q2]
    return ((ub << 2) | vb).astype(np.uint8)


def rmat_edges(scale: int, n_edges: int, rng: np.random.Generator,
               abcd=(0.57, 0.19, 0.19, 0.05), permute: bool = True):
    """R-MAT edge endpoints over 2**scale ids.  Each level picks one of the four
    quadrants with probabilities (a, b, c, d) and appends one bit to each
    endpoint; two levels are drawn at a time from one 16-bit uniform (see
    ``_pair_table``).  Ids are then relabelled by a random permutation."""
    table = _pair_table(abcd)
    u = np.zeros(n_edges, dtype=np.uint32)
    v = np.zeros(n_edges, dtype=np.uint32)
    level = 0
    while level < scale:
        r = rng.integers(0, 65536, size=n_edges, dtype=np.uint16)
        t = table[r]
        if scale - level >= 2:
            u <<= np.uint32(2)
            v <<= np.uint32(2)
            u |= t >> np.uint8(2)
            v |= t & np.uint8(3)
            level += 2
        else:                                   # odd scale: use the first level
            u <<= np.uint32(1)
            v <<= np.uint32(1)
            u |= t >> np.uint8(3)
            v |= (t >> np.uint8(1)) & np.uint8(1)
            level += 1
        del r, t
    if permute:
        perm = rng.permutation(1 << scale).astype(np.uint32)
        u = perm[u]
        v = perm[v]
    return u, v


def rmat_graph(scale: int = 22, edge_factor: int = 16, seed: int = 3,
               abcd=(0.57, 0.19, 0.19, 0.05), wmax: int = 255, pmax: int = 128,
               n_sources: int = 4, V: int | None = None) -> Graph:
    """R-MAT power-law graph, edge_factor * 2**scale directed edges before
    self-loop and duplicate removal.  With ``V`` given (< 2**scale) ids are
    folded onto [0, V) after the permutation."""
    rng = rng_for(seed)
    nv = 1 << scale
    m = int(edge_factor * (V if V is not None else nv))
    u, v = rmat_edges(scale, m, rng, abcd)
    if V is not None:
        u %= np.uint32(V)
        v %= np.uint32(V)
        nv = V
    return _finish(f"rmat{scale}", nv, u, v, rng, wmax, pmax, n_sources)


def random_graph(V: int, E: int, seed: int, wlo: int = -10, whi: int = 20,
                 dedupe: bool = True) -> Graph:
    """Uniform random directed graph with weights ~ U[wlo, whi] (no potential
    structure: negative cycles may exist).  Source 0."""
    rng = rng_for(seed)
    u = rng.integers(0, V, size=E, dtype=np.int64)
    v = rng.integers(0, V, size=E, dtype=np.int64)
    row_ptr, col, _ = csr_from_edges(V, u, v, dedupe=dedupe)
    w = rng.integers(wlo, whi, size=len(col), endpoint=True, dtype=np.int32)
    return Graph(f"rand{V}_{E}", row_ptr, col, w, np.array([0], np.int32))


def random_potential_graph(V: int, E: int, seed: int, wmax: int = 20,
                               pmax: int = 30) -> Graph:
    """Random directed graph with potential-shifted weights (negative edges,
    no negative cycle).  Source 0."""
    rng = rng_for(seed)
    u = rng.integers(0, V, size=E, dtype=np.int64)
    v = rng.integers(0, V, size=E, dtype=np.int64)
    return _finish(f"randpot{V}_{E}", V, u, v, rng, wmax, pmax, 0, wmin=0,
                   src_fixed=[0])


def reachable(row_ptr: np.ndarray, col: np.ndarray, src: int) -> np.ndarray:
    """Boolean mask of vertices reachable from ``src`` (level-synchronous
    search, vectorised over each frontier)."""
    V = len(row_ptr) - 1
    seen = np.zeros(V, dtype=bool)
    seen[src] = True
    frontier = np.array([src], dtype=np.int64)
    while frontier.size:
        starts = row_ptr[frontier].astype(np.int64)
        ends = row_ptr[frontier + 1].astype(np.int64)
        lens = ends - starts
        total = int(lens.sum())
        if total == 0:
            break
        offs = np.repeat(starts - np.concatenate([[0], np.cumsum(lens)[:-1]]), lens)
        nbr = col[np.arange(total, dtype=np.int64) + offs].astype(np.int64)
        nbr = np.unique(nbr[~seen[nbr]])
        seen[nbr] = True
        frontier = nbr
    return seen


def plant_negative_cycle(g: Graph, length: int = 5, seed: int = 7,
                         reachable_from=None, base_weight: int = -1) -> Graph:
    """Add a cycle of ``length`` edges whose base weights sum to
    length * base_weight < 0, potential-shifted like the other edges (the shift
    cancels around a cycle).  Cycle vertices are drawn from the vertices
    reachable from every vertex of ``reachable_from`` (default: g.sources);
    pass an empty list to draw from vertices reachable from none of them.
    An existing edge on the cycle is replaced."""
    rng = rng_for(seed)
    V = g.V
    srcs = g.sources if reachable_from is None else np.asarray(reachable_from)
    if len(srcs):
        mask = np.ones(V, dtype=bool)
        for s in srcs:
            mask &= reachable(g.row_ptr, g.col, int(s))
    else:
        mask = np.ones(V, dtype=bool)
        for s in g.sources:
            mask &= ~reachable(g.row_ptr, g.col, int(s))
    cand = np.nonzero(mask)[0]
    if len(cand) < length:
        raise ValueError("not enough candidate vertices for the cycle")
    cyc = rng.choice(cand, size=length, replace=False).astype(np.int64)
    tails = g.tails().astype(np.int64)
    cu = cyc
    cv = np.roll(cyc, -1)
    u = np.concatenate([cu, tails])           # cycle edges first: kept by dedupe
    v = np.concatenate([cv, g.col.astype(np.int64)])
    p = g.potential if g.potential is not None else np.zeros(V, np.int32)
    bw_old = g.base_w if g.base_w is not None else g.w
    bw = np.concatenate([np.full(length, base_weight, np.int64), bw_old.astype(np.int64)])
    row_ptr, col, order = csr_from_edges(V, u, v, dedupe=True, drop_self_loops=True,
                                         return_order=True)
    base_w = bw[order].astype(np.int32)
    w = potential_shift(row_ptr, col, base_w, p)
    return Graph(g.name + "+negcycle", row_ptr, col, w, g.sources.copy(),
                 base_w=None, potential=p, cycle=cyc.astype(np.int32))


def path_graph(V: int, weights) -> Graph:
    """0 -> 1 -> ... -> V-1 with the given V-1 weights."""
    weights = np.asarray(weights, dtype=np.int32)
    row_ptr = np.concatenate([np.arange(V, dtype=np.int32), [V - 1]]).astype(np.int32)
    col = np.arange(1, V, dtype=np.int32)
    return Graph(f"path{V}", row_ptr, col, weights, np.array([0], np.int32))


def star_graph(V: int, weights) -> Graph:
    """0 -> i for i = 1..V-1 with the given weights."""
    weights = np.asarray(weights, dtype=np.int32)
    row_ptr = np.full(V + 1, V - 1, dtype=np.int32)
    row_ptr[0] = 0
    col = np.arange(1, V, dtype=np.int32)
    return Graph(f"star{V}", row_ptr, col, weights, np.array([0], np.int32))


# ---------------------------------------------------------------------------
# Named workloads
# ---------------------------------------------------------------------------

def workload_grid4k() -> Graph:
    """64x64 grid, base w U[1,100], p U[0,50], source 0 (V=4096, E=16128)."""
    return grid_graph(64, 64, seed=101, wmax=100, pmax=50, src=0)


def workload_road1m(n: int = 1024) -> Graph:
    """1024^2 road-like grid: 10% edges dropped, 1% shortcuts, w U[1,1000],
    p U[0,500], 8 sources."""
    return road_graph(n, seed=202, drop=0.10, shortcut_frac=0.01, wmax=1000,
                      pmax=500, n_sources=8)


def workload_rmat(scale: int = 22, edge_factor: int = 16) -> Graph:
    """R-MAT (0.57,0.19,0.19,0.05), w U[1,255], p U[0,128], 4 sources with
    out-degree >= 1."""
    return rmat_graph(scale, edge_factor, seed=303 + scale, wmax=255, pmax=128,
                      n_sources=4)


def workload_batched(n_graphs: int = 64, seed: int = 404, vmin: float = 1e3,
                     vmax: float = 1e6, sources_per_graph: int = 8,
                     cycle_frac: float = 0.10):
    """The batched mix: ``n_graphs`` graphs, V log-uniform in [vmin, vmax],
    average degree U[4,16], alternating grid-with-shortcuts and R-MAT, each
    with its own potential-shifted weights; round(cycle_frac * n_graphs) of
    them get a planted 5-edge negative cycle reachable from all of their
    sources.  Returns (graphs, queries) with queries an int32 array of
    (graph_id, src) rows, sources_per_graph per graph."""
    rng = rng_for(seed)
    graphs = []
    for i in range(n_graphs):
        V = int(round(math.exp(rng.uniform(math.log(vmin), math.log(vmax)))))
        deg = float(rng.uniform(4.0, 16.0))
        gseed = int(rng.integers(0, 2**31 - 1))
        if i % 2 == 0:
            rows = max(2, int(round(math.sqrt(V))))
            cols = max(2, int(round(V / rows)))
            V = rows * cols
            grng = rng_for(gseed)
            a, b = _grid_undirected(rows, cols)
            ns = int(round(max(0.0, deg - 4.0) / 2.0 * V))
            sa = grng.integers(0, V, size=ns, dtype=np.int64)
            sb = grng.integers(0, V, size=ns, dtype=np.int64)
            a = np.concatenate([a, sa])
            b = np.concatenate([b, sb])
            g = _finish(f"b{i}_grid{rows}x{cols}", V, np.concatenate([a, b]),
                        np.concatenate([b, a]), grng, 100, 50, sources_per_graph)
        else:
            scale = max(1, int(math.ceil(math.log2(V))))
            grng = rng_for(gseed)
            u, v = rmat_edges(scale, int(round(deg * V)), grng)
            u %= np.uint32(V)
            v %= np.uint32(V)
            g = _finish(f"b{i}_rmat{V}", V, u, v, grng, 255, 128, sources_per_graph)
        graphs.append(g)
    n_cyc = int(round(cycle_frac * n_graphs))
    cyc_ids = rng.choice(n_graphs, size=n_cyc, replace=False) if n_cyc else []
    for gi in sorted(int(x) for x in cyc_ids):
        g = graphs[gi]
        # sources from the largest set reachable from one source: keep the
        # sources that reach a common set of at least 5 vertices
        big = reachable(g.row_ptr, g.col, int(g.sources[0]))
        srcs = [s for s in g.sources if big[s]] or [int(g.sources[0])]
        g.sources = np.asarray(srcs, dtype=np.int32)
        # top up to sources_per_graph with vertices inside the reached set
        if len(g.sources) < sources_per_graph:
            pool = np.setdiff1d(np.nonzero(big & (np.diff(g.row_ptr) > 0))[0], g.sources)
            extra = rng.choice(pool, size=min(len(pool), sources_per_graph - len(g.sources)),
                               replace=False)
            g.sources = np.sort(np.concatenate([g.sources, extra])).astype(np.int32)
        graphs[gi] = plant_negative_cycle(g, 5, seed=gseed_for(seed, gi))
    q = []
    for gi, g in enumerate(graphs):
        for s in g.sources:
            q.append((gi, int(s)))
    return graphs, np.asarray(q, dtype=np.int32)


def gseed_for(seed: int, i: int) -> int:
    return (seed * 1_000_003 + i * 7919) % (2**31 - 1)
