"""Seeded synthetic graph generators (inputs only; no algebraic-distance arithmetic).

The paper evaluates on 18 real social, biological and citation networks
(Table 2: 1M-34M edges, heavy-tailed degrees, min degree 1).  Those files are
not available here, so benchmarks and tests use synthetic graphs with the same
shapes: 2-D grids, R-MAT (Chakrabarti et al.), Barabasi-Albert preferential
attachment and Watts-Strogatz small worlds.

Every generator returns an undirected simple graph as a symmetric CSR with
sorted columns (``row_ptr`` int64[n+1], ``col`` int32[nnz]) and an optional
FP32 weight per CSR entry (both directions of an edge carry the same weight).
The upper-triangle pairs (i < j) in row-major order are the edge ids used by
the library; ``edges_upper`` lists them in that order.

This module is shared by the tests, the benchmark and the FP64 reference; it
holds none of the method's arithmetic.
"""
from __future__ import annotations

import dataclasses
import hashlib

import numpy as np


@dataclasses.dataclass
class Graph:
    n: int
    row_ptr: np.ndarray          # int64 [n+1]
    col: np.ndarray              # int32 [nnz]
    weight: np.ndarray | None    # float32 [nnz] or None (unit weights)
    name: str = ""

    @property
    def nnz(self) -> int:
        return int(self.row_ptr[-1])

    @property
    def m(self) -> int:
        return self.nnz // 2

    def degrees(self) -> np.ndarray:
        return np.diff(self.row_ptr)

    def edges_upper(self):
        """(u, v) with u < v for every edge, in edge-id order."""
        rows = np.repeat(np.arange(self.n, dtype=np.int64), self.degrees())
        up = self.col > rows
        return rows[up].astype(np.int32), self.col[up].copy()

    def edge_weights(self) -> np.ndarray | None:
        """Weight of each undirected edge in edge-id order (None for unit weights)."""
        if self.weight is None:
            return None
        rows = np.repeat(np.arange(self.n, dtype=np.int64), self.degrees())
        return self.weight[self.col > rows].copy()

    def digest(self) -> str:
        h = hashlib.sha256()
        h.update(np.int64(self.n).tobytes())
        h.update(self.row_ptr.tobytes())
        h.update(self.col.tobytes())
        if self.weight is not None:
            h.update(self.weight.tobytes())
        return h.hexdigest()[:16]


def from_edges(n: int, u, v, edge_weight=None, name: str = "") -> Graph:
    """Symmetric CSR from an undirected edge list.  Self loops are dropped and
    duplicate pairs merged (the first weight of a duplicated pair is kept)."""
    u = np.asarray(u, dtype=np.int64)
    v = np.asarray(v, dtype=np.int64)
    keep = u != v
    a, b = np.minimum(u[keep], v[keep]), np.maximum(u[keep], v[keep])
    key = a * np.int64(n) + b
    w = None
    if edge_weight is not None:
        order = np.argsort(key, kind="stable")
        key = key[order]
        w = np.asarray(edge_weight, dtype=np.float32)[keep][order]
    else:
        key = np.sort(key)
    first = np.ones(len(key), dtype=bool)
    first[1:] = key[1:] != key[:-1]
    key = key[first]
    if w is not None:
        w = w[first]
    # upper pairs (a < b) in (a, b) order = edge-id order
    a = (key // n).astype(np.int64)
    b = (key % n).astype(np.int64)
    m = len(key)
    cnt_up = np.bincount(a, minlength=n)
    cnt_lo = np.bincount(b, minlength=n)
    row_ptr = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(cnt_up + cnt_lo, out=row_ptr[1:])
    col = np.empty(2 * m, dtype=np.int32)
    # row i = its lower entries (columns a < i, in a order) then its upper entries (b > i)
    lo_order = np.argsort(b, kind="stable")
    lo_start = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(cnt_lo, out=lo_start[1:])
    bl = b[lo_order]
    pos_lo = row_ptr[bl] + (np.arange(m, dtype=np.int64) - lo_start[bl])
    col[pos_lo] = a[lo_order]
    up_start = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(cnt_up, out=up_start[1:])
    pos_up = row_ptr[a] + cnt_lo[a] + (np.arange(m, dtype=np.int64) - up_start[a])
    col[pos_up] = b
    weight = None
    if w is not None:
        weight = np.empty(2 * m, dtype=np.float32)
        weight[pos_lo] = w[lo_order]
        weight[pos_up] = w
    return Graph(n=n, row_ptr=row_ptr, col=col, weight=weight, name=name)


def with_edge_weights(g: Graph, edge_weight) -> Graph:
    """Attach one weight per undirected edge (edge-id order) to both CSR directions."""
    ew = np.asarray(edge_weight, dtype=np.float32)
    assert ew.shape == (g.m,)
    rows = np.repeat(np.arange(g.n, dtype=np.int64), g.degrees())
    # edge id of every CSR entry: upper entries are numbered in order; a lower
    # entry (i, j < i) shares the id of the upper entry (j, i).
    up = g.col > rows
    eid = np.full(g.nnz, -1, dtype=np.int64)
    eid[up] = np.arange(g.m)
    key_up = rows[up] * g.n + g.col[up]
    key_lo = g.col[~up].astype(np.int64) * g.n + rows[~up]
    eid[~up] = np.searchsorted(key_up, key_lo)
    return Graph(n=g.n, row_ptr=g.row_ptr, col=g.col, weight=ew[eid].astype(np.float32), name=g.name)


# --------------------------------------------------------------------------- families
def grid2d(rows: int, cols: int) -> Graph:
    """4-neighbour grid, vertex id = r * cols + c, unit weights."""
    idx = np.arange(rows * cols, dtype=np.int64).reshape(rows, cols)
    u = np.concatenate([idx[:, :-1].ravel(), idx[:-1, :].ravel()])
    v = np.concatenate([idx[:, 1:].ravel(), idx[1:, :].ravel()])
    return from_edges(rows * cols, u, v, name=f"grid{rows}x{cols}")


def rmat(scale: int, edge_factor: int = 16, a=0.57, b=0.19, c=0.19, seed: int = 2) -> Graph:
    """R-MAT without noise; symmetrised, self loops and duplicates removed,
    vertex ids as generated (isolated vertices kept)."""
    n = 1 << scale
    E = edge_factor * n
    rng = np.random.default_rng(seed)
    src = np.zeros(E, dtype=np.uint32)
    dst = np.zeros(E, dtype=np.uint32)
    ab, abc = np.float32(a + b), np.float32(a + b + c)
    fa = np.float32(a)
    for _ in range(scale):
        r = rng.random(E, dtype=np.float32)
        src <<= 1
        src |= (r >= ab)                                       # quadrants c, d: lower half
        dst <<= 1
        dst |= ((r >= fa) & (r < ab)) | (r >= abc)             # quadrants b, d: right half
    return from_edges(n, src, dst, name=f"rmat{scale}_ef{edge_factor}")


def barabasi_albert(n: int, m: int = 8, seed: int = 3) -> Graph:
    """Preferential attachment through the repeated-endpoints list: a clique on
    m + 1 vertices, then vertex t adds m edges whose far ends are uniform picks
    from the endpoint list of all earlier edges (Batagelj-Brandes).  Repeated
    picks of one vertex collapse into one edge."""
    m0 = m + 1
    cu, cv = np.triu_indices(m0, 1)
    n_clique = len(cu)
    n_new = (n - m0) * m
    E = n_clique + n_new
    src = np.empty(E, dtype=np.int64)
    tgt = np.full(E, -1, dtype=np.int64)
    src[:n_clique] = cu
    tgt[:n_clique] = cv
    t = np.repeat(np.arange(m0, n, dtype=np.int64), m)
    src[n_clique:] = t
    rng = np.random.default_rng(seed)
    # endpoint list position of edge f: 2f (its source) and 2f+1 (its target);
    # new vertex t may pick any position before its own first edge.
    first_edge = n_clique + (t - m0) * m
    pos = np.floor(rng.random(n_new) * (2 * first_edge)).astype(np.int64)
    ptr = np.full(E, -1, dtype=np.int64)     # for unresolved targets: edge whose target we copy
    res = tgt.copy()
    even = (pos % 2) == 0
    idx_new = np.arange(n_clique, E)
    res[idx_new[even]] = src[pos[even] // 2]
    ptr[idx_new[~even]] = pos[~even] // 2
    pending = idx_new[~even]
    while len(pending):
        f = ptr[pending]
        done = res[f] >= 0
        res[pending[done]] = res[f[done]]
        pending = pending[~done]
        ptr[pending] = ptr[f[~done]]                      # pointer jumping
    return from_edges(n, src, res, name=f"ba{n}_m{m}")


def watts_strogatz(n: int, k: int = 10, p: float = 0.1, seed: int = 4) -> Graph:
    """Ring lattice with k/2 neighbours per side; each lattice edge has its far
    end rewired with probability p to a uniform vertex (self loops redrawn,
    duplicates merged)."""
    half = k // 2
    base = np.arange(n, dtype=np.int64)
    u = np.repeat(base, half)
    v = (u + np.tile(np.arange(1, half + 1, dtype=np.int64), n)) % n
    rng = np.random.default_rng(seed)
    rew = rng.random(len(u)) < p
    nv = rng.integers(0, n, size=int(rew.sum()))
    bad = nv == u[rew]
    while bad.any():
        nv[bad] = rng.integers(0, n, size=int(bad.sum()))
        bad = nv == u[rew]
    v = v.copy()
    v[rew] = nv
    return from_edges(n, u, v, name=f"ws{n}_k{k}")


# --------------------------------------------------------------------------- weights / subsets
def lognormal_edge_weights(m: int, mu=0.0, sigma=1.0, seed: int = 5) -> np.ndarray:
    return np.random.default_rng(seed).lognormal(mu, sigma, size=m).astype(np.float32)


def uniform_edge_weights(m: int, lo=0.5, hi=2.0, seed: int = 6) -> np.ndarray:
    return np.random.default_rng(seed).uniform(lo, hi, size=m).astype(np.float32)


def random_edge_subset(m: int, fraction: float = 0.01, seed: int = 7) -> np.ndarray:
    """Sorted edge ids of a seeded Bernoulli(fraction) subset."""
    return np.nonzero(np.random.default_rng(seed).random(m) < fraction)[0].astype(np.int64)


def ws_batch(G: int = 512, n_lo=1000, n_hi=200000, k=10, p=0.1, seed: int = 8):
    """The batched workload: G Watts-Strogatz graphs with n ~ U{n_lo..n_hi}."""
    rng = np.random.default_rng(seed)
    sizes = rng.integers(n_lo, n_hi + 1, size=G)
    return [watts_strogatz(int(s), k, p, seed=seed * 100003 + i) for i, s in enumerate(sizes)]


def concat(graphs) -> tuple[np.ndarray, Graph]:
    """Disjoint union of graphs as one block-diagonal CSR (graph g owns
    vertices voff[g]..voff[g+1]-1), built by offsetting the CSR arrays.
    Returns (voff int64[G+1], union)."""
    voff = np.zeros(len(graphs) + 1, dtype=np.int64)
    voff[1:] = np.cumsum([gg.n for gg in graphs])
    eoff = np.zeros(len(graphs) + 1, dtype=np.int64)
    eoff[1:] = np.cumsum([gg.nnz for gg in graphs])
    row_ptr = np.empty(int(voff[-1]) + 1, dtype=np.int64)
    col = np.empty(int(eoff[-1]), dtype=np.int32)
    weighted = any(gg.weight is not None for gg in graphs)
    weight = np.empty(int(eoff[-1]), dtype=np.float32) if weighted else None
    for gg, v0, e0 in zip(graphs, voff, eoff):
        row_ptr[v0:v0 + gg.n] = gg.row_ptr[:-1] + e0
        col[e0:e0 + gg.nnz] = gg.col + np.int32(v0)
        if weighted:
            weight[e0:e0 + gg.nnz] = 1.0 if gg.weight is None else gg.weight
    row_ptr[-1] = eoff[-1]
    return voff, Graph(n=int(voff[-1]), row_ptr=row_ptr, col=col, weight=weight, name="union")


def random_scores(m: int, n_distinct: int | None = None, seed: int = 9) -> np.ndarray:
    """Non-negative FP32 edge scores for selection tests; with n_distinct the
    values repeat so that ties occur."""
    rng = np.random.default_rng(seed)
    if n_distinct is None:
        return rng.random(m).astype(np.float32)
    vals = np.sort(rng.random(n_distinct).astype(np.float32))
    return vals[rng.integers(0, n_distinct, size=m)]


def planted_partition(n_clusters=3, size=20, p_in=0.6, n_cut=2, seed: int = 10) -> tuple[Graph, np.ndarray]:
    """Dense clusters joined by a few cut edges (the shape of Fig. 1).  Returns
    the graph and a 0/1 flag per edge (edge-id order) marking cut edges."""
    rng = np.random.default_rng(seed)
    us, vs = [], []
    for c in range(n_clusters):
        base = c * size
        iu, iv = np.triu_indices(size, 1)
        sel = rng.random(len(iu)) < p_in
        us.append(base + iu[sel])
        vs.append(base + iv[sel])
        # a Hamiltonian path keeps each cluster connected
        us.append(base + np.arange(size - 1))
        vs.append(base + np.arange(1, size))
    for c in range(n_clusters):
        d = (c + 1) % n_clusters
        for _ in range(n_cut):
            us.append(np.array([c * size + rng.integers(size)]))
            vs.append(np.array([d * size + rng.integers(size)]))
    g = from_edges(n_clusters * size, np.concatenate(us), np.concatenate(vs), name="planted")
    eu, ev = g.edges_upper()
    cut = (eu // size) != (ev // size)
    return g, cut.astype(np.uint8)
