"""The synthetic inputs (no method arithmetic): every generator returns a simple
undirected graph as a symmetric CSR with strictly sorted rows -- the contract
the library's validation, the oracle and the edge numbering rely on -- with
the structure its recipe states, determined by its seed."""
import numpy as np
import pytest

from paper_1601_05527_gb300 import graphgen


def check_csr(g):
    rp, col = g.row_ptr, g.col
    assert rp.dtype == np.int64 and col.dtype == np.int32
    assert rp[0] == 0 and rp[-1] == len(col) and (np.diff(rp) >= 0).all()
    assert len(col) % 2 == 0 and g.m == len(col) // 2
    rows = np.repeat(np.arange(g.n, dtype=np.int64), g.degrees())
    assert ((col >= 0) & (col < g.n)).all()
    assert (col != rows).all()                                   # no self loops
    same_row = rows[1:] == rows[:-1]
    assert (col[1:][same_row] > col[:-1][same_row]).all()        # sorted, no duplicates
    fwd = rows * g.n + col
    rev = col.astype(np.int64) * g.n + rows
    order = np.argsort(fwd)
    pos = np.searchsorted(fwd[order], rev)
    assert (fwd[order][pos] == rev).all()                        # every entry has its mirror
    mirror = order[pos]
    if g.weight is not None:
        assert np.array_equal(g.weight, g.weight[mirror])        # mirrored entries share the weight
        assert (g.weight > 0).all() and np.isfinite(g.weight).all()
    eu, ev = g.edges_upper()
    assert len(eu) == g.m and (eu < ev).all()
    assert (np.diff(eu.astype(np.int64) * g.n + ev) > 0).all()   # edge ids in row-major order


GENERATORS = {
    "grid": lambda s: graphgen.grid2d(7, 9),
    "rmat": lambda s: graphgen.rmat(11, 16, seed=s),
    "ba": lambda s: graphgen.barabasi_albert(3000, 8, seed=s),
    "ws": lambda s: graphgen.watts_strogatz(2000, 10, 0.1, seed=s),
    "planted": lambda s: graphgen.planted_partition(4, 30, 0.3, 3, seed=s)[0],
}


@pytest.mark.parametrize("name", list(GENERATORS))
def test_valid_symmetric_csr_and_seeded(name):
    g = GENERATORS[name](5)
    check_csr(g)
    assert GENERATORS[name](5).digest() == g.digest()
    if name != "grid":
        assert GENERATORS[name](6).digest() != g.digest()


def test_grid_degrees_and_ids():
    r, c = 7, 9
    g = graphgen.grid2d(r, c)
    assert g.n == r * c and g.m == 2 * r * c - r - c
    d = g.degrees().reshape(r, c)
    assert d[0, 0] == d[0, -1] == d[-1, 0] == d[-1, -1] == 2
    assert (d[1:-1, 1:-1] == 4).all() and (d[0, 1:-1] == 3).all() and (d[1:-1, 0] == 3).all()
    i = 3 * c + 4                                                # vertex (3, 4)
    assert g.col[g.row_ptr[i]:g.row_ptr[i + 1]].tolist() == [i - c, i - 1, i + 1, i + c]


def test_rmat_is_heavy_tailed_with_isolated_vertices():
    g = graphgen.rmat(14, 16, seed=2)
    d = g.degrees()
    assert g.n == 1 << 14
    assert (d == 0).mean() > 0.2                                 # ids as generated: many isolated
    assert d.max() > 40 * d[d > 0].mean()                        # hubs
    assert d[:64].mean() > 10 * d.mean()                         # low ids favoured (a = 0.57)


def test_barabasi_albert_min_degree_and_edge_count():
    n, m = 3000, 8
    g = graphgen.barabasi_albert(n, m, seed=3)
    d = g.degrees()
    assert (d[:m + 1] >= m).all()                                # the seed clique
    assert d.min() >= 1
    assert g.m <= m * (m + 1) // 2 + (n - m - 1) * m             # repeated picks collapse
    assert g.m >= 0.9 * m * n
    assert d.max() > 10 * m                                      # preferential attachment


def test_watts_strogatz_keeps_the_ring_edge_count():
    n, k = 2000, 10
    g0 = graphgen.watts_strogatz(n, k, 0.0, seed=4)
    assert g0.m == n * k // 2 and (g0.degrees() == k).all()
    g = graphgen.watts_strogatz(n, k, 0.1, seed=4)
    assert 0.99 * n * k / 2 <= g.m <= n * k / 2                  # rewired duplicates merge


def test_weights_attach_to_both_directions():
    g = graphgen.barabasi_albert(500, 4, seed=9)
    ew = graphgen.lognormal_edge_weights(g.m, seed=9)
    gw = graphgen.with_edge_weights(g, ew)
    check_csr(gw)
    np.testing.assert_array_equal(gw.edge_weights(), ew)
    u = graphgen.uniform_edge_weights(10000, seed=1)
    assert u.min() >= 0.5 and u.max() <= 2.0


def test_concat_is_block_diagonal():
    parts = [graphgen.grid2d(3, 4), graphgen.watts_strogatz(50, 4, 0.2, seed=1), graphgen.rmat(6, 4, seed=1)]
    voff, u = graphgen.concat(parts)
    check_csr(u)
    assert voff.tolist() == [0, 12, 62, 62 + 64] and u.m == sum(p.m for p in parts)
    for gpart, v0, v1 in zip(parts, voff[:-1], voff[1:]):
        rp = u.row_ptr[v0:v1 + 1] - u.row_ptr[v0]
        np.testing.assert_array_equal(rp, gpart.row_ptr)
        np.testing.assert_array_equal(u.col[u.row_ptr[v0]:u.row_ptr[v1]] - v0, gpart.col)


def test_planted_cut_flags_mark_edges_between_clusters():
    g, cut = graphgen.planted_partition(3, 20, 0.6, 2, seed=10)
    eu, ev = g.edges_upper()
    assert np.array_equal(cut.astype(bool), (eu // 20) != (ev // 20))
    assert 1 <= cut.sum() <= 6


def test_scores_and_subsets():
    s = graphgen.random_scores(1000, 7, seed=2)
    assert s.dtype == np.float32 and len(np.unique(s)) <= 7 and (s >= 0).all()
    S = graphgen.random_edge_subset(100000, 0.01, seed=3)
    assert (np.diff(S) > 0).all() and S.min() >= 0 and S.max() < 100000
    assert 800 < len(S) < 1200
