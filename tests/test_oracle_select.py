"""Pins for the oracle's ranking and sampling (Sec. 4, Alg. 2; whole-graph ranking).

The kept sets are checked against characterisations that determine them
uniquely, evaluated by brute force (pairwise comparisons, no sorting):
  * whole graph: exactly K edges, and every kept edge precedes every dropped
    edge in the mode's order (score, then edge id);
  * per node (Alg. 2): every node's first T(d_i, e) incident edges are kept,
    and every kept edge is among the first T of at least one endpoint;
  * T(d, e) of "top d_i^e" at the boundary exponents and at exact powers;
  * the fraction -> e bisection returns the smallest 2^-40 grid point that
    reaches K edges.
"""
import numpy as np
import pytest

import oracle
from paper_1601_05527_gb300 import graphgen


def precedes(s_a, e_a, s_b, e_b, mode):
    if mode == "local":
        return (s_a < s_b) | ((s_a == s_b) & (e_a < e_b))
    return (s_a > s_b) | ((s_a == s_b) & (e_a < e_b))


@pytest.mark.parametrize("mode", ["local", "global"])
@pytest.mark.parametrize("m,n_distinct,K", [(50, None, 20), (200, 7, 63), (300, 3, 150), (64, 64, 0), (40, 5, 40)])
def test_whole_graph_keeps_the_first_K(mode, m, n_distinct, K):
    s = graphgen.random_scores(m, n_distinct, seed=m + K).astype(np.float64)
    keep = oracle.select_whole_graph(s, mode, K)
    assert keep.sum() == K
    ids = np.arange(m)
    a, b = np.nonzero(keep)[0], np.nonzero(keep == 0)[0]
    if len(a) and len(b):
        assert np.all(precedes(s[a][:, None], ids[a][:, None], s[b][None, :], ids[b][None, :], mode))


def test_local_and_global_are_complements_on_distinct_scores():
    m = 101
    s = graphgen.random_scores(m, seed=3).astype(np.float64)
    assert len(np.unique(s)) == m
    for K in (0, 1, 30, 100, 101):
        np.testing.assert_array_equal(oracle.select_whole_graph(s, "local", K),
                                      1 - oracle.select_whole_graph(s, "global", m - K))


def test_degree_target_values():
    assert oracle.degree_target(0, 0.5) == 0
    for d in (1, 2, 7, 64, 1000):
        assert oracle.degree_target(d, 0.0) == 1          # at least one edge per node
        assert oracle.degree_target(d, 1.0) == d          # e = 1 keeps every edge
    assert oracle.degree_target(4, 0.5) == 2
    assert oracle.degree_target(100, 0.5) == 10           # exact power: no round-up
    assert oracle.degree_target(1000, 1.0 / 3.0) == 10    # pow rounds just below 10
    assert oracle.degree_target(10, 0.5) == 4             # ceil(3.162...)
    assert oracle.degree_target(50, 0.3) == 4             # ceil(3.233...)
    prev = 0
    for e in np.linspace(0, 1, 101):
        t = oracle.degree_target(37, float(e))
        assert t >= prev
        prev = t


def incident_ranks(g, score, mode):
    """rank[p] of CSR entry p inside its row = number of incident edges that precede it."""
    eid = oracle.entry_edge_ids(g.row_ptr, g.col)
    rank = np.zeros(g.nnz, dtype=np.int64)
    for i in range(g.n):
        lo, hi = g.row_ptr[i], g.row_ptr[i + 1]
        e = eid[lo:hi]
        s = score[e]
        P = precedes(s[None, :], e[None, :], s[:, None], e[:, None], mode)    # P[a, b]: b precedes a
        rank[lo:hi] = P.sum(1)
    return eid, rank


def check_per_node(g, score, mode, e, keep):
    eid, rank = incident_ranks(g, score, mode)
    rows = np.repeat(np.arange(g.n), g.degrees())
    T = np.array([oracle.degree_target(int(d), e) for d in g.degrees()])
    in_top = rank < T[rows]
    assert np.all(keep[eid[in_top]] == 1)                      # every node's top T kept
    covered = np.zeros(g.m, dtype=bool)
    covered[eid[in_top]] = True
    assert np.all(covered[keep == 1])                          # nothing else kept
    act = g.degrees() > 0
    kept_deg = np.bincount(rows, weights=keep[eid], minlength=g.n)
    assert np.all(kept_deg[act] >= 1)                          # >= 1 edge per node


@pytest.mark.parametrize("mode", ["local", "global"])
@pytest.mark.parametrize("e", [0.0, 0.3, 0.55, 0.9, 1.0])
def test_per_node_union_of_tops(mode, e):
    g = graphgen.barabasi_albert(120, 4, seed=2)
    s = graphgen.random_scores(g.m, 25, seed=5).astype(np.float64)   # ties included
    keep, c = oracle.select_per_node(g.row_ptr, g.col, s, mode, e)
    assert c == keep.sum()
    check_per_node(g, s, mode, e, keep)
    if e == 1.0:
        assert c == g.m


@pytest.mark.parametrize("mode", ["local", "global"])
@pytest.mark.parametrize("fraction", [0.3, 0.5, 0.77, 1.0])
def test_fraction_bisection_is_minimal(mode, fraction):
    g = graphgen.rmat(8, 8, seed=3)
    s = graphgen.random_scores(g.m, seed=4).astype(np.float64)
    keep, kept, e = oracle.sparsify(g.row_ptr, g.col, s, mode, "per_node", fraction)
    K = oracle.target_count(g.m, fraction)
    assert K == int(np.floor(fraction * g.m + 0.5))
    assert kept == keep.sum() >= K
    assert e * 2 ** 40 == np.round(e * 2 ** 40)                  # on the 2^-40 grid
    if e > 2 ** -40:
        _, below = oracle.select_per_node(g.row_ptr, g.col, s, mode, e - 2 ** -40)
        assert below < K
    check_per_node(g, s, mode, e, keep)


@pytest.mark.parametrize("mode", ["local", "global"])
def test_whole_graph_scope_fraction(mode):
    g = graphgen.grid2d(8, 8)
    s = graphgen.random_scores(g.m, 9, seed=1).astype(np.float64)
    keep, kept, e = oracle.sparsify(g.row_ptr, g.col, s, mode, "whole_graph", 0.5)
    assert kept == keep.sum() == oracle.target_count(g.m, 0.5) == g.m // 2
    assert e == -1.0
    np.testing.assert_array_equal(keep, oracle.select_whole_graph(s, mode, kept))


def test_strong_and_weak_selection_on_planted_clusters():
    # Fig. 1 (b)/(c): keeping delta-strong edges drops the cuts, keeping delta-weak keeps them
    g, cut = graphgen.planted_partition(3, 20, 0.6, 2, seed=1)
    rho = oracle.algebraic_distance(g.row_ptr, g.col, None, R=16, k=20, omega=0.5, seed=1)
    K = int(cut.sum())
    assert np.all(oracle.select_whole_graph(rho, "global", K) == cut)
    assert np.all(oracle.select_whole_graph(rho, "local", g.m - K) == 1 - cut)


def test_target_count_is_the_nearest_integer():
    """K = floor(f m + 1/2): the integer nearest to f m, halves rounding up."""
    cases = [(10, 0.25, 3), (10, 0.24, 2), (10, 0.26, 3), (7, 0.5, 4), (3, 1 / 3, 1), (100, 0.304, 30),
             (100, 0.306, 31), (0, 0.5, 0), (57, 0.0, 0), (57, 1.0, 57)]
    for m, f, K in cases:
        assert oracle.target_count(m, f) == K, (m, f)

