"""Pins of the oracle's Local Degree comparator (Sec. 1.1, Sec. 6): every
node takes the edges to its T(d, e) neighbours of largest degree."""
import numpy as np

import oracle
from paper_1601_05527_gb300 import graphgen


def two_hubs():
    """Centre c = 0 joined to 1..10; vertex k has k - 1 private leaves and an
    edge to a large hub M = 11 (which has 100 further leaves).  At T = 1 every
    k takes its edge to M (the largest degree around it), so an edge (0, k) is
    kept only when 0 itself takes it: its largest-degree neighbour, k = 10."""
    u, v, nxt = [], [], 12
    for k in range(1, 11):
        u += [0, k]
        v += [k, 11]
        for _ in range(k - 1):
            u.append(k)
            v.append(nxt)
            nxt += 1
    for _ in range(100):
        u.append(11)
        v.append(nxt)
        nxt += 1
    return graphgen.from_edges(nxt, np.array(u), np.array(v))


def test_centre_takes_its_largest_degree_neighbour():
    g = two_hubs()
    eu, ev = g.edges_upper()
    keep, kept, e = oracle.sparsify_local_degree(g.row_ptr, g.col, 0.0)
    assert e == 2.0 ** -40                       # the smallest grid point: T(d, e) = 1 for every d here
    centre = {int(b): int(keep[t]) for t, (a_, b) in enumerate(zip(eu, ev)) if a_ == 0}
    assert centre == {k: int(k == 10) for k in range(1, 11)}


def test_fit_is_the_brute_force_union():
    g = graphgen.barabasi_albert(400, 3, seed=2)
    d = np.diff(g.row_ptr)
    eid = oracle.entry_edge_ids(g.row_ptr, g.col)

    def union(e):
        keep = np.zeros(g.m, np.uint8)
        for i in range(g.n):
            p0, p1 = g.row_ptr[i], g.row_ptr[i + 1]
            order = sorted(range(p0, p1), key=lambda p: (-d[g.col[p]], p))
            for p in order[:oracle.degree_target(int(d[i]), e)]:
                keep[eid[p]] = 1
        return keep

    for f in (0.0, 0.4, 0.75, 1.0):
        keep, kept, e = oracle.sparsify_local_degree(g.row_ptr, g.col, f)
        K = oracle.target_count(g.m, f)
        np.testing.assert_array_equal(keep, union(e))
        assert kept >= K
        if e > 2.0 ** -40:
            assert union(e - 2.0 ** -40).sum() < K


def equal_degree_ring():
    """Centre 0 joined to 1..10; every k also has an edge to a hub H = 11 and a
    private leaf, so all of the centre's neighbours have degree 3.  H has five
    more leaves (degree 15), so at T = 1 every k takes its edge to H and the
    centre's edges are kept only by the centre's own choice."""
    u, v, nxt = [], [], 12
    for k in range(1, 11):
        u += [0, k, k]
        v += [k, 11, nxt]
        nxt += 1
    for _ in range(5):
        u.append(11)
        v.append(nxt)
        nxt += 1
    return graphgen.from_edges(nxt, np.array(u), np.array(v))


def test_equal_degrees_go_to_the_smaller_position():
    """Reading 14: among neighbours of equal degree the one earlier in the row
    (the smaller id) ranks first, so at T = 1 the centre keeps its edge to 1."""
    g = equal_degree_ring()
    d = np.diff(g.row_ptr)
    assert set(int(d[k]) for k in range(1, 11)) == {3} and d[0] == 10 and d[11] == 15
    eu, ev = g.edges_upper()
    keep, kept, e = oracle.sparsify_local_degree(g.row_ptr, g.col, 0.0)
    assert e == 2.0 ** -40
    centre = {int(b): int(keep[t]) for t, (a_, b) in enumerate(zip(eu, ev)) if a_ == 0}
    assert centre == {k: int(k == 1) for k in range(1, 11)}
    hub = {int(a_): int(keep[t]) for t, (a_, b) in enumerate(zip(eu, ev)) if b == 11}
    assert hub == {k: 1 for k in range(1, 11)}      # every k takes its largest-degree neighbour


def test_every_active_vertex_keeps_an_edge_and_e_one_keeps_all():
    g = graphgen.rmat(9, 8, seed=6)
    d = np.diff(g.row_ptr)
    eid = oracle.entry_edge_ids(g.row_ptr, g.col)
    for f in (0.0, 0.2, 0.5):
        keep, _, _ = oracle.sparsify_local_degree(g.row_ptr, g.col, f)
        for i in np.flatnonzero(d > 0):
            assert keep[eid[g.row_ptr[i]:g.row_ptr[i + 1]]].any()
    keep, kept, e = oracle.sparsify_local_degree(g.row_ptr, g.col, 1.0)
    assert kept == g.m and keep.all()
