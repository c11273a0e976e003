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
