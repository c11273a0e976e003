"""The paper's quality measures (Sec. 2) pinned by closed forms and library
routines, then the synthetic sanity comparison of the selection methods
(Sec. 6): keeping delta-strong edges preserves the clustering coefficient,
keeping delta-weak edges destroys it, the binned mixture lands in between,
and Local Degree preserves the degree ranking.  Distances and selections come
from the FP64 oracle with the paper's parameters (R = 10, k = 40)."""
import json
import os

import numpy as np
import pytest

import oracle
from paper_1601_05527_gb300 import graphgen
from quality import average_ranks, clustering_coefficient, kept_graph, local_clustering, spearman

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def g_of(n, pairs):
    u, v = zip(*pairs)
    return graphgen.from_edges(n, np.array(u), np.array(v))


def test_clustering_closed_forms():
    assert clustering_coefficient(g_of(3, [(0, 1), (1, 2), (0, 2)])) == 1.0            # triangle
    assert clustering_coefficient(g_of(6, [(0, k) for k in range(1, 6)])) == 0.0      # star: V' = {centre}
    k5 = [(i, j) for i in range(5) for j in range(i + 1, 5)]
    assert clustering_coefficient(g_of(5, k5)) == 1.0
    assert clustering_coefficient(g_of(4, [(0, 1), (1, 2), (2, 3), (0, 3)])) == 0.0   # 4-cycle
    paw = g_of(4, [(0, 1), (0, 2), (1, 2), (0, 3)])                                   # triangle + pendant
    c = local_clustering(paw)
    assert c[0] == pytest.approx(1 / 3) and c[1] == c[2] == 1.0 and np.isnan(c[3])
    assert clustering_coefficient(paw) == pytest.approx(7 / 9)


def test_clustering_matches_networkx():
    nx = pytest.importorskip("networkx")
    g = graphgen.watts_strogatz(300, 6, 0.2, seed=1)
    G = nx.Graph()
    G.add_nodes_from(range(g.n))
    G.add_edges_from(zip(*g.edges_upper()))
    ref = nx.clustering(G)
    c = local_clustering(g)
    d = g.degrees()
    for i in range(g.n):
        if d[i] > 1:
            assert c[i] == pytest.approx(ref[i], abs=1e-12)


def test_spearman_closed_forms():
    x = np.arange(10.0)
    assert spearman(x, x) == 1.0 and spearman(x, -x) == -1.0
    # ties share the mean rank: y ranks 1, 2, 3.5, 5, 3.5; sum p^2 = 3.5
    assert average_ranks([5, 6, 7, 8, 7]).tolist() == [1, 2, 3.5, 5, 3.5]
    assert spearman([1, 2, 3, 4, 5], [5, 6, 7, 8, 7]) == pytest.approx(1 - 6 * 3.5 / (5 * 24))


def test_spearman_matches_scipy_on_distinct_values():
    stats = pytest.importorskip("scipy.stats")
    rng = np.random.default_rng(3)
    x = rng.random(200)
    y = x + 0.5 * rng.random(200)
    assert spearman(x, y) == pytest.approx(stats.spearmanr(x, y)[0], abs=1e-12)


def sparsified(g, method, fraction, rho):
    if method in ("local", "global"):
        return oracle.sparsify(g.row_ptr, g.col, rho, method, "per_node", fraction)[0]
    if method == "binned":
        return oracle.sparsify_binned(g.row_ptr, g.col, rho, 5, fraction)[0]
    return oracle.sparsify_local_degree(g.row_ptr, g.col, fraction)[0]


GRAPHS = {
    "small_world": lambda: graphgen.watts_strogatz(2000, 10, 0.1, seed=4),
    "planted": lambda: graphgen.planted_partition(20, 50, 0.3, 40, seed=3)[0],
}


@pytest.mark.parametrize("name", list(GRAPHS))
def test_methods_against_the_papers_observations(name):
    par = json.load(open(os.path.join(GOLDEN, "paper_parameters.json")))
    g = GRAPHS[name]()
    rho = oracle.algebraic_distance(g.row_ptr, g.col, None, R=par["R"], k=par["k"], omega=1 - par["alpha"], seed=1)
    C0, d0 = clustering_coefficient(g), g.degrees()
    cc, deg = {}, {}
    for method in ("local", "global", "binned", "ld"):
        s = kept_graph(g, sparsified(g, method, 0.3, rho))
        cc[method] = clustering_coefficient(s) / C0
        deg[method] = spearman(d0, s.degrees())
    # delta-strong keeps the local (triangle-rich) structure, delta-weak loses it
    assert cc["local"] > 0.5 and cc["global"] < 0.2
    # the mixture lies between the two
    assert cc["global"] <= cc["binned"] <= cc["local"]
    # Local Degree keeps the hubs, so the degree ranking survives best
    assert deg["ld"] > max(deg["local"], deg["global"], deg["binned"]) + 0.2
