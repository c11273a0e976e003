"""Pins for the oracle's ComputeAlgDist (Alg. 1): JOR sweeps, rescale, distance.

Independent routes used here:
  * dense closed form: x_k = rescale(M^k x_0) with M = (1-omega) I + omega D^-1 W
    (numpy matrix power on the dense matrix; equal to the sweep loop with a
    rescale after every sweep because M commutes with affine maps of a vector);
  * complete graph K_n: every vertex pair is an adjacent twin pair, so for
    every k >= 1 the rescaled vectors are +-(x_0 - min)/(max - min) - const
    and rho_ij depends only on x_0;
  * a single-edge component at omega = 1/2 has y_i = y_j after one sweep;
  * non-adjacent twins keep the ratio of their differences;
  * vertices of degree 0 do not change any distance;
  * relabelling vertices permutes the distances (with permuted x_0).
"""
import numpy as np
import pytest

import oracle
from paper_1601_05527_gb300 import graphgen


def random_graph(n, p, seed, weighted=True, isolated=0):
    rng = np.random.default_rng(seed)
    iu, iv = np.triu_indices(n, 1)
    sel = rng.random(len(iu)) < p
    u, v = iu[sel], iv[sel]
    w = rng.uniform(0.5, 2.0, size=len(u)).astype(np.float32) if weighted else None
    return graphgen.from_edges(n + isolated, u, v, w)


def dense_W(g):
    n = g.n
    W = np.zeros((n, n))
    rows = np.repeat(np.arange(n), g.degrees())
    W[rows, g.col] = 1.0 if g.weight is None else g.weight.astype(np.float64)
    return W


def dense_rho(g, R, k, omega, x0, normalize=False):
    W = dense_W(g)
    D = W.sum(1)
    act = D > 0
    M = np.eye(g.n)
    M[act] = (1 - omega) * np.eye(g.n)[act] + omega * W[act] / D[act, None]
    X = np.linalg.matrix_power(M, k) @ x0
    lo = X[act].min(0)
    hi = X[act].max(0)
    Xs = np.where(hi > lo, (X - lo) / np.where(hi > lo, hi - lo, 1.0) - 0.5, 0.0)
    eu, ev = g.edges_upper()
    rho = np.sqrt(((Xs[eu] - Xs[ev]) ** 2).sum(1))
    if normalize:
        rho = rho * np.sqrt(D[eu] * D[ev])
    return rho, Xs


def wts(g):
    return None if g.weight is None else g.weight.astype(np.float64)


def close(a, b, rtol):
    scale = max(np.sqrt(np.mean(b ** 2)), 1e-300)
    assert np.all(np.abs(a - b) <= rtol * np.maximum(np.abs(b), scale)), np.max(np.abs(a - b) / scale)


CASES = [
    ("er40w", lambda: random_graph(40, 0.15, 1, True, isolated=3)),
    ("er60", lambda: random_graph(60, 0.08, 2, False)),
    ("grid6x7", lambda: graphgen.grid2d(6, 7)),
    ("ba50", lambda: graphgen.barabasi_albert(50, 3, seed=4)),
    ("ws50", lambda: graphgen.watts_strogatz(50, 4, 0.2, seed=5)),
]


@pytest.mark.parametrize("name,make", CASES)
@pytest.mark.parametrize("omega,k", [(0.5, 1), (0.5, 7), (0.3, 12), (0.8, 20)])
def test_matches_dense_matrix_power(name, make, omega, k):
    g = make()
    R = 6
    rho, xf = oracle.algebraic_distance(g.row_ptr, g.col, wts(g), R=R, k=k, omega=omega, seed=17,
                                        return_x=True)
    x0 = oracle.init_vectors(g.n, R, seed=17)
    ref, Xs = dense_rho(g, R, k, omega, x0)
    close(rho, ref, 1e-9)
    act = g.degrees() > 0
    assert np.max(np.abs(xf[act] - Xs[act])) < 1e-9


@pytest.mark.parametrize("name,make", CASES[:3])
def test_normalized_score_matches_dense(name, make):
    g = make()
    rho = oracle.algebraic_distance(g.row_ptr, g.col, wts(g), R=5, k=9, omega=0.5, seed=3, normalize=True)
    ref, _ = dense_rho(g, 5, 9, 0.5, oracle.init_vectors(g.n, 5, seed=3), normalize=True)
    close(rho, ref, 1e-9)


@pytest.mark.parametrize("name,make", CASES)
def test_rescale_once_equals_rescale_every_sweep(name, make):
    g = make()
    a = oracle.algebraic_distance(g.row_ptr, g.col, wts(g), R=4, k=8, omega=0.5, seed=2, rescale="per_sweep")
    b = oracle.algebraic_distance(g.row_ptr, g.col, wts(g), R=4, k=8, omega=0.5, seed=2, rescale="end")
    close(a, b, 1e-9)


def test_constant_vectors_are_fixed_points():
    g = random_graph(30, 0.2, 7)
    x0 = np.tile(np.linspace(-0.4, 0.4, 5), (g.n, 1))     # vector r is the constant c_r
    rho, xf = oracle.algebraic_distance(g.row_ptr, g.col, wts(g), R=5, k=3, omega=0.5, seed=0, x0=x0,
                                        return_x=True)
    # M c = c, so after every sweep hi == lo and the vector rescales to 0
    assert np.all(rho == 0.0)
    assert np.all(xf[g.degrees() > 0] == 0.0)


@pytest.mark.parametrize("n,omega,k", [(6, 0.5, 1), (9, 0.3, 5), (12, 0.7, 20), (5, 0.6, 40)])
def test_complete_graph_closed_form(n, omega, k):
    iu, iv = np.triu_indices(n, 1)
    g = graphgen.from_edges(n, iu, iv)
    R = 7
    x0 = oracle.init_vectors(n, R, seed=23)
    rho = oracle.algebraic_distance(g.row_ptr, g.col, None, R=R, k=k, omega=omega, seed=23)
    span = x0.max(0) - x0.min(0)
    eu, ev = g.edges_upper()
    ref = np.sqrt((((x0[eu] - x0[ev]) / span) ** 2).sum(1))
    close(rho, ref, 1e-10)


def test_single_edge_components():
    # components: three isolated edges plus a triangle
    u = np.array([0, 2, 4, 6, 6, 7])
    v = np.array([1, 3, 5, 7, 8, 8])
    g = graphgen.from_edges(9, u, v)
    rho = oracle.algebraic_distance(g.row_ptr, g.col, None, R=8, k=4, omega=0.5, seed=1)
    eu, ev = g.edges_upper()
    k2 = (eu < 6)
    assert np.all(rho[k2] == 0.0)          # y_i = y_j exactly at omega = 1/2
    assert np.all(rho[~k2] > 0.0)
    # a graph that is one edge: at omega != 1/2 the two values rescale to +-1/2
    g1 = graphgen.from_edges(2, [0], [1])
    r1 = oracle.algebraic_distance(g1.row_ptr, g1.col, None, R=8, k=3, omega=0.3, seed=1)
    assert r1[0] == pytest.approx(np.sqrt(8), rel=1e-14)


def test_nonadjacent_twins_keep_difference_ratios():
    # vertices 0,1 are twins (both adjacent to 2,3,4) and 5,6 are twins (adjacent to 3,4)
    u = np.array([0, 0, 0, 1, 1, 1, 2, 3, 5, 5, 6, 6, 7])
    v = np.array([2, 3, 4, 2, 3, 4, 3, 4, 3, 4, 3, 4, 4])
    g = graphgen.from_edges(8, u, v)
    R, k, omega = 5, 6, 0.4
    x0 = oracle.init_vectors(g.n, R, seed=8)
    _, xf = oracle.algebraic_distance(g.row_ptr, g.col, None, R=R, k=k, omega=omega, seed=8, return_x=True)
    # both differences shrink by (1-omega) per sweep times the same rescale factor
    np.testing.assert_allclose((xf[0] - xf[1]) / (xf[5] - xf[6]), (x0[0] - x0[1]) / (x0[5] - x0[6]), rtol=1e-9)


def test_isolated_vertices_do_not_change_distances():
    g = random_graph(40, 0.1, 3, True)
    g2 = random_graph(40, 0.1, 3, True, isolated=25)
    a = oracle.algebraic_distance(g.row_ptr, g.col, wts(g), R=8, k=10, omega=0.5, seed=4)
    b = oracle.algebraic_distance(g2.row_ptr, g2.col, wts(g2), R=8, k=10, omega=0.5, seed=4)
    np.testing.assert_array_equal(a, b)


def test_relabelling_permutes_distances():
    g = random_graph(35, 0.15, 11, True)
    R = 6
    x0 = oracle.init_vectors(g.n, R, seed=6)
    rho = oracle.algebraic_distance(g.row_ptr, g.col, wts(g), R=R, k=9, omega=0.5, seed=6)
    perm = np.random.default_rng(0).permutation(g.n)      # old id -> new id
    eu, ev = g.edges_upper()
    gp = graphgen.from_edges(g.n, perm[eu], perm[ev], g.edge_weights())
    x0p = np.empty_like(x0)
    x0p[perm] = x0
    rhop = oracle.algebraic_distance(gp.row_ptr, gp.col, wts(gp), R=R, k=9, omega=0.5, seed=0, x0=x0p)
    pu, pv = gp.edges_upper()
    lookup = {(int(a), int(b)): float(r) for a, b, r in zip(pu, pv, rhop)}
    for a, b, r in zip(perm[eu], perm[ev], rho):
        assert lookup[(min(a, b), max(a, b))] == pytest.approx(r, rel=1e-12, abs=1e-15)


def test_cut_edges_of_planted_clusters_are_longest():
    # Fig. 1: edges between dense clusters are long-range (delta-weak)
    g, cut = graphgen.planted_partition(3, 20, 0.6, 2, seed=1)
    rho = oracle.algebraic_distance(g.row_ptr, g.col, None, R=16, k=20, omega=0.5, seed=1)
    assert rho[cut == 1].min() > np.quantile(rho[cut == 0], 0.9)


def test_edge_order_and_counts():
    g = graphgen.grid2d(4, 5)
    assert oracle.count_edges(g.row_ptr, g.col) == 4 * 4 + 3 * 5
    eu, ev = oracle.edge_list(g.row_ptr, g.col)
    gu, gv = g.edges_upper()
    np.testing.assert_array_equal(eu, gu)
    np.testing.assert_array_equal(ev, gv)
    eid = oracle.entry_edge_ids(g.row_ptr, g.col)
    rows = np.repeat(np.arange(g.n), g.degrees())
    # both directions of an edge carry the same id, and the id lists (min, max)
    np.testing.assert_array_equal(np.minimum(rows, g.col), eu[eid])
    np.testing.assert_array_equal(np.maximum(rows, g.col), ev[eid])


def test_weighted_degree():
    g = random_graph(30, 0.3, 2, True)
    np.testing.assert_allclose(oracle.weighted_degree(g.row_ptr, g.col, wts(g)), dense_W(g).sum(1), rtol=1e-15)


def test_thread_count_does_not_change_the_distances():
    """The oracle's row loops may run on several host threads; each row is still
    one thread's sequential sum, so the FP64 distances are bit-identical."""
    g = graphgen.rmat(11, 16, seed=6)
    w = graphgen.uniform_edge_weights(g.m, seed=2)
    gw = graphgen.with_edge_weights(g, w)
    out = []
    for t in (1, max(2, oracle.max_threads())):
        oracle.set_threads(t)
        out.append(oracle.algebraic_distance(gw.row_ptr, gw.col, gw.weight.astype(np.float64), R=8, k=7,
                                             omega=0.45, seed=3))
    oracle.set_threads(oracle.max_threads())
    np.testing.assert_array_equal(out[0], out[1])
    ph = oracle.last_phase_seconds()
    assert set(ph) == {"init", "sweeps", "distance"} and all(v >= 0 for v in ph.values())
