"""Pins for the oracle's multilevel framework (Sec. 5, Eq. (P), Alg. 6).

  * seeds: the greedy traversal is checked through the condition that
    determines its result uniquely (vertex i is a seed iff its weight to the
    seeds that precede it in the visiting order is <= Q D_i);
  * P: the argmax of Eq. (P) on a dense matrix of delta = 1/rho;
  * Galerkin: P^T L_f P computed densely equals the Laplacian of the coarse CSR;
  * uncoarsening: brute force over fine edges;
  * the level-span ratio vectors of the paper's 6-level example (golden), and
    the reading for an odd remainder;
  * the stall guard on disjoint triangles, which keep 2/3 of their vertices;
  * Alg. 6 on two levels rebuilt from its steps (Philox streams of the way
    down and up, ratio order);
  * the fitted keep fraction is the smallest 2^-20 grid point reaching K.
"""
import json
import os

import numpy as np
import pytest

import oracle
from paper_1601_05527_gb300 import graphgen

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def weighted_ba(n, m, seed):
    g = graphgen.barabasi_albert(n, m, seed=seed)
    return graphgen.with_edge_weights(g, graphgen.lognormal_edge_weights(g.m, seed=seed + 1))


def dense_W(g):
    W = np.zeros((g.n, g.n))
    rows = np.repeat(np.arange(g.n), g.degrees())
    W[rows, g.col] = 1.0 if g.weight is None else g.weight.astype(np.float64)
    return W


@pytest.mark.parametrize("weighted", [True, False])
@pytest.mark.parametrize("Q", [0.3, 0.5, 0.8])
def test_seeds_satisfy_the_greedy_condition(Q, weighted):
    # unit weights make coupling == Q D_i occur, where "<=" decides
    g = weighted_ba(300, 3, 1) if weighted else graphgen.barabasi_albert(300, 4, seed=1)
    w = g.weight.astype(np.float64) if weighted else None
    seed = oracle.create_seeds(g.row_ptr, g.col, w, Q)
    W = dense_W(g)
    D = W.sum(1)
    order = np.lexsort((np.arange(g.n), -D))            # decreasing D, ties by id
    pos = np.empty(g.n, dtype=np.int64)
    pos[order] = np.arange(g.n)
    earlier_seed = (seed[None, :] == 1) & (pos[None, :] < pos[:, None])
    coupling = (W * earlier_seed).sum(1)
    np.testing.assert_array_equal(seed == 1, coupling <= Q * D)
    F = seed == 0
    assert np.all((W[F][:, seed == 1]).sum(1) > Q * D[F])


def test_seeds_skip_isolated_vertices():
    g = graphgen.from_edges(6, [0, 1], [1, 2])
    s = oracle.create_seeds(g.row_ptr, g.col, None, 0.5)
    assert np.all(s[3:] == 0)


def test_aggregation_is_eq_P_argmax():
    g = weighted_ba(200, 4, 3)
    w = g.weight.astype(np.float64)
    seed = oracle.create_seeds(g.row_ptr, g.col, w, 0.5)
    rho = graphgen.random_scores(g.m, seed=2).astype(np.float64) + 0.01
    agg, nc = oracle.aggregate(g.row_ptr, g.col, rho, seed)
    assert nc == seed.sum()
    eu, ev = g.edges_upper()
    delta = np.zeros((g.n, g.n))
    delta[eu, ev] = 1.0 / rho
    delta[ev, eu] = 1.0 / rho
    dC = delta * (seed[None, :] == 1)
    frac = dC / np.maximum(dC.sum(1, keepdims=True), 1e-300)
    coarse_id = np.cumsum(seed) - 1
    for i in range(g.n):
        if seed[i]:
            assert agg[i] == coarse_id[i]
        else:
            assert agg[i] == coarse_id[np.argmax(frac[i])]


def test_aggregation_ties_go_to_smaller_seed():
    # F vertex 0 with three seed neighbours at equal distance
    g = graphgen.from_edges(4, [0, 0, 0], [1, 2, 3])
    seed = np.array([0, 1, 1, 1], dtype=np.uint8)
    agg, nc = oracle.aggregate(g.row_ptr, g.col, np.ones(3), seed)
    assert nc == 3 and agg[0] == 0 and list(agg[1:]) == [0, 1, 2]


@pytest.mark.parametrize("seed_", [1, 2, 3])
def test_galerkin_is_PtLP(seed_):
    g = weighted_ba(150, 3, seed_)
    w = g.weight.astype(np.float64)
    is_seed = oracle.create_seeds(g.row_ptr, g.col, w, 0.5)
    rho = oracle.algebraic_distance(g.row_ptr, g.col, w, R=4, k=5, omega=0.5, seed=seed_)
    agg, nc = oracle.aggregate(g.row_ptr, g.col, rho, is_seed)
    rpc, cic, wc, f2c = oracle.galerkin(g.row_ptr, g.col, w, agg, nc)
    W = dense_W(g)
    L = np.diag(W.sum(1)) - W
    P = np.zeros((g.n, nc))
    P[np.arange(g.n)[agg >= 0], agg[agg >= 0]] = 1.0
    Lc_ref = P.T @ L @ P
    Wc = np.zeros((nc, nc))
    Wc[np.repeat(np.arange(nc), np.diff(rpc)), cic] = wc
    np.testing.assert_allclose(np.diag(Wc.sum(1)) - Wc, Lc_ref, rtol=1e-12, atol=1e-12)
    assert np.all(np.diff(rpc) >= 0) and np.all(Wc == Wc.T)
    for r in range(nc):                                    # sorted rows, no self loops
        row = cic[rpc[r]:rpc[r + 1]]
        assert np.all(np.diff(row) > 0) and not np.any(row == r)
    cu, cv = graphgen.Graph(nc, rpc, cic, None).edges_upper()
    eu, ev = g.edges_upper()
    for e in range(g.m):
        I, J = agg[eu[e]], agg[ev[e]]
        if I == J:
            assert f2c[e] == -1
        else:
            assert (cu[f2c[e]], cv[f2c[e]]) == (min(I, J), max(I, J))


def test_uncoarsen_brute_force():
    rng = np.random.default_rng(0)
    f2c = rng.integers(-1, 20, size=500)
    keep_c = (rng.random(20) < 0.5).astype(np.uint8)
    kf = oracle.uncoarsen(f2c, keep_c)
    for e in range(500):
        assert kf[e] == (1 if f2c[e] < 0 else keep_c[f2c[e]])


def test_level_span_segments_match_paper_example():
    gold = json.load(open(os.path.join(GOLDEN, "level_span_segments.json")))
    for seg in ("coarse", "middle", "fine"):
        r = oracle.segment_ratios(gold["levels"], seg, gold["level_span"], gold["value"])
        np.testing.assert_array_equal(r, gold[seg])


def test_hierarchy_and_target_fraction():
    g = weighted_ba(2000, 4, 7)
    w = g.weight.astype(np.float64)
    ml = oracle.Multilevel(g.row_ptr, g.col, w, R=8, k=10, omega=0.5, seed=5, coarsest_n=60)
    L = ml.levels
    assert L >= 3
    sizes = [ml.level_size(l) for l in range(L)]
    assert sizes[0] == (g.n, g.m)
    for l in range(1, L):
        assert sizes[l][0] <= 0.9 * sizes[l - 1][0]
    # nothing sparsified -> every edge kept; ratio 1 everywhere -> every edge kept
    keep, kept, _ = ml.sparsify(-np.ones(L))
    assert kept == g.m and keep.all()
    keep, kept, _ = ml.sparsify(np.ones(L))
    assert kept == g.m
    # coarse-level control to 40% of the edges
    ratios = oracle.segment_ratios(L, "coarse", max(1, L // 3), 1.0)
    keep, kept, r = ml.sparsify(ratios, target_fraction=0.4)
    K = oracle.target_count(g.m, 0.4)
    assert kept == keep.sum() >= K
    if r > 2 ** -20:
        r_below = np.where(ratios >= 0, r - 2 ** -20, -1.0)
        _, kb, _ = ml.sparsify(r_below)
        assert kb < K
    # fine-level control re-computes distances on the sparsified finest graph
    ratios = oracle.segment_ratios(L, "fine", 1, 0.5)
    keep_f, kept_f, _ = ml.sparsify(ratios)
    assert kept_f == keep_f.sum() >= oracle.target_count(g.m, 0.5)
    ml.close()


def test_middle_segment_of_an_odd_remainder():
    """The paper's example has L - level_span even.  Reading for an odd
    remainder: the middle segment starts floor((L - span) / 2) levels from the
    coarsest, i.e. it leans coarse."""
    np.testing.assert_array_equal(oracle.segment_ratios(5, "middle", 2, 0.3), [-1, 0.3, 0.3, -1, -1])
    np.testing.assert_array_equal(oracle.segment_ratios(7, "middle", 2, 0.3), [-1, -1, 0.3, 0.3, -1, -1, -1])


def triangles(T):
    u = np.concatenate([3 * np.arange(T), 3 * np.arange(T), 3 * np.arange(T) + 1])
    v = np.concatenate([3 * np.arange(T) + 1, 3 * np.arange(T) + 2, 3 * np.arange(T) + 2])
    return graphgen.from_edges(3 * T, u, v)


def test_triangles_coarsen_by_two_thirds():
    """In a unit-weight triangle the first vertex is a seed, the second one too
    (its weight to seeds, 1, is <= Q D = 1), the third not (2 > 1): each level
    keeps 2/3 of the vertices, which the stall guard (n_c > 0.9 n_f) accepts."""
    T = 50
    g = triangles(T)
    seeds = oracle.create_seeds(g.row_ptr, g.col, None, Q=0.5)
    assert seeds.reshape(T, 3).tolist() == [[1, 1, 0]] * T
    ml = oracle.Multilevel(g.row_ptr, g.col, None, R=4, k=5, omega=0.5, seed=3, coarsest_n=10)
    assert ml.levels >= 2
    assert ml.level_size(1) == (2 * T, T)          # one coarse edge per triangle
    ml.close()
    # a level of exactly coarsest_n vertices is small enough: the hierarchy stops there
    for cn, more in ((3 * T, False), (3 * T - 1, True)):
        ml = oracle.Multilevel(g.row_ptr, g.col, None, R=4, k=5, omega=0.5, seed=3, coarsest_n=cn)
        assert (ml.levels > 1) == more, cn
        ml.close()


@pytest.mark.parametrize("mode,om", [("local", 0.5), ("global", 0.5), ("local", 0.35)])
def test_two_levels_compose_the_steps_of_alg6(mode, om):
    """A two-level hierarchy against Alg. 6 rebuilt from its steps: distances on
    the way down use Philox stream 2l, the recomputed ones on the way up 2l + 1;
    ratios[0] belongs to the coarsest level."""
    g = weighted_ba(400, 4, 11)
    w = g.weight.astype(np.float64)
    R, k, seed, f = 8, 10, 21, 0.4
    ml = oracle.Multilevel(g.row_ptr, g.col, w, R=R, k=k, omega=om, seed=seed, max_levels=2, coarsest_n=1,
                           mode=mode)
    assert ml.levels == 2
    rho0 = oracle.algebraic_distance(g.row_ptr, g.col, w, R=R, k=k, omega=om, seed=seed, stream=0)
    agg, nc = oracle.aggregate(g.row_ptr, g.col, rho0, oracle.create_seeds(g.row_ptr, g.col, w, Q=0.5))
    rpc, cic, wc, f2c = oracle.galerkin(g.row_ptr, g.col, w, agg, nc)
    assert ml.level_size(1) == (nc, len(cic) // 2)
    # coarsest level only: select on the coarse graph, then uncoarsen
    rho1 = oracle.algebraic_distance(rpc, cic, wc, R=R, k=k, omega=om, seed=seed, stream=2)
    keep_c, _, _ = oracle.sparsify(rpc, cic, rho1, mode, "per_node", f)
    keep, _, _ = ml.sparsify([f, -1.0])
    np.testing.assert_array_equal(keep, oracle.uncoarsen(f2c, keep_c))
    # finest level only: every edge survives the coarse level, distances are recomputed
    rho0_up = oracle.algebraic_distance(g.row_ptr, g.col, w, R=R, k=k, omega=om, seed=seed, stream=1)
    keep_f, _, _ = oracle.sparsify(g.row_ptr, g.col, rho0_up, mode, "per_node", f)
    keep, _, _ = ml.sparsify([-1.0, f])
    np.testing.assert_array_equal(keep, keep_f)
    ml.close()

