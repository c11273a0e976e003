"""GPU parity of ranking and sampling (Sec. 4, Alg. 2) and of batched graphs.

Selection is integer work: given identical FP32 scores (seeded synthetic
arrays with ties), the kept edge sets must equal the oracle's bit for bit,
and so must the fitted exponent e.  End to end (GPU distances vs FP64 oracle
distances) the selected sets are compared by Jaccard index."""
import numpy as np
import pytest

import oracle
from paper_1601_05527_gb300 import graphgen
from gpu_util import RHO_TOL, assert_rho_close, entry_weights_f64, jaccard, lib, rho_error

pytestmark = pytest.mark.gpu

SEL_GRAPHS = {
    "rmat12": lambda: graphgen.rmat(12, 16, seed=3),
    "ba2000": lambda: graphgen.barabasi_albert(2000, 6, seed=2),
    "grid32": lambda: graphgen.grid2d(32, 32),
    "rmat14": lambda: graphgen.rmat(14, 16, seed=5),
    "hubs": lambda: hub_graph(),                           # rows of degree 4500..9000 (the large CTA sort)
}


def hub_graph(n=30000, seed=6):
    """Sparse random graph plus four hubs of degree 4500..9000."""
    rng = np.random.default_rng(seed)
    u = [rng.integers(0, n, 60000)]
    v = [rng.integers(0, n, 60000)]
    for h, d in zip(range(4), (4500, 6000, 7500, 9000)):
        u.append(np.full(d, h))
        v.append(rng.choice(np.arange(4, n), d, replace=False))
    return graphgen.from_edges(n, np.concatenate(u), np.concatenate(v))


def gpu_select(g, scores, fraction, mode, scope):
    L = lib()
    h = L.ad_graph_create(g.n, g.row_ptr, g.col, g.weight)
    try:
        keep = np.zeros(g.m, np.uint8)
        kept, e = L.ad_sparsify_scores(h, scores, fraction, mode, scope, keep)
        return keep, kept, e
    finally:
        L.ad_graph_destroy(h)


@pytest.mark.parametrize("name", list(SEL_GRAPHS))
@pytest.mark.parametrize("mode", ["local", "global"])
@pytest.mark.parametrize("ties", [None, 40])
def test_whole_graph_bit_exact(name, mode, ties):
    g = SEL_GRAPHS[name]()
    s = graphgen.random_scores(g.m, ties, seed=11)
    for f in (0.0, 0.25, 0.5, 0.999, 1.0):
        keep, kept, e = gpu_select(g, s, f, mode, "whole_graph")
        ref, rk, _ = oracle.sparsify(g.row_ptr, g.col, s.astype(np.float64), mode, "whole_graph", f)
        assert kept == rk and e == -1.0
        np.testing.assert_array_equal(keep, ref)


@pytest.mark.parametrize("name", list(SEL_GRAPHS))
@pytest.mark.parametrize("mode", ["local", "global"])
@pytest.mark.parametrize("ties", [None, 40])
def test_per_node_fit_bit_exact(name, mode, ties):
    g = SEL_GRAPHS[name]()
    s = graphgen.random_scores(g.m, ties, seed=12)
    for f in (0.3, 0.6, 1.0):
        keep, kept, e = gpu_select(g, s, f, mode, "per_node")
        ref, rk, re_ = oracle.sparsify(g.row_ptr, g.col, s.astype(np.float64), mode, "per_node", f)
        assert e == re_ and kept == rk
        np.testing.assert_array_equal(keep, ref)


@pytest.mark.parametrize("mode", ["local", "global"])
@pytest.mark.parametrize("e", [0.0, 0.2, 0.5, 0.77, 1.0])
def test_per_node_at_exponent_bit_exact(mode, e):
    L = lib()
    g = graphgen.rmat(13, 16, seed=9)
    s = graphgen.random_scores(g.m, 100, seed=13)
    h = L.ad_graph_create(g.n, g.row_ptr, g.col, None)
    keep = np.zeros(g.m, np.uint8)
    kept = L.ad_select_per_node(h, s, e, mode, keep)
    L.ad_graph_destroy(h)
    ref, rk = oracle.select_per_node(g.row_ptr, g.col, s.astype(np.float64), mode, e)
    assert kept == rk
    np.testing.assert_array_equal(keep, ref)


def boundary_graph(seed=8):
    """Rows of degree 8, 9, 16, 17, 32, 33, 512, 513, 1024, 4095, 4096, 4097,
    12288 and 12289 -- the edges of the per-row ranking classes (lane-group
    counting by 8, 16 and 32 lanes, warp sort, CTA sorts in shared memory of
    two sizes, radix sort of whole rows) -- over a sparse random background
    that avoids them."""
    rng = np.random.default_rng(seed)
    degs = (8, 9, 16, 17, 32, 33, 512, 513, 1024, 4095, 4096, 4097, 12288, 12289)
    H, n = len(degs), 20000
    u = [rng.integers(H, n, 30000)]
    v = [rng.integers(H, n, 30000)]
    for h, d in enumerate(degs):
        u.append(np.full(d, h))
        v.append(rng.choice(np.arange(H, n), d, replace=False))
    return graphgen.from_edges(n, np.concatenate(u), np.concatenate(v)), degs


@pytest.mark.parametrize("mode", ["local", "global"])
@pytest.mark.parametrize("ties", [None, 3, 1])
def test_rank_class_boundaries_bit_exact(mode, ties):
    """Per-node selection at fixed exponents on rows at every class edge; with
    one distinct score every row is a single tie run (each radix pass finds one
    digit and is skipped), with three the runs span many warps."""
    g, degs = boundary_graph()
    assert tuple(int(x) for x in np.diff(g.row_ptr)[:len(degs)]) == degs
    s = np.full(g.m, 0.5, np.float32) if ties == 1 else graphgen.random_scores(g.m, ties, seed=21)
    L = lib()
    h = L.ad_graph_create(g.n, g.row_ptr, g.col, None)
    try:
        for e in (0.3, 0.6, 0.8, 0.95):
            keep = np.zeros(g.m, np.uint8)
            kept = L.ad_select_per_node(h, s, e, mode, keep)
            ref, rk = oracle.select_per_node(g.row_ptr, g.col, s.astype(np.float64), mode, e)
            assert kept == rk, (e, kept, rk)
            np.testing.assert_array_equal(keep, ref)
    finally:
        L.ad_graph_destroy(h)


def test_invalid_scores_rejected():
    L = lib()
    g = graphgen.grid2d(5, 5)
    h = L.ad_graph_create(g.n, g.row_ptr, g.col, None)
    s = np.ones(g.m, np.float32)
    s[3] = -1.0
    with pytest.raises(L.ADError):
        L.ad_sparsify_scores(h, s, 0.5, "local", "whole_graph", np.zeros(g.m, np.uint8))
    with pytest.raises(L.ADError) as ei:
        L.ad_sparsify(h, 0.5, "local", "whole_graph", np.zeros(g.m, np.uint8))   # no distances yet
    assert ei.value.status == 9
    L.ad_graph_destroy(h)


@pytest.mark.parametrize("scope,fraction", [("whole_graph", 0.5), ("per_node", 0.3)])
@pytest.mark.parametrize("mode", ["local", "global"])
def test_end_to_end_selection_jaccard(scope, fraction, mode):
    L = lib()
    g = graphgen.grid2d(64, 64) if scope == "whole_graph" else graphgen.rmat(12, 16, seed=3)
    R = 8 if scope == "whole_graph" else 32
    h = L.ad_graph_create(g.n, g.row_ptr, g.col, None)
    rho = np.zeros(g.m, np.float32)
    L.ad_algebraic_distance(h, R, 20, 0.5, 1, 0, "fp32", 0, rho)
    keep = np.zeros(g.m, np.uint8)
    kept, e = L.ad_sparsify(h, fraction, mode, scope, keep)
    L.ad_graph_destroy(h)
    ref_rho = oracle.algebraic_distance(g.row_ptr, g.col, None, R=R, k=20, omega=0.5, seed=1)
    assert_rho_close(rho, ref_rho)
    ref, rk, re_ = oracle.sparsify(g.row_ptr, g.col, ref_rho, mode, scope, fraction)
    assert jaccard(keep, ref) >= 0.999
    # given the GPU's own FP32 distances the selection is exact
    ref32, rk32, re32 = oracle.sparsify(g.row_ptr, g.col, rho.astype(np.float64), mode, scope, fraction)
    np.testing.assert_array_equal(keep, ref32)
    assert kept == rk32 and e == re32


def make_batch(sizes, seed=0):
    graphs = [graphgen.watts_strogatz(int(n), 10, 0.1, seed=seed + i) for i, n in enumerate(sizes)]
    graphs.append(graphgen.rmat(9, 8, seed=seed + 99))
    voff = np.zeros(len(graphs) + 1, np.int64)
    voff[1:] = np.cumsum([gg.n for gg in graphs])
    u, v = [], []
    for gg, off in zip(graphs, voff):
        a, b = gg.edges_upper()
        u.append(a.astype(np.int64) + off)
        v.append(b.astype(np.int64) + off)
    big = graphgen.from_edges(int(voff[-1]), np.concatenate(u), np.concatenate(v))
    return graphs, voff, big


@pytest.mark.parametrize("storage", ["fp32", "bf16"])
def test_batched_graphs_match_each_graph_alone(storage):
    L = lib()
    graphs, voff, big = make_batch([1000, 2345, 1500, 5000, 1200], seed=4)
    h = L.ad_graph_create_batched(voff, big.n, big.row_ptr, big.col, None)
    eoff = L.ad_graph_edge_offsets(h)
    rho = np.zeros(big.m, np.float32)
    L.ad_algebraic_distance(h, 16, 15, 0.5, 7, 0, storage, 0, rho)
    for k, gg in enumerate(graphs):
        single = L.ad_graph_create(gg.n, gg.row_ptr, gg.col, None)
        r1 = np.zeros(gg.m, np.float32)
        L.ad_algebraic_distance(single, 16, 15, 0.5, 7, 0, storage, 0, r1)
        L.ad_graph_destroy(single)
        part = rho[eoff[k]:eoff[k + 1]]
        if storage == "fp32":
            assert_rho_close(part, oracle.algebraic_distance(gg.row_ptr, gg.col, None, R=16, k=15, omega=0.5, seed=7))
        # same kernels; the streaming sweep cuts rows at other places in the batch than
        # alone, so the two differ only in the order of FP32 additions (and, with 16-bit
        # storage, in the roundings that order can flip)
        assert rho_error(part, r1.astype(np.float64)) <= (RHO_TOL if storage == "fp32" else 0.05)
    # per-graph sparsification targets on identical scores
    s = graphgen.random_scores(big.m, 30, seed=5)
    for scope in ("whole_graph", "per_node"):
        keep = np.zeros(big.m, np.uint8)
        L.ad_sparsify_scores(h, s, 0.25, "global", scope, keep)
        for k, gg in enumerate(graphs):
            ref, _, _ = oracle.sparsify(gg.row_ptr, gg.col, s[eoff[k]:eoff[k + 1]].astype(np.float64), "global",
                                        scope, 0.25)
            np.testing.assert_array_equal(keep[eoff[k]:eoff[k + 1]], ref)
    L.ad_graph_destroy(h)


def test_full_size_rmat20_selection_bit_exact():
    """Selection at the benchmark's size (R-MAT scale 20, 15.7M edges) on one
    seeded score array with ties: 30% per node, local and global."""
    g = graphgen.rmat(20, 16, seed=2)
    s = graphgen.random_scores(g.m, 1 << 16, seed=21)
    L = lib()
    h = L.ad_graph_create(g.n, g.row_ptr, g.col, None)
    for mode in ("local", "global"):
        keep = np.zeros(g.m, np.uint8)
        kept, e = L.ad_sparsify_scores(h, s, 0.3, mode, "per_node", keep)
        ref, rk, re_ = oracle.sparsify(g.row_ptr, g.col, s.astype(np.float64), mode, "per_node", 0.3)
        assert e == re_ and kept == rk
        np.testing.assert_array_equal(keep, ref)
    keep = np.zeros(g.m, np.uint8)
    kept, _ = L.ad_sparsify_scores(h, s, 0.3, "local", "whole_graph", keep)
    np.testing.assert_array_equal(keep, oracle.select_whole_graph(s.astype(np.float64), "local", kept))
    L.ad_graph_destroy(h)


def test_cached_ranks_follow_the_distances():
    """Ranks of the handle's own distances are kept between calls; they must
    be rebuilt after the distances change and never be reused for user
    scores (Alg. 2 on whatever scores the call names)."""
    L = lib()
    g = graphgen.rmat(13, 16, seed=8)
    h = L.ad_graph_create(g.n, g.row_ptr, g.col, None)
    rho = np.zeros(g.m, np.float32)
    keep = np.zeros(g.m, np.uint8)

    def check_own(mode):
        kept, e = L.ad_sparsify(h, 0.3, mode, "per_node", keep)
        ref, rk, re_ = oracle.sparsify(g.row_ptr, g.col, rho.astype(np.float64), mode, "per_node", 0.3)
        assert e == re_ and kept == rk
        np.testing.assert_array_equal(keep, ref)

    L.ad_algebraic_distance(h, 16, 10, 0.5, 1, 0, "fp32", 0, rho)
    for mode in ("local", "global", "local"):
        check_own(mode)
    s = graphgen.random_scores(g.m, 25, seed=9)
    kept, e = L.ad_sparsify_scores(h, s, 0.3, "global", "per_node", keep)
    np.testing.assert_array_equal(keep, oracle.sparsify(g.row_ptr, g.col, s.astype(np.float64), "global",
                                                        "per_node", 0.3)[0])
    check_own("global")
    L.ad_algebraic_distance(h, 16, 10, 0.5, 2, 0, "fp32", 0, rho)     # new seed: new distances
    check_own("global")
    check_own("local")
    L.ad_graph_destroy(h)


def test_ranking_follows_every_kind_of_distance_call():
    """The handle's cached ranking of its own distances must follow each new
    distance call -- run directly, replayed from a recorded CUDA graph, as the
    persistent launch, with normalised scores -- and survive other rankings
    in between (Local Degree's, a caller's scores).  Every selection must be
    the oracle's on the distances of the call."""
    import torch
    L = lib()
    g = graphgen.rmat(12, 16, seed=5)
    st = torch.cuda.Stream()
    h = L.ad_graph_create(g.n, g.row_ptr, g.col, None, 0, st)
    rho = np.zeros(g.m, np.float32)
    keep = np.zeros(g.m, np.uint8)

    def check(mode):
        kept, e = L.ad_sparsify(h, 0.3, mode, "per_node", keep)
        ref, rk, re_ = oracle.sparsify(g.row_ptr, g.col, rho.astype(np.float64), mode, "per_node", 0.3)
        assert e == re_ and kept == rk
        np.testing.assert_array_equal(keep, ref)

    calls = [(1, 0), (2, 0), (2, 0), (2, 0), (2, 0), (3, L.AD_DIST_PERSISTENT), (4, L.AD_DIST_NORMALIZE),
             (4, L.AD_DIST_NORMALIZE), (5, 0)]
    try:
        for i, (seed, flags) in enumerate(calls):
            L.ad_algebraic_distance(h, 16, 8, 0.5, seed, 0, "fp32", flags, rho)
            check("local")
            check("global")
            if i == 3:
                L.ad_sparsify_local_degree(h, 0.3, keep)
            if i == 6:
                L.ad_sparsify_scores(h, graphgen.random_scores(g.m, 25, seed=3), 0.3, "local", "per_node", keep)
        kl, kg = np.zeros(g.m, np.uint8), np.zeros(g.m, np.uint8)
        L.ad_algebraic_distance(h, 16, 8, 0.5, 6, 0, "fp32", 0, rho)
        L.ad_sparsify_local_global(h, 0.3, kl, kg)
        for mode, k in (("local", kl), ("global", kg)):
            np.testing.assert_array_equal(k, oracle.sparsify(g.row_ptr, g.col, rho.astype(np.float64), mode,
                                                             "per_node", 0.3)[0])
    finally:
        L.ad_graph_destroy(h)


@pytest.mark.parametrize("name", ["rmat13", "hubs", "batch"])
def test_local_and_global_in_one_call(name):
    """ad_sparsify_local_global (one ranking, one two-problem exponent search)
    against the oracle's per-node selections in each order, on the GPU's own
    distances: kept sets, counts and exponents exact."""
    import torch
    L = lib()
    if name == "batch":
        graphs, voff, big = make_batch([1000, 2345, 1500, 5000, 1200], seed=9)
        h = L.ad_graph_create_batched(voff, big.n, big.row_ptr, big.col, None)
        eoff = L.ad_graph_edge_offsets(h)
        g = big
    else:
        g = graphgen.rmat(13, 16, seed=8) if name == "rmat13" else hub_graph()
        graphs, eoff = [g], [0, g.m]
        h = L.ad_graph_create(g.n, g.row_ptr, g.col, None)
    try:
        rho = np.zeros(g.m, np.float32)
        L.ad_algebraic_distance(h, 16, 10, 0.5, 3, 0, "fp32", 0, rho)
        for f in (0.1, 0.3, 0.75):
            kl = np.zeros(g.m, np.uint8)
            kg = torch.zeros(g.m, dtype=torch.uint8, device="cuda")
            (nl, ng), (el, eg) = L.ad_sparsify_local_global(h, f, kl, kg)
            kg = kg.cpu().numpy()
            tot = [0, 0]
            for k, gg in enumerate(graphs):
                part = rho[eoff[k]:eoff[k + 1]].astype(np.float64)
                for j, (mode, keep) in enumerate((("local", kl), ("global", kg))):
                    ref, rk, re_ = oracle.sparsify(gg.row_ptr, gg.col, part, mode, "per_node", f)
                    np.testing.assert_array_equal(keep[eoff[k]:eoff[k + 1]], ref)
                    tot[j] += rk
                    if k == 0:
                        assert (el, eg)[j] == re_
            assert (nl, ng) == tuple(tot)
    finally:
        L.ad_graph_destroy(h)
