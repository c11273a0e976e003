"""GPU parity of the multilevel framework (Sec. 5, Eq. (P), Alg. 6).

Coarsening components on identical FP32 scores must match the oracle
exactly: seeds, the aggregate map of Eq. (P), the coarse graph of the
Galerkin product (structure exactly, weights to FP32 rounding of the FP64
sums) and the fine-to-coarse edge map.  The whole hierarchy (distances on
the GPU vs FP64 in the oracle) is compared level by level and by the
Jaccard index of the final edge sets."""
import numpy as np
import pytest

import oracle
from paper_1601_05527_gb300 import graphgen
from gpu_util import jaccard, lib

pytestmark = pytest.mark.gpu


def weighted(g, seed):
    return graphgen.with_edge_weights(g, graphgen.lognormal_edge_weights(g.m, seed=seed))


@pytest.mark.parametrize("name,make,Q", [
    ("ba_unit", lambda: graphgen.barabasi_albert(3000, 6, seed=1), 0.5),
    ("rmat_unit", lambda: graphgen.rmat(12, 8, seed=2), 0.5),
    ("ba_lognormal", lambda: weighted(graphgen.barabasi_albert(3000, 8, seed=3), 4), 0.5),
    ("ws_unit_q03", lambda: graphgen.watts_strogatz(4000, 10, 0.1, seed=5), 0.3),
])
def test_coarsening_matches_oracle(name, make, Q):
    L = lib()
    g = make()
    score = graphgen.random_scores(g.m, 50, seed=7) + np.float32(0.01)   # ties included
    h = L.ad_graph_create(g.n, g.row_ptr, g.col, g.weight)
    agg = np.zeros(g.n, np.int32)
    f2c = np.zeros(g.m, np.int64)
    nc, hc = L.ad_coarsen(h, score, Q, agg, f2c)
    rpc, cic, wc = L.ad_graph_export(hc)
    L.ad_graph_destroy(hc)
    L.ad_graph_destroy(h)
    w64 = None if g.weight is None else g.weight.astype(np.float64)
    seeds = oracle.create_seeds(g.row_ptr, g.col, w64, Q)
    ragg, rnc = oracle.aggregate(g.row_ptr, g.col, score.astype(np.float64), seeds)
    assert nc == rnc
    np.testing.assert_array_equal(agg, ragg)
    rrpc, rcic, rwc, rf2c = oracle.galerkin(g.row_ptr, g.col, w64, ragg, rnc)
    np.testing.assert_array_equal(rpc, rrpc)
    np.testing.assert_array_equal(cic, rcic)
    np.testing.assert_array_equal(f2c, rf2c)
    np.testing.assert_array_equal(wc, rwc.astype(np.float32))


def test_hierarchy_and_sparsification_against_oracle():
    L = lib()
    g = weighted(graphgen.barabasi_albert(20000, 8, seed=11), 12)
    w64 = g.weight.astype(np.float64)
    h = L.ad_graph_create(g.n, g.row_ptr, g.col, g.weight)
    ml = L.ad_ml_build(h, R=16, k=20, omega=0.5, seed=5, Q=0.5, coarsest_n=300, mode="local")
    ref = oracle.Multilevel(g.row_ptr, g.col, w64, R=16, k=20, omega=0.5, seed=5, Q=0.5, coarsest_n=300, mode="local")
    Lv = L.ad_ml_levels(ml)
    assert Lv == ref.levels and Lv >= 3
    for l in range(Lv):
        assert L.ad_ml_level_size(ml, l) == ref.level_size(l)
    # nothing sparsified -> all kept
    keep = np.zeros(g.m, np.uint8)
    kept, _ = L.ad_ml_sparsify(ml, -np.ones(Lv), -1.0, keep)
    assert kept == g.m and keep.all()
    # coarse-level control to 40%, fine-level control to 50%
    for seg, tf in (("coarse", 0.4), ("fine", -1.0)):
        ratios = L.ad_ml_segment_ratios(Lv, seg, max(1, Lv // 3), 1.0 if tf >= 0 else 0.5)
        kept, r = L.ad_ml_sparsify(ml, ratios, tf, keep)
        rkeep, rkept, rr = ref.sparsify(ratios, tf)
        assert kept == keep.sum()
        if tf >= 0:
            assert kept >= oracle.target_count(g.m, tf)
            assert r * 2 ** 20 == np.round(r * 2 ** 20)
        assert jaccard(keep, rkeep) >= 0.99, (seg, jaccard(keep, rkeep))
    L.ad_ml_destroy(ml)
    ref.close()
    L.ad_graph_destroy(h)


def test_one_shot_multilevel_call_against_oracle():
    """ad_multilevel (Alg. 6 MLSparsify in one call) on the 20K hierarchy whose
    levels equal the oracle's: coarse-level control to 40%, and a ratio vector
    shorter than the hierarchy (the finer levels are then not sparsified)."""
    L = lib()
    g = weighted(graphgen.barabasi_albert(20000, 8, seed=11), 12)
    w64 = g.weight.astype(np.float64)
    h = L.ad_graph_create(g.n, g.row_ptr, g.col, g.weight)
    ref = oracle.Multilevel(g.row_ptr, g.col, w64, R=16, k=20, omega=0.5, seed=5, Q=0.5, coarsest_n=300, mode="local")
    Lv = ref.levels
    keep = np.zeros(g.m, np.uint8)
    span = max(1, Lv // 3)
    ratios = oracle.segment_ratios(Lv, "coarse", span, 1.0)
    nl = L.ad_multilevel(h, ratios[:span], 0.4, keep, R=16, k=20, omega=0.5, seed=5, Q=0.5, coarsest_n=300,
                         mode="local")
    assert nl == Lv
    rkeep, rkept, _ = ref.sparsify(ratios, 0.4)
    assert keep.sum() >= oracle.target_count(g.m, 0.4)
    assert jaccard(keep, rkeep) >= 0.99
    nl = L.ad_multilevel(h, None, -1.0, keep, R=16, k=20, omega=0.5, seed=5, Q=0.5, coarsest_n=300)
    assert nl == Lv and keep.all()
    ref.close()
    L.ad_graph_destroy(h)


def test_multilevel_rejects_bad_parameters():
    L = lib()
    g = graphgen.grid2d(10, 10)
    h = L.ad_graph_create(g.n, g.row_ptr, g.col, None)
    with pytest.raises(L.ADError):
        L.ad_ml_build(h, R=8, k=5, omega=0.5, seed=1, Q=1.0)
    ml = L.ad_ml_build(h, R=8, k=5, omega=0.5, seed=1, coarsest_n=10)
    with pytest.raises(L.ADError):
        L.ad_ml_sparsify(ml, np.ones(L.ad_ml_levels(ml) + 1), -1.0, np.zeros(g.m, np.uint8))
    L.ad_ml_destroy(ml)
    L.ad_graph_destroy(h)
