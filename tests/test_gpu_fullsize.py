"""Parity at the full sizes of the multilevel, batched and differentiable
workloads (the benchmark's own R-MAT scale-20 workload is covered in
test_gpu_distance.py and test_gpu_select.py).

Where the FP64 oracle cannot finish the whole workload in seconds, it is
compared on sampled units it can compute alone (whole graphs of a batch) or at
a reduced sweep count on the full graph; the rest is checked through
properties that hold at any size."""
import numpy as np
import pytest

import oracle
from paper_1601_05527_gb300 import graphgen
from gpu_util import assert_rho_close, jaccard, lib

pytestmark = pytest.mark.gpu

SEED = 0x1601055270000000


def test_batched_512_watts_strogatz_sampled_graphs():
    """512 Watts-Strogatz graphs, n ~ U{1000..200000}, ring degree 10, p = 0.1,
    R = 16, k = 15, all in one handle; per-graph 25% global per-node
    sparsification.  Sampled graphs (smallest, largest, three seeded others)
    are run through the oracle alone."""
    L = lib()
    graphs = graphgen.ws_batch(512, seed=5)
    voff, big = graphgen.concat(graphs)
    assert big.m > 200_000_000
    h = L.ad_graph_create_batched(voff, big.n, big.row_ptr, big.col, None)
    eoff = L.ad_graph_edge_offsets(h)
    sizes = np.array([gg.n for gg in graphs])
    rng = np.random.default_rng(5)
    sample = sorted({int(np.argmin(sizes)), int(np.argmax(sizes)), *rng.choice(512, 3, replace=False).tolist()})
    rho = np.zeros(big.m, np.float32)
    L.ad_algebraic_distance(h, 16, 15, 0.5, SEED, 0, "fp32", 0, rho)
    keep = np.zeros(big.m, np.uint8)
    L.ad_sparsify(h, 0.25, "global", "per_node", keep)
    rho16 = np.zeros(big.m, np.float32)
    L.ad_algebraic_distance(h, 16, 15, 0.5, SEED, 0, "bf16", 0, rho16)
    L.ad_graph_destroy(h)
    for gi in sample:
        gg = graphs[gi]
        sl = slice(int(eoff[gi]), int(eoff[gi + 1]))
        ref = oracle.algebraic_distance(gg.row_ptr, gg.col, None, R=16, k=15, omega=0.5, seed=SEED)
        assert_rho_close(rho[sl], ref)
        # BF16 storage: the rescaled distances stay within 5% (RMS-relative) on these graphs
        d = rho16[sl].astype(np.float64) - ref
        assert np.sqrt(np.mean(d ** 2)) <= 0.05 * np.sqrt(np.mean(ref ** 2))
        # selection on the GPU's own FP32 scores is exact, graph by graph
        rk, _, _ = oracle.sparsify(gg.row_ptr, gg.col, rho[sl].astype(np.float64), "global", "per_node", 0.25)
        np.testing.assert_array_equal(keep[sl], rk)


def _subgraph(level, mask):
    """CSR of the edges of a level kept by mask (edge-id order preserved) and
    the level edge id of each of its edges."""
    gl = graphgen.Graph(len(level["row_ptr"]) - 1, level["row_ptr"], level["col"], level["weight"])
    u, v = gl.edges_upper()
    ew = gl.edge_weights()
    sel = np.flatnonzero(mask)
    sub = graphgen.from_edges(gl.n, u[sel], v[sel], None if ew is None else ew[sel])
    return sub, sel


def test_multilevel_barabasi_albert_2m():
    """Barabasi-Albert n = 2,000,000, m = 8, lognormal(0, 1) weights, R = 16,
    k = 20, hierarchy to about 1,000 vertices, 40% controlled at the coarse
    levels (Sec. 5, Eq. (P), Alg. 6).

    Level by level, on the GPU's own inputs: each level's downward distances
    against the FP64 oracle on that level's graph (Philox stream 2l), and the
    oracle's seeds, Eq. (P) aggregates, Galerkin coarse graph and
    fine-to-coarse map computed from the GPU's level graph and FP32 distances
    must equal the GPU's next level exactly.  On the way up (traced): every
    level's inherited edges equal the oracle's uncoarsening of the coarser
    level's kept set, its kept set equals the oracle's Alg. 2 selection on the
    GPU's recomputed distances, and those distances on G_f^s match the oracle's
    (stream 2l + 1).  End to end against the oracle's own hierarchy, where the
    finest levels decide the selection, the kept sets agree at Jaccard >= 0.99;
    deeper, the two hierarchies are different random draws of the method
    (FP32 / FP64 near-ties in Eq. (P) renumber coarse vertices, whose Philox
    vectors follow their number), which the conditional checks above
    factor out."""
    L = lib()
    g = graphgen.barabasi_albert(2_000_000, 8, seed=4)
    g = graphgen.with_edge_weights(g, graphgen.lognormal_edge_weights(g.m, seed=4))
    w64 = g.weight.astype(np.float64)
    h = L.ad_graph_create(g.n, g.row_ptr, g.col, g.weight)
    ml = L.ad_ml_build(h, R=16, k=20, omega=0.5, seed=SEED, Q=0.5, coarsest_n=1000, mode="local")
    Lv = L.ad_ml_levels(ml)
    assert Lv >= 5
    levels = [L.ad_ml_level_export(ml, lvl) for lvl in range(Lv)]
    np.testing.assert_array_equal(levels[0]["row_ptr"], g.row_ptr)
    np.testing.assert_array_equal(levels[0]["col"], g.col)
    np.testing.assert_array_equal(levels[0]["weight"], g.weight)
    for lvl in range(Lv):
        lv = levels[lvl]
        rp, ci, wl = lv["row_ptr"], lv["col"], lv["weight"].astype(np.float64)
        assert_rho_close(lv["rho"], oracle.algebraic_distance(rp, ci, wl, R=16, k=20, omega=0.5, seed=SEED,
                                                              stream=2 * lvl))
        n_l = len(rp) - 1
        if lvl == Lv - 1:
            assert n_l <= 1000 or len(levels[lvl - 1]["row_ptr"]) - 1 < n_l / 0.9
            break
        seeds = oracle.create_seeds(rp, ci, wl, 0.5)
        ragg, rnc = oracle.aggregate(rp, ci, lv["rho"].astype(np.float64), seeds)
        np.testing.assert_array_equal(lv["agg"], ragg)
        nxt = levels[lvl + 1]
        assert len(nxt["row_ptr"]) - 1 == rnc
        rrpc, rcic, rwc, rf2c = oracle.galerkin(rp, ci, wl, ragg, rnc)
        np.testing.assert_array_equal(nxt["row_ptr"], rrpc)
        np.testing.assert_array_equal(nxt["col"], rcic)
        np.testing.assert_array_equal(nxt["weight"], rwc.astype(np.float32))
        np.testing.assert_array_equal(lv["f2c"], rf2c)

    # upward half, 40% controlled at the coarse third of the levels, traced
    L.ad_ml_set_trace(ml, True)
    span = max(1, Lv // 3)
    ratios = L.ad_ml_segment_ratios(Lv, "coarse", span, 1.0)
    keep = np.zeros(g.m, np.uint8)
    kept, r = L.ad_ml_sparsify(ml, ratios, 0.4, keep)
    assert kept == keep.sum() and kept >= oracle.target_count(g.m, 0.4)
    prev = None
    for lvl in reversed(range(Lv)):
        inh, kp, rup = L.ad_ml_level_trace(ml, lvl)
        lv = levels[lvl]
        ratio = r if ratios[Lv - 1 - lvl] >= 0 else -1.0
        if lvl == Lv - 1:
            assert inh.all()
        else:
            np.testing.assert_array_equal(inh, oracle.uncoarsen(lv["f2c"], prev))
        if ratio < 0:
            np.testing.assert_array_equal(kp, inh)
        elif lvl == Lv - 1:
            rk, _, _ = oracle.sparsify(lv["row_ptr"], lv["col"], lv["rho"].astype(np.float64), "local", "per_node",
                                       ratio)
            np.testing.assert_array_equal(kp, rk)
        else:
            sub, sel = _subgraph(lv, inh)
            rk, _, _ = oracle.sparsify(sub.row_ptr, sub.col, rup[sel].astype(np.float64), "local", "per_node", ratio)
            expect = np.zeros_like(kp)
            expect[sel] = rk
            np.testing.assert_array_equal(kp, expect)
            assert_rho_close(rup[sel], oracle.algebraic_distance(sub.row_ptr, sub.col, sub.weight.astype(np.float64),
                                                                 R=16, k=20, omega=0.5, seed=SEED,
                                                                 stream=2 * lvl + 1))
        prev = kp
    np.testing.assert_array_equal(keep, prev)

    # end to end against the oracle's own hierarchy
    ref = oracle.Multilevel(g.row_ptr, g.col, w64, R=16, k=20, omega=0.5, seed=SEED, Q=0.5, coarsest_n=1000,
                            mode="local")
    fine = max(1, min(Lv, ref.levels) // 3)
    kept, _ = L.ad_ml_sparsify(ml, L.ad_ml_segment_ratios(Lv, "fine", fine, 0.5), -1.0, keep)
    rkeep, rkept, _ = ref.sparsify(L.ad_ml_segment_ratios(ref.levels, "fine", fine, 0.5), -1.0)
    assert jaccard(keep, rkeep) >= 0.99, (jaccard(keep, rkeep), kept, rkept)
    L.ad_ml_destroy(ml)
    ref.close()
    L.ad_graph_destroy(h)


def _loss_grad(L, h, m, S, R, k):
    rho = np.zeros(m, np.float32)
    L.ad_algebraic_distance(h, R, k, 0.5, SEED, 0, "fp32", L.AD_DIST_KEEP_STATE, rho)
    rb = np.zeros(m, np.float32)
    rb[S] = 2.0 * rho[S]
    wb = np.zeros(m, np.float32)
    L.ad_algebraic_distance_backward(h, rb, wb)
    return float((rho[S].astype(np.float64) ** 2).sum()), wb


def test_gradient_rmat22():
    """R-MAT scale 22, uniform(0.5, 2) weights, R = 32, loss over a seeded 1%
    edge subset.  At k = 2 the whole gradient is compared with the oracle's
    FP64 reverse mode; at the workload's k = 30 (sqrt(k) checkpoints) the
    gradient must reproduce a central difference of the loss along the
    gradient's sign pattern, and satisfy sum_e w_e dL/dw_e = 0, which follows
    from D^-1 W (hence every rho) being unchanged when all weights are scaled."""
    L = lib()
    g = graphgen.rmat(22, 16, seed=6)
    ew = graphgen.uniform_edge_weights(g.m, seed=6)
    g = graphgen.with_edge_weights(g, ew)
    S = graphgen.random_edge_subset(g.m, 0.01, seed=6)
    h = L.ad_graph_create(g.n, g.row_ptr, g.col, g.weight)
    loss, wb = _loss_grad(L, h, g.m, S, 32, 2)
    ref_loss, ref = oracle.loss_grad(g.row_ptr, g.col, g.weight.astype(np.float64), S, R=32, k=2, omega=0.5,
                                     seed=SEED)
    assert loss == pytest.approx(ref_loss, rel=1e-4)
    assert np.max(np.abs(wb - ref)) <= 1e-3 * np.max(np.abs(ref))

    loss, wb = _loss_grad(L, h, g.m, S, 32, 30)
    wb64 = wb.astype(np.float64)
    ew64 = ew.astype(np.float64)
    # scaling every weight by c leaves the loss unchanged: sum_e w_e dL/dw_e = 0
    assert abs(np.dot(ew64, wb64)) <= 1e-4 * np.sum(np.abs(ew64 * wb64))
    # central difference along v = sign(grad) * w (relative step 1e-3)
    v = np.sign(wb64) * ew64
    hstep = 1e-3
    lp = lm = None
    for sgn in (1.0, -1.0):
        L.ad_graph_set_edge_weights(h, (ew64 + sgn * hstep * v).astype(np.float32))
        rho = np.zeros(g.m, np.float32)
        L.ad_algebraic_distance(h, 32, 30, 0.5, SEED, 0, "fp32", 0, rho)
        val = float((rho[S].astype(np.float64) ** 2).sum())
        lp, lm = (val, lm) if sgn > 0 else (lp, val)
    fd = (lp - lm) / (2 * hstep)
    an = float(np.dot(wb64, v))
    assert fd == pytest.approx(an, rel=2e-2), (fd, an, loss)
    L.ad_graph_destroy(h)
