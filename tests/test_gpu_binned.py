"""GPU parity of SparsifyB (Alg. 3, the binned "mixture" selection of Sec. 4).

Given identical FP32 scores the bins, the random orders and the fitted
exponent are integer decisions taken with the same FP64 operations on both
sides, so the kept edge set, its size and e must equal the oracle's exactly."""
import numpy as np
import pytest

import oracle
from paper_1601_05527_gb300 import graphgen
from gpu_util import lib

pytestmark = pytest.mark.gpu


def star_mix(seed=3):
    """Hubs whose incident distances form clusters of different widths."""
    rng = np.random.default_rng(seed)
    n = 6000
    u = [rng.integers(0, n, 20000)]
    v = [rng.integers(0, n, 20000)]
    for hub, d in zip(range(3), (300, 1500, 5000)):
        u.append(np.full(d, hub))
        v.append(rng.choice(np.arange(3, n), d, replace=False))
    return graphgen.from_edges(n, np.concatenate(u), np.concatenate(v))


GRAPHS = {
    "rmat12": lambda: graphgen.rmat(12, 16, seed=3),
    "ba2000": lambda: graphgen.barabasi_albert(2000, 6, seed=2),
    "grid32": lambda: graphgen.grid2d(32, 32),
    "hubs": star_mix,
}


def scores_for(g, kind, seed):
    rng = np.random.default_rng(seed)
    if kind == "uniform":
        return rng.random(g.m).astype(np.float32)
    if kind == "skewed":                         # heavy right tail: many bins at hubs
        return (rng.random(g.m) ** 4).astype(np.float32)
    return graphgen.random_scores(g.m, 7, seed=seed)   # few distinct values: equal distances, sigma 0 rows


@pytest.mark.parametrize("name", list(GRAPHS))
@pytest.mark.parametrize("kind", ["uniform", "skewed", "ties"])
def test_binned_matches_oracle(name, kind):
    L = lib()
    g = GRAPHS[name]()
    s = scores_for(g, kind, 17)
    h = L.ad_graph_create(g.n, g.row_ptr, g.col, None)
    try:
        for f, seed in ((0.0, 1), (0.3, 2), (0.6, 0x1601055270000000), (1.0, 3)):
            keep = np.zeros(g.m, np.uint8)
            kept, e = L.ad_sparsify_binned(h, s, f, seed, keep)
            ref, rk, re_ = oracle.sparsify_binned(g.row_ptr, g.col, s.astype(np.float64), seed, f)
            assert kept == rk and e == re_, (f, kept, rk, e, re_)
            np.testing.assert_array_equal(keep, ref)
    finally:
        L.ad_graph_destroy(h)


def test_binned_on_own_distances_and_device_buffers():
    import torch
    L = lib()
    g = graphgen.rmat(11, 16, seed=8)
    h = L.ad_graph_create(g.n, g.row_ptr, g.col, None)
    rho = np.zeros(g.m, np.float32)
    L.ad_algebraic_distance(h, 16, 10, 0.5, 5, 0, "fp32", 0, rho)
    keep_d = torch.zeros(g.m, dtype=torch.uint8, device="cuda")
    kept, e = L.ad_sparsify_binned(h, None, 0.4, 77, keep_d)
    ref, rk, re_ = oracle.sparsify_binned(g.row_ptr, g.col, rho.astype(np.float64), 77, 0.4)
    assert kept == rk and e == re_
    np.testing.assert_array_equal(keep_d.cpu().numpy(), ref)
    L.ad_graph_destroy(h)


def test_binned_rejects_bad_input():
    L = lib()
    g = graphgen.grid2d(6, 6)
    h = L.ad_graph_create(g.n, g.row_ptr, g.col, None)
    keep = np.zeros(g.m, np.uint8)
    with pytest.raises(L.ADError) as ei:
        L.ad_sparsify_binned(h, None, 0.5, 1, keep)           # no distances yet
    assert ei.value.status == 9
    with pytest.raises(L.ADError):
        L.ad_sparsify_binned(h, np.full(g.m, -1.0, np.float32), 0.5, 1, keep)
    with pytest.raises(L.ADError):
        L.ad_sparsify_binned(h, np.ones(g.m, np.float32), 1.5, 1, keep)
    L.ad_graph_destroy(h)


def test_full_size_rmat20_binned_bit_exact():
    """The benchmark's graph (R-MAT scale 20, 15.7M edges) at 30%."""
    L = lib()
    g = graphgen.rmat(20, 16, seed=2)
    s = (np.random.default_rng(4).random(g.m) ** 2).astype(np.float32)
    h = L.ad_graph_create(g.n, g.row_ptr, g.col, None)
    keep = np.zeros(g.m, np.uint8)
    kept, e = L.ad_sparsify_binned(h, s, 0.3, 9, keep)
    L.ad_graph_destroy(h)
    ref, rk, re_ = oracle.sparsify_binned(g.row_ptr, g.col, s.astype(np.float64), 9, 0.3)
    assert kept == rk and e == re_
    np.testing.assert_array_equal(keep, ref)
