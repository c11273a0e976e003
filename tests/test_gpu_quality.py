"""Synthetic quality check of the selection methods (Fig. 1 and Sec. 4):
on dense planted clusters joined by sparse cuts, keeping delta-strong edges
(local) drops the cut edges, keeping delta-weak edges (global) keeps them,
and the binned mixture (Alg. 3) keeps them as well as a share of the
intra-cluster edges; Local Degree (the comparison method) ignores the
cluster structure.  Distances come from the GPU path."""
import numpy as np
import pytest

from paper_1601_05527_gb300 import graphgen
from gpu_util import lib

pytestmark = pytest.mark.gpu


def test_cut_edges_by_method():
    L = lib()
    g, cut = graphgen.planted_partition(20, 100, 0.15, 30, seed=3)
    cut = cut.astype(bool)
    h = L.ad_graph_create(g.n, g.row_ptr, g.col, None)
    L.ad_algebraic_distance(h, 16, 20, 0.5, 1, 0, "fp32", 0, None)
    kept = {}
    for name in ("local", "global", "binned", "ld"):
        keep = np.zeros(g.m, np.uint8)
        if name in ("local", "global"):
            n_kept, _ = L.ad_sparsify(h, 0.3, name, "per_node", keep)
        elif name == "binned":
            n_kept, _ = L.ad_sparsify_binned(h, None, 0.3, 5, keep)
        else:
            n_kept, _ = L.ad_sparsify_local_degree(h, 0.3, keep)
        assert n_kept == keep.sum() >= round(0.3 * g.m)
        kept[name] = (keep[cut].mean(), keep[~cut].mean())
    L.ad_graph_destroy(h)
    assert kept["local"][0] <= 0.02                 # bridges dropped
    assert kept["global"][0] >= 0.98                # bridges kept
    assert kept["binned"][0] >= 0.9 and kept["binned"][1] >= 0.2   # both kinds kept
    assert 0.05 <= kept["ld"][0] <= 0.9             # degree-driven: no preference either way
