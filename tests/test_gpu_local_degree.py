"""GPU parity of the Local Degree comparator (Sec. 1.1, Sec. 6): integer
work on degrees, so the kept set, its size and the fitted e equal the
oracle's exactly."""
import numpy as np
import pytest

import oracle
from paper_1601_05527_gb300 import graphgen
from gpu_util import lib
from test_gpu_select import hub_graph

pytestmark = pytest.mark.gpu

GRAPHS = {
    "rmat12": lambda: graphgen.rmat(12, 16, seed=3),
    "ba3000": lambda: graphgen.barabasi_albert(3000, 5, seed=1),
    "ws2000": lambda: graphgen.watts_strogatz(2000, 10, 0.2, seed=2),   # many equal degrees: ties
    "hubs": hub_graph,                                                   # rows above the per-CTA sort cap
}


@pytest.mark.parametrize("name", list(GRAPHS))
def test_local_degree_matches_oracle(name):
    L = lib()
    g = GRAPHS[name]()
    h = L.ad_graph_create(g.n, g.row_ptr, g.col, None)
    try:
        for f in (0.0, 0.25, 0.5, 1.0):
            keep = np.zeros(g.m, np.uint8)
            kept, e = L.ad_sparsify_local_degree(h, f, keep)
            ref, rk, re_ = oracle.sparsify_local_degree(g.row_ptr, g.col, f)
            assert kept == rk and e == re_, (f, kept, rk, e, re_)
            np.testing.assert_array_equal(keep, ref)
    finally:
        L.ad_graph_destroy(h)
