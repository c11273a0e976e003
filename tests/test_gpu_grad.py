"""GPU reverse mode of the per-sweep rescale form of Alg. 1 against the FP64
oracle's reverse mode (itself pinned by finite differences and by torch FP64
autograd of a dense formulation): loss = sum over a seeded edge subset S of
rho_e^2, gradient with respect to the undirected edge weights."""
import numpy as np
import pytest

import oracle
from paper_1601_05527_gb300 import graphgen
from gpu_util import lib

pytestmark = pytest.mark.gpu

GRAD_TOL = 1e-3     # relative error bound against the FP64 reverse mode (normwise max)


def weighted(g, seed):
    return graphgen.with_edge_weights(g, graphgen.uniform_edge_weights(g.m, seed=seed))


def grad_error(gpu, ref):
    scale = max(float(np.max(np.abs(ref))), 1e-30)
    return float(np.max(np.abs(gpu.astype(np.float64) - ref)) / scale)


def gpu_loss_grad(g, S, R, k, omega, seed, extra_flags=0):
    L = lib()
    h = L.ad_graph_create(g.n, g.row_ptr, g.col, g.weight)
    rho = np.zeros(g.m, np.float32)
    L.ad_algebraic_distance(h, R, k, omega, seed, 0, "fp32", L.AD_DIST_KEEP_STATE | extra_flags, rho)
    rb = np.zeros(g.m, np.float32)
    rb[S] = 2.0 * rho[S]
    wb = np.zeros(g.m, np.float32)
    L.ad_algebraic_distance_backward(h, rb, wb)
    L.ad_graph_destroy(h)
    return float((rho[S].astype(np.float64) ** 2).sum()), wb


@pytest.mark.parametrize("k", [1, 9, 12])
def test_every_iterate_kept_equals_sqrt_checkpoints(k):
    """The backward either uses every kept iterate or recomputes them from
    ceil(sqrt k) checkpoints; the sweep is deterministic, so the two gradients
    must be identical bit for bit (k = 9: whole segments, k = 12: a short last one)."""
    L = lib()
    g = weighted(graphgen.rmat(11, 16, seed=4), 3)
    S = graphgen.random_edge_subset(g.m, 0.05, seed=2)
    la, wa = gpu_loss_grad(g, S, 16, k, 0.5, 7)
    lb, wb = gpu_loss_grad(g, S, 16, k, 0.5, 7, L.AD_DIST_SQRT_CHECKPOINTS)
    assert la == lb
    np.testing.assert_array_equal(wa, wb)


@pytest.mark.parametrize("name,make,R,k", [
    ("ba500", lambda: weighted(graphgen.barabasi_albert(500, 4, seed=1), 2), 8, 6),
    ("rmat10", lambda: weighted(graphgen.rmat(10, 8, seed=3), 4), 16, 12),
    ("ws800", lambda: weighted(graphgen.watts_strogatz(800, 6, 0.2, seed=5), 6), 12, 9),
    ("rmat13_hubs", lambda: weighted(graphgen.rmat(13, 16, seed=7), 8), 32, 10),
    ("grid_unit", lambda: graphgen.grid2d(24, 24), 8, 20),
])
def test_gradient_matches_fp64_reverse_mode(name, make, R, k):
    g = make()
    S = graphgen.random_edge_subset(g.m, 0.05, seed=9)
    omega, seed = 0.5, 13
    loss, wb = gpu_loss_grad(g, S, R, k, omega, seed)
    w64 = None if g.weight is None else g.weight.astype(np.float64)
    ref_loss, ref = oracle.loss_grad(g.row_ptr, g.col, w64, S, R=R, k=k, omega=omega, seed=seed)
    assert loss == pytest.approx(ref_loss, rel=1e-4)
    assert grad_error(wb, ref) < GRAD_TOL


def test_torch_autograd_function():
    import torch
    from paper_1601_05527_gb300 import Graph
    from paper_1601_05527_gb300.autograd import algebraic_distance
    lib()
    g = weighted(graphgen.rmat(10, 8, seed=3), 4)
    S = graphgen.random_edge_subset(g.m, 0.05, seed=9)
    graph = Graph.from_graphgen(g)
    w = torch.tensor(g.edge_weights(), device="cuda", requires_grad=True)
    rho = algebraic_distance(w, graph, 16, 12, 0.5, 13)
    idx = torch.tensor(S, device="cuda")
    (rho[idx] ** 2).sum().backward()
    _, ref = oracle.loss_grad(g.row_ptr, g.col, g.weight.astype(np.float64), S, R=16, k=12, omega=0.5, seed=13)
    assert grad_error(w.grad.cpu().numpy(), ref) < GRAD_TOL
    graph.close()


def test_backward_without_state_is_rejected():
    L = lib()
    g = graphgen.grid2d(4, 4)
    h = L.ad_graph_create(g.n, g.row_ptr, g.col, None)
    with pytest.raises(L.ADError) as ei:
        L.ad_algebraic_distance_backward(h, np.zeros(g.m, np.float32), np.zeros(g.m, np.float32))
    assert ei.value.status == 9
    L.ad_graph_destroy(h)
