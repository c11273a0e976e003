"""Pins for the oracle's reverse mode of Alg. 1 (per-sweep rescale form).

Loss L(w) = sum_{e in S} rho_e^2 over a seeded edge subset S, differentiated
with respect to the undirected edge weights.  Checked against
  * the forward value of the independent oracle.algebraic_distance;
  * central finite differences of that forward value (FP64);
  * torch autograd (CPU, FP64) of a dense formulation of the same forward:
    W(w) dense, D = W 1, x <- (1-omega) x + omega D^-1 W x, min/max rescale.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_1601_05527_gb300 import graphgen


def weighted(g, seed):
    return graphgen.with_edge_weights(g, graphgen.uniform_edge_weights(g.m, seed=seed))


def loss_fwd(g, w_edges, S, R, k, omega, seed):
    # FP64 weight per CSR entry (finite differences perturb them below FP32 resolution)
    eid = oracle.entry_edge_ids(g.row_ptr, g.col)
    w_entry = np.asarray(w_edges, dtype=np.float64)[eid]
    rho = oracle.algebraic_distance(g.row_ptr, g.col, w_entry, R=R, k=k, omega=omega, seed=seed)
    return float((rho[S] ** 2).sum())


def torch_dense_grad(g, w_edges, S, R, k, omega, seed):
    eu, ev = g.edges_upper()
    w = torch.tensor(np.asarray(w_edges, dtype=np.float64), requires_grad=True)
    W = torch.zeros(g.n, g.n, dtype=torch.float64)
    W = W.index_put((torch.tensor(eu, dtype=torch.long), torch.tensor(ev, dtype=torch.long)), w)
    W = W + W.T
    D = W.sum(1)
    act = torch.tensor(g.degrees() > 0)
    x = torch.tensor(oracle.init_vectors(g.n, R, seed=seed))
    for _ in range(k):
        y = torch.where(act[:, None], (1 - omega) * x + omega * (W @ x) / D.clamp_min(1e-300)[:, None], x)
        lo = y[act].min(0).values
        hi = y[act].max(0).values
        x = torch.where(act[:, None], (y - lo) / (hi - lo) - 0.5, x)
    d = x[torch.tensor(eu[S], dtype=torch.long)] - x[torch.tensor(ev[S], dtype=torch.long)]
    L = (d ** 2).sum()
    L.backward()
    return float(L.detach()), w.grad.numpy()


CASES = [
    ("ba60", lambda: weighted(graphgen.barabasi_albert(60, 3, seed=1), 2)),
    ("ws40", lambda: weighted(graphgen.watts_strogatz(40, 4, 0.2, seed=3), 4)),
    ("rmat7", lambda: weighted(graphgen.rmat(7, 4, seed=5), 6)),
]


@pytest.mark.parametrize("name,make", CASES)
@pytest.mark.parametrize("omega,k", [(0.5, 3), (0.35, 8)])
def test_grad_matches_torch_dense_autograd(name, make, omega, k):
    g = make()
    R, seed = 4, 21
    S = graphgen.random_edge_subset(g.m, 0.3, seed=1)
    w_edges = g.edge_weights().astype(np.float64)
    eid = oracle.entry_edge_ids(g.row_ptr, g.col)
    L, grad = oracle.loss_grad(g.row_ptr, g.col, w_edges[eid], S, R=R, k=k, omega=omega, seed=seed)
    Lt, gt = torch_dense_grad(g, w_edges, S, R, k, omega, seed)
    assert L == pytest.approx(Lt, rel=1e-11)
    assert L == pytest.approx(loss_fwd(g, w_edges, S, R, k, omega, seed), rel=1e-12)
    scale = np.max(np.abs(gt))
    np.testing.assert_allclose(grad, gt, rtol=1e-8, atol=1e-10 * scale)


def test_grad_matches_central_differences():
    g = weighted(graphgen.barabasi_albert(40, 3, seed=8), 9)
    R, k, omega, seed = 3, 6, 0.5, 2
    S = graphgen.random_edge_subset(g.m, 0.25, seed=3)
    w_edges = g.edge_weights().astype(np.float64)
    eid = oracle.entry_edge_ids(g.row_ptr, g.col)
    _, grad = oracle.loss_grad(g.row_ptr, g.col, w_edges[eid], S, R=R, k=k, omega=omega, seed=seed)
    h = 1e-6
    fd = np.zeros(g.m)
    for e in range(g.m):
        wp = w_edges.copy(); wp[e] += h
        wm = w_edges.copy(); wm[e] -= h
        fd[e] = (loss_fwd(g, wp, S, R, k, omega, seed) - loss_fwd(g, wm, S, R, k, omega, seed)) / (2 * h)
    scale = np.max(np.abs(fd))
    np.testing.assert_allclose(grad, fd, rtol=1e-5, atol=1e-6 * scale)


def test_unit_weight_grad_equals_explicit_ones():
    g = graphgen.watts_strogatz(30, 4, 0.1, seed=2)
    S = np.arange(0, g.m, 3)
    L1, g1 = oracle.loss_grad(g.row_ptr, g.col, None, S, R=4, k=5, omega=0.5, seed=3)
    L2, g2 = oracle.loss_grad(g.row_ptr, g.col, np.ones(g.nnz), S, R=4, k=5, omega=0.5, seed=3)
    assert L1 == L2
    np.testing.assert_array_equal(g1, g2)
