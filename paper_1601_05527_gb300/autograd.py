"""torch.autograd binding of the algebraic distance (marshalling only).

``algebraic_distance(w, graph, R, k, omega, seed)`` returns rho[m] for the
undirected edge weights w[m] (CUDA float32, edge-id order) and is
differentiable in w: the forward runs the library's sweeps with checkpoints
(``AD_DIST_KEEP_STATE``), the backward calls ``ad_algebraic_distance_backward``
(reverse mode of the per-sweep rescale form of Alg. 1).  One pending backward
per graph handle: a later forward on the same handle replaces the kept state.
"""
import torch

from . import _lib as L


class AlgebraicDistanceFunction(torch.autograd.Function):
    @staticmethod
    def forward(ctx, w_edges, handle, m, R, k, omega, seed):
        w = w_edges.detach().contiguous()
        L.ad_graph_set_edge_weights(handle, w)
        rho = torch.empty(m, dtype=torch.float32, device=w.device)
        L.ad_algebraic_distance(handle, R, k, omega, seed, 0, "fp32", L.AD_DIST_KEEP_STATE, rho)
        ctx.handle = handle
        ctx.m = m
        return rho

    @staticmethod
    def backward(ctx, grad_rho):
        wbar = torch.empty(ctx.m, dtype=torch.float32, device=grad_rho.device)
        L.ad_algebraic_distance_backward(ctx.handle, grad_rho.detach().contiguous().float(), wbar)
        return wbar, None, None, None, None, None, None


def algebraic_distance(w_edges, graph, R, k, omega=0.5, seed=0):
    """rho[m] of Alg. 1 (per-sweep rescale), differentiable in the edge weights."""
    return AlgebraicDistanceFunction.apply(w_edges, graph.handle, graph.m, R, k, omega, seed)
