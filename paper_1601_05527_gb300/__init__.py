"""GB300-native (sm_103a) network sparsification by algebraic distance.

John & Safro, "Single- and Multi-level Network Sparsification by Algebraic
Distance" (arXiv 1601.05527): Philox-seeded test vectors relaxed by Jacobi
over-relaxation sweeps with a per-sweep rescale, per-edge algebraic
distances, edge ranking and sampling (Alg. 2, local or global filtering) and
the multilevel framework of Alg. 6.  The compute path is the CUDA library
libad.so behind the C ABI of include/ad.h; ``_lib`` is its ctypes binding
(same names as the C functions), ``graphgen`` builds seeded synthetic inputs.
"""
from . import graphgen  # noqa: F401
from ._lib import (  # noqa: F401
    ADError, AD_DIST_KEEP_STATE, AD_DIST_NORMALIZE, AD_CREATE_SKIP_VALIDATION, MODES, SCOPES, STORAGES,
    ad_algebraic_distance, ad_algebraic_distance_backward, ad_coarsen, ad_graph_create, ad_graph_create_batched,
    ad_graph_autotune, ad_graph_destroy, ad_graph_edge_offsets, ad_graph_export, ad_graph_info, ad_graph_phase_time, ad_graph_set_edge_weights,
    ad_graph_set_profiling, ad_kernel_launch_count, ad_last_error, ad_ml_build, ad_ml_destroy, ad_ml_level_size,
    ad_ml_levels, ad_ml_segment_ratios, ad_ml_sparsify, ad_select_per_node, ad_sparsify, ad_sparsify_binned,
    ad_sparsify_local_degree, ad_sparsify_scores,
    ad_status_string, ad_version, load, use_default_allocator, use_torch_allocator,
)


class Graph:
    """Owning wrapper of an ad_graph_t handle (argument marshalling only)."""

    def __init__(self, row_ptr, col, weight=None, *, n=None, vertex_offset=None, validate=True, stream=None):
        n = len(row_ptr) - 1 if n is None else n
        flags = 0 if validate else AD_CREATE_SKIP_VALIDATION
        if vertex_offset is None:
            self.handle = ad_graph_create(n, row_ptr, col, weight, flags, stream)
        else:
            self.handle = ad_graph_create_batched(vertex_offset, n, row_ptr, col, weight, flags, stream)
        info = ad_graph_info(self.handle)
        self.n, self.m, self.nnz, self.n_active, self.n_graphs = (info["n"], info["m"], info["nnz"],
                                                                  info["n_active"], info["n_graphs"])

    @classmethod
    def from_graphgen(cls, g, **kw):
        return cls(g.row_ptr, g.col, g.weight, n=g.n, **kw)

    def algebraic_distance(self, R, k, omega=0.5, seed=0, *, stream_id=0, storage="fp32", normalize=False,
                           out=None, keep_state=False):
        flags = (AD_DIST_NORMALIZE if normalize else 0) | (AD_DIST_KEEP_STATE if keep_state else 0)
        return ad_algebraic_distance(self.handle, R, k, omega, seed, stream_id, storage, flags, out)

    def sparsify(self, fraction, mode="local", scope="per_node", keep_out=None, scores=None):
        import numpy as np
        keep = keep_out if keep_out is not None else np.zeros(self.m, dtype=np.uint8)
        if scores is None:
            kept, e = ad_sparsify(self.handle, fraction, mode, scope, keep)
        else:
            kept, e = ad_sparsify_scores(self.handle, scores, fraction, mode, scope, keep)
        return keep, kept, e

    def close(self):
        if getattr(self, "handle", None) is not None:
            ad_graph_destroy(self.handle)
            self.handle = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
