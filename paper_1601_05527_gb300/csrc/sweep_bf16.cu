// sweep_bf16.cu -- sweep / distance / init kernels for __nv_bfloat16 storage.
#include "sweep_kernels.cuh"

namespace ad {

ad_status dispatch_bf16(ad_graph_t g, const Config &cf, bool sweep, const SweepArgs &a, int64_t n_tasks,
                        size_t smem) {
    return dispatch<__nv_bfloat16>(g, cf, sweep, a, n_tasks, smem);
}

ad_status relax_bf16(ad_graph_t g, const Config &cf, RelaxArgs &r) { return relax_dispatch<__nv_bfloat16>(g, cf, r); }

ad_status launch_init_bf16(ad_graph_t g, int blocks, int32_t stride, uint64_t seed, uint32_t stream_id, void *x) {
    AD_LAUNCH(k_init<__nv_bfloat16>, blocks, 256, 0, g->stream, g->rp, g->n, stride, (uint32_t)seed, (uint32_t)(seed >> 32),
              stream_id, g->voff, g->G, static_cast<__nv_bfloat16 *>(x));
    return AD_OK;
}

}  // namespace ad
