// sweep_f32.cu -- sweep / distance / init kernels for float storage.
#include "sweep_kernels.cuh"

namespace ad {

ad_status dispatch_f32(ad_graph_t g, const Config &cf, bool sweep, const SweepArgs &a, int64_t n_tasks,
                        size_t smem) {
    return dispatch<float>(g, cf, sweep, a, n_tasks, smem);
}

ad_status relax_f32(ad_graph_t g, const Config &cf, RelaxArgs &r) { return relax_dispatch<float>(g, cf, r); }

ad_status launch_init_f32(ad_graph_t g, int blocks, int32_t stride, uint64_t seed, uint32_t stream_id, void *x) {
    AD_LAUNCH(k_init<float>, blocks, 256, 0, g->stream, g->rp, g->n, stride, (uint32_t)seed, (uint32_t)(seed >> 32),
              stream_id, g->voff, g->G, static_cast<float *>(x));
    return AD_OK;
}

}  // namespace ad
