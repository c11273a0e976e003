// grad.cu -- reverse mode of ComputeAlgDist (per-sweep rescale form of Alg. 1).
#include "ad_internal.cuh"

namespace ad {

struct ad_graph_s_saved_placeholder {};

ad_status algebraic_distance_keep(ad_graph_t g, int32_t, int32_t, double, uint64_t, uint32_t, float *) {
    (void)g;
    return fail(AD_ERR_STATE, "backward state is not available in this build");
}

void free_saved(ad_graph_t g) { g->saved = nullptr; }

}  // namespace ad

extern "C" ad_status ad_algebraic_distance_backward(ad_graph_t g, const float *, float *) {
    if (!g) return ad::fail(AD_ERR_INVALID_ARG, "NULL graph");
    return ad::fail(AD_ERR_STATE, "no kept state");
}
