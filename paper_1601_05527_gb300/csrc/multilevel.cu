// multilevel.cu -- Sec. 5 / Alg. 6 (MLSparsify) on the device.
#include "ad_internal.cuh"

extern "C" ad_status ad_ml_build(ad_graph_t g, const ad_ml_params *, ad_ml_t *out) {
    if (out) *out = nullptr;
    if (!g) return ad::fail(AD_ERR_INVALID_ARG, "NULL graph");
    return ad::fail(AD_ERR_STATE, "multilevel hierarchy not available in this build");
}
extern "C" ad_status ad_ml_levels(ad_ml_t, int32_t *) { return ad::fail(AD_ERR_STATE, "no hierarchy"); }
extern "C" ad_status ad_ml_level_size(ad_ml_t, int32_t, int64_t *, int64_t *) { return ad::fail(AD_ERR_STATE, "no hierarchy"); }
extern "C" ad_status ad_ml_sparsify(ad_ml_t, const double *, int32_t, double, uint8_t *, int64_t *, double *) {
    return ad::fail(AD_ERR_STATE, "no hierarchy");
}
extern "C" ad_status ad_ml_segment_ratios(int32_t n_levels, int32_t segment, int32_t level_span, double value,
                                          double *ratios_out) {
    if (n_levels < 1 || level_span < 1 || segment < 1 || segment > 3 || !ratios_out)
        return ad::fail(AD_ERR_INVALID_ARG, "bad segment arguments");
    const int32_t s = level_span < n_levels ? level_span : n_levels;
    int32_t start = segment == 1 ? 0 : (segment == 2 ? (n_levels - s) / 2 : n_levels - s);
    for (int32_t t = 0; t < n_levels; ++t) ratios_out[t] = (t >= start && t < start + s) ? value : -1.0;
    return AD_OK;
}
extern "C" ad_status ad_ml_destroy(ad_ml_t) { return AD_OK; }
extern "C" ad_status ad_coarsen(ad_graph_t g, const float *, double, int32_t *, int64_t *, ad_graph_t *, int64_t *) {
    if (!g) return ad::fail(AD_ERR_INVALID_ARG, "NULL graph");
    return ad::fail(AD_ERR_STATE, "coarsening not available in this build");
}
