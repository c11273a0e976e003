// sweep.cu -- host side of ComputeAlgDist (Alg. 1): work plans, scratch, the
// k sweep launches and the distance launch.  Kernels: sweep_kernels.cuh.
#include "sweep_kernels.cuh"

namespace ad {

ad_status launch_init_f32(ad_graph_t g, int blocks, int32_t stride, uint64_t seed, uint32_t stream_id, void *x);
ad_status launch_init_bf16(ad_graph_t g, int blocks, int32_t stride, uint64_t seed, uint32_t stream_id, void *x);
ad_status launch_init_f16(ad_graph_t g, int blocks, int32_t stride, uint64_t seed, uint32_t stream_id, void *x);
ad_status launch_init_q16(ad_graph_t g, int blocks, int32_t stride, uint64_t seed, uint32_t stream_id, void *x);

ad_status launch_init(ad_graph_t g, ad_storage storage, int blocks, int32_t stride, uint64_t seed, uint32_t stream_id,
                      void *x) {
    switch (storage) {
        case AD_STORAGE_BF16: return launch_init_bf16(g, blocks, stride, seed, stream_id, x);
        case AD_STORAGE_FP16: return launch_init_f16(g, blocks, stride, seed, stream_id, x);
        case AD_STORAGE_Q16: return launch_init_q16(g, blocks, stride, seed, stream_id, x);
        default: return launch_init_f32(g, blocks, stride, seed, stream_id, x);
    }
}

// Natural shape: the row's 16-byte chunks, rounded up to a power of two, over
// as many lanes as possible (at most AD_MAX_LPR); a shape chosen by
// ad_graph_autotune for this (R, storage) replaces it.
Config natural_config(int R, ad_storage storage) {
    Config c;
    c.V = storage == AD_STORAGE_FP32 ? 4 : 8;
    c.nchunks = (R + c.V - 1) / c.V;
    int p2 = 1;
    while (p2 < c.nchunks) p2 <<= 1;
    c.lpr = p2 < AD_MAX_LPR ? p2 : AD_MAX_LPR;
    c.cpl = p2 / c.lpr;
    c.stride = p2 * c.V;
    return c;
}

void natural_shape(int R, ad_storage storage, int *lpr, int *cpl) {
    const Config c = natural_config(R, storage);
    *lpr = c.lpr;
    *cpl = c.cpl;
}

static Config pick_config(ad_graph_t g, int R, ad_storage storage) {
    Config c = natural_config(R, storage);
    for (const auto &t : g->tuned)
        if (t.R == R && t.storage == (int32_t)storage) {
            c.lpr = t.lpr;
            c.cpl = t.cpl;
            c.per_sm = t.per_sm;
        }
    return c;
}

// Degree bound of the group-per-row class: a group walks its row alone, so keep
// it to rows whose gathers fit a few rounds of one warp-wide pass.
static int small_max_for(int groups) { return groups >= 4 ? 2 * groups : 0; }

static ad_status dispatch_storage(ad_graph_t g, ad_storage storage, const Config &cf, bool sweep,
                                  const SweepArgs &a, size_t smem) {
    switch (storage) {
        case AD_STORAGE_BF16: return dispatch_bf16(g, cf, sweep, a, a.n_tasks, smem);
        case AD_STORAGE_FP16: return dispatch_f16(g, cf, sweep, a, a.n_tasks, smem);
        case AD_STORAGE_Q16: return dispatch_q16(g, cf, sweep, a, a.n_tasks, smem);
        default: return dispatch_f32(g, cf, sweep, a, a.n_tasks, smem);
    }
}

ad_status get_row_plan(ad_graph_t g, int groups, bool upper, RowPlan **out);
static ad_status get_plan(ad_graph_t g, int groups, bool upper, RowPlan **out) { return get_row_plan(g, groups, upper, out); }
ad_status get_row_plan(ad_graph_t g, int groups, bool upper, RowPlan **out) {
    auto &plans = upper ? g->dist_plans : g->sweep_plans;
    for (auto &p : plans)
        if (p.groups == groups) { *out = &p; return AD_OK; }
    RowPlan p;
    AD_TRY(build_row_plan(g, groups, upper ? groups : small_max_for(groups), upper, p));
    plans.push_back(p);
    *out = &plans.back();
    return AD_OK;
}

static void fill_plan(SweepArgs &a, const RowPlan &p) {
    a.big_row = p.big_row; a.big_chunk = p.big_chunk; a.medium_row = p.medium_row; a.small_row = p.small_row;
    a.big_counter = p.big_counter;
    a.n_big = p.n_big; a.n_medium = p.n_medium; a.n_small_rows = p.n_small_rows;
    a.n_tasks = p.tasks();
}

static void ev_begin(ad_graph_t g) {
    if (g->profiling) cudaEventRecord(g->ev0, g->stream);
}
static void ev_end(ad_graph_t g, double &acc, int64_t &cnt) {
    if (!g->profiling) return;
    cudaEventRecord(g->ev1, g->stream);
    cudaEventSynchronize(g->ev1);
    float ms = 0.f;
    cudaEventElapsedTime(&ms, g->ev0, g->ev1);
    acc += ms;
    cnt += 1;
}

// One sweep of stored vectors x_in -> x_out (previous affine from pmin/pmax,
// nullptr = none) reducing min/max into mn/mx; used to recompute iterates.
ad_status sweep_step(ad_graph_t g, ad_storage storage, int32_t R, double omega, const void *x_in, void *x_out,
                     const uint32_t *pmin, const uint32_t *pmax, uint32_t *mn, uint32_t *mx) {
    const Config cf = pick_config(g, R, storage);
    RowPlan *sp = nullptr;
    AD_TRY(get_plan(g, 32 / cf.lpr, false, &sp));
    AD_TRY(ensure(g, g->part, (size_t)(sp->n_big > 0 ? sp->n_big : 1) * cf.stride * sizeof(float)));
    SweepArgs a;
    memset(&a, 0, sizeof(a));
    a.rp = g->rp; a.col = g->col; a.w = g->w; a.Dinv = g->Dinv; a.D = g->D;
    a.upos = g->upos; a.eoff = g->eoff;
    a.part = static_cast<float *>(g->part.ptr);
    a.stride = cf.stride; a.nchunks = cf.nchunks; a.R = R;
    a.omega = (float)omega;
    a.voff = g->voff; a.G = g->G; a.blocked = g->G > 1 ? 1 : 0;
    a.anchor = g->anchor;
    AD_TRY(ensure(g, g->ac, (size_t)g->G * 2 * cf.stride * sizeof(float)));
    a.ac = static_cast<float *>(g->ac.ptr);
    fill_plan(a, *sp);
    a.x_in = x_in; a.x_out = x_out;
    a.mm_prev_min = pmin; a.mm_prev_max = pmax; a.mm_min = mn; a.mm_max = mx;
    return dispatch_storage(g, storage, cf, true, a, 2 * 8 * (size_t)cf.stride * sizeof(float));
}

// ----------------------------------------------------------------------------
// Persistent form (k_relax): init, k sweeps and distances in one cooperative
// launch with bounded grid barriers between sweeps.  A barrier that runs out
// leaves AD_ERR_TIMEOUT in the handle's flag, which a direct call reads back
// (inside a stream capture the call cannot wait, and the flag is not read).
// ----------------------------------------------------------------------------
static ad_status relax_storage(ad_graph_t g, ad_storage storage, const Config &cf, RelaxArgs &r) {
    switch (storage) {
        case AD_STORAGE_BF16: return relax_bf16(g, cf, r);
        case AD_STORAGE_FP16: return relax_f16(g, cf, r);
        case AD_STORAGE_Q16: return relax_q16(g, cf, r);
        default: return relax_f32(g, cf, r);
    }
}

static ad_status relax_persistent(ad_graph_t g, const Config &cf, int32_t R, int32_t k, double omega, uint64_t seed,
                                  uint32_t stream_id, ad_storage storage, int32_t flags, float *rho_dev,
                                  const RowPlan &sp, const RowPlan &dp) {
    AD_TRY(ensure(g, g->relax_sync, (kBarrierSlots + 4) * sizeof(unsigned int)));
    unsigned int *sync = static_cast<unsigned int *>(g->relax_sync.ptr);
    AD_CUDA_TRY(cudaMemsetAsync(sync, 0, (kBarrierSlots + 4) * sizeof(unsigned int), g->stream));
    RelaxArgs r;
    memset(&r, 0, sizeof(r));
    SweepArgs &a = r.s;
    a.rp = g->rp; a.col = g->col; a.w = g->w; a.Dinv = g->Dinv; a.D = g->D;
    a.upos = g->upos; a.eoff = g->eoff;
    a.part = static_cast<float *>(g->part.ptr);
    a.stride = cf.stride; a.nchunks = cf.nchunks; a.R = R;
    a.omega = (float)omega;
    a.normalize = (flags & AD_DIST_NORMALIZE) ? 1 : 0;
    a.voff = g->voff; a.G = 1; a.blocked = 0;
    a.anchor = g->anchor;
    r.d = a;
    fill_plan(r.s, sp);
    fill_plan(r.d, dp);
    r.d.rho = rho_dev;
    r.n = g->n;
    r.k = k;
    r.x0 = g->x0.ptr;
    r.x1 = g->x1.ptr;
    const size_t mm_words = (size_t)(k > 0 ? k : 1) * cf.stride;
    r.mm_min = static_cast<uint32_t *>(g->mm.ptr);
    r.mm_max = r.mm_min + mm_words;
    r.seed_lo = (uint32_t)seed;
    r.seed_hi = (uint32_t)(seed >> 32);
    r.stream_id = stream_id;
    r.bar = sync;
    r.err = reinterpret_cast<int *>(sync + kBarrierSlots);
    r.polls = AD_BARRIER_POLLS;
    r.extra = 0;
    AD_TRY(relax_storage(g, storage, cf, r));
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    AD_CUDA_TRY(cudaStreamIsCapturing(g->stream, &cs));
    if (cs == cudaStreamCaptureStatusNone) {
        int err = 0;
        AD_TRY(copy_out(g, &err, r.err, sizeof(int)));
        if (err != 0) return fail((ad_status)err, "a grid barrier of the persistent relaxation ran out of time");
    }
    return AD_OK;
}

// Self-test of the bounded grid barrier: a cooperative launch of two CTAs
// whose barrier waits for one arrival that never comes.
static __device__ unsigned int g_selftest_sync[kBarrierSlots + 4];

__global__ void k_barrier_selftest(RelaxArgs r) {
    if (grid_barrier(r, 1) && threadIdx.x == 0) atomicAdd(r.bar + kBarrierSlots + 1, 1u);   // CTAs that passed
}

}  // namespace ad

extern "C" ad_status ad_selftest_barrier_timeout(void *stream, uint32_t polls, int32_t *status_out) {
    using namespace ad;
    if (!status_out) return fail(AD_ERR_INVALID_ARG, "status_out is NULL");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    void *p = nullptr;
    AD_CUDA_TRY(cudaGetSymbolAddress(&p, g_selftest_sync));
    unsigned int *sync = static_cast<unsigned int *>(p);
    AD_CUDA_TRY(cudaMemsetAsync(sync, 0, (kBarrierSlots + 4) * sizeof(unsigned int), st));
    RelaxArgs r;
    memset(&r, 0, sizeof(r));
    r.bar = sync;
    r.err = reinterpret_cast<int *>(sync + kBarrierSlots);
    r.polls = polls;
    r.extra = 1;
    void *args[] = {&r};
    g_launches.fetch_add(1, std::memory_order_relaxed);
    AD_CUDA_TRY(cudaLaunchCooperativeKernel((const void *)k_barrier_selftest, dim3(2), dim3(64), args, 0, st));
    unsigned int h[kBarrierSlots + 4] = {};
    AD_CUDA_TRY(cudaMemcpyAsync(h, sync, sizeof(h), cudaMemcpyDeviceToHost, st));
    AD_CUDA_TRY(cudaStreamSynchronize(st));
    *status_out = (int32_t)h[kBarrierSlots];
    if (h[kBarrierSlots + 1] != 0) return fail(AD_ERR_STATE, "a CTA passed a barrier that could not complete");
    return AD_OK;
}

namespace ad {

ad_status algebraic_distance(ad_graph_t g, int32_t R, int32_t k, double omega, uint64_t seed,
                             uint32_t stream_id, ad_storage storage, int32_t flags, float *rho_dev,
                             const KeepSpec *keep) {
    if (g->m == 0) return AD_OK;   // no edges: nothing to relax and no distance to write
    const Config cf = pick_config(g, R, storage);
    const int groups = 32 / cf.lpr;
    const size_t esz = storage == AD_STORAGE_FP32 ? 4 : 2;
    const size_t xbytes = ((size_t)g->n + 1) * cf.stride * esz;
    AD_TRY(ensure(g, g->x0, xbytes));
    AD_TRY(ensure(g, g->x1, xbytes));
    const size_t mm_words = (size_t)(k > 0 ? k : 1) * g->G * cf.stride;
    AD_TRY(ensure(g, g->mm, 2 * mm_words * sizeof(uint32_t)));
    uint32_t *mm_min = static_cast<uint32_t *>(g->mm.ptr);
    uint32_t *mm_max = mm_min + mm_words;
    AD_CUDA_TRY(cudaMemsetAsync(mm_min, 0xff, mm_words * sizeof(uint32_t), g->stream));
    AD_CUDA_TRY(cudaMemsetAsync(mm_max, 0x00, mm_words * sizeof(uint32_t), g->stream));

    RowPlan *sp = nullptr, *dp = nullptr;
    AD_TRY(get_plan(g, groups, false, &sp));
    AD_TRY(get_plan(g, groups, true, &dp));
    AD_TRY(ensure(g, g->part, (size_t)(sp->n_big > 0 ? sp->n_big : 1) * cf.stride * sizeof(float)));

    // small single graphs (or on request): the whole computation in one persistent launch
    const bool persist = g->G == 1 && !keep && !g->profiling &&
                         ((flags & AD_DIST_PERSISTENT) || g->nnz <= kPersistMaxNnz);
    if (persist) return relax_persistent(g, cf, R, k, omega, seed, stream_id, storage, flags, rho_dev, *sp, *dp);

    // init
    {
        const int64_t total = g->n * (cf.stride / 4);
        int64_t blocks = (total + 255) / 256;
        if (blocks > (int64_t)g->num_sms * 16) blocks = (int64_t)g->num_sms * 16;
        if (blocks < 1) blocks = 1;
        ev_begin(g);
        AD_TRY(launch_init(g, storage, (int)blocks, cf.stride, seed, stream_id, g->x0.ptr));
        ev_end(g, g->init_ms, g->init_launches);
    }
    if (keep && !keep->ckpt.empty())
        AD_CUDA_TRY(cudaMemcpyAsync(keep->ckpt[0], g->x0.ptr, (size_t)g->n * cf.stride * esz, cudaMemcpyDeviceToDevice,
                                    g->stream));

    SweepArgs a;
    memset(&a, 0, sizeof(a));
    a.rp = g->rp; a.col = g->col; a.w = g->w; a.Dinv = g->Dinv; a.D = g->D;
    a.upos = g->upos; a.eoff = g->eoff;
    a.part = static_cast<float *>(g->part.ptr);
    a.stride = cf.stride; a.nchunks = cf.nchunks; a.R = R;
    a.omega = (float)omega;
    a.normalize = (flags & AD_DIST_NORMALIZE) ? 1 : 0;
    a.voff = g->voff;
    a.G = g->G;
    a.blocked = g->G > 1 ? 1 : 0;
    a.anchor = g->anchor;
    AD_TRY(ensure(g, g->ac, (size_t)g->G * 2 * cf.stride * sizeof(float)));
    a.ac = static_cast<float *>(g->ac.ptr);

    void *xin = g->x0.ptr, *xout = g->x1.ptr;
    // every iterate kept: the sweeps read and write the kept buffers directly
    const bool direct = keep && keep->every == 1 && keep->ckpt.size() == (size_t)k + 1;
    if (direct) xin = keep->ckpt[0];
    const size_t smem = 2 * 8 * (size_t)cf.stride * sizeof(float);
    fill_plan(a, *sp);
    for (int32_t t = 0; t < k; ++t) {
        if (direct) xout = keep->ckpt[t + 1];
        a.x_in = xin; a.x_out = xout;
        const size_t slot = (size_t)g->G * cf.stride;
        a.mm_prev_min = t > 0 ? mm_min + (size_t)(t - 1) * slot : nullptr;
        a.mm_prev_max = t > 0 ? mm_max + (size_t)(t - 1) * slot : nullptr;
        a.mm_min = mm_min + (size_t)t * slot;
        a.mm_max = mm_max + (size_t)t * slot;
        ev_begin(g);
        AD_TRY(dispatch_storage(g, storage, cf, true, a, smem));
        ev_end(g, g->sweep_ms, g->sweep_launches);
        if (keep && !direct && (t + 1) % keep->every == 0 && (size_t)((t + 1) / keep->every) < keep->ckpt.size())
            AD_CUDA_TRY(cudaMemcpyAsync(keep->ckpt[(t + 1) / keep->every], xout, (size_t)g->n * cf.stride * esz,
                                        cudaMemcpyDeviceToDevice, g->stream));
        void *tmp = xin; xin = xout; xout = tmp;
    }
    if (keep && keep->mm_copy)
        AD_CUDA_TRY(cudaMemcpyAsync(keep->mm_copy, g->mm.ptr, 2 * mm_words * sizeof(uint32_t), cudaMemcpyDeviceToDevice,
                                    g->stream));

    fill_plan(a, *dp);
    a.x_in = xin;
    a.mm_prev_min = k > 0 ? mm_min + (size_t)(k - 1) * g->G * cf.stride : nullptr;
    a.mm_prev_max = k > 0 ? mm_max + (size_t)(k - 1) * g->G * cf.stride : nullptr;
    a.rho = rho_dev;
    ev_begin(g);
    if (g->m > 0) AD_TRY(dispatch_storage(g, storage, cf, false, a, 0));
    ev_end(g, g->dist_ms, g->dist_launches);
    return AD_OK;
}

}  // namespace ad
