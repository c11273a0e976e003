// api.cu -- the C ABI of include/ad.h: handles, memory, argument checks and
// host/device pointer handling around the kernels of graph.cu, sweep.cu,
// select.cu, multilevel.cu and grad.cu.
#include "ad_internal.cuh"

#include <algorithm>
#include <climits>
#include <cmath>
#include <cstring>
#include <mutex>

namespace ad {

std::atomic<uint64_t> g_launches{0};

static thread_local std::string t_err;

void set_error(const std::string &msg) { t_err = msg; }

ad_status fail(ad_status s, const std::string &msg) {
    t_err = std::string(ad_status_string(s)) + ": " + msg;
    return s;
}

static std::mutex g_alloc_mu;
static Allocator g_alloc;

Allocator current_allocator() {
    std::lock_guard<std::mutex> lk(g_alloc_mu);
    return g_alloc;
}

ad_status dalloc(ad_graph_t g, size_t bytes, void **out) {
    *out = nullptr;
    if (bytes == 0) bytes = 16;
    void *p = nullptr;
    if (g->allocator.alloc) {
        p = g->allocator.alloc(bytes, (void *)g->stream, g->allocator.ctx);
        if (!p) return fail(AD_ERR_OOM, "device allocation of " + std::to_string(bytes) + " bytes failed");
    } else {
        cudaError_t e = cudaMallocAsync(&p, bytes, g->stream);
        if (e != cudaSuccess) {
            cudaGetLastError();
            return fail(AD_ERR_OOM, "cudaMallocAsync(" + std::to_string(bytes) + "): " + cudaGetErrorString(e));
        }
    }
    g->owned.push_back(DevBuf{p, bytes});
    *out = p;
    return AD_OK;
}

static void release(ad_graph_t g, const DevBuf &b) {
    if (g->allocator.release) g->allocator.release(b.ptr, b.bytes, (void *)g->stream, g->allocator.ctx);
    else cudaFreeAsync(b.ptr, g->stream);
}

void dfree(ad_graph_t g, void *p) {
    if (!p) return;
    for (size_t k = g->owned.size(); k-- > 0;) {
        if (g->owned[k].ptr == p) {
            release(g, g->owned[k]);
            g->owned[k] = g->owned.back();
            g->owned.pop_back();
            return;
        }
    }
}

ad_status ensure(ad_graph_t g, DevBuf &b, size_t bytes) {
    if (b.ptr && b.bytes >= bytes) return AD_OK;
    if (b.ptr) dfree(g, b.ptr);
    b = DevBuf();
    void *p = nullptr;
    AD_TRY(dalloc(g, bytes, &p));
    b.ptr = p;
    b.bytes = bytes;
    return AD_OK;
}

bool is_device_ptr(const void *p) {
    if (!p) return false;
    cudaPointerAttributes at;
    cudaError_t e = cudaPointerGetAttributes(&at, p);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

ad_status copy_in(ad_graph_t g, void *dst_dev, const void *src, size_t bytes) {
    if (bytes == 0) return AD_OK;
    AD_CUDA_TRY(cudaMemcpyAsync(dst_dev, src, bytes, cudaMemcpyDefault, g->stream));
    return AD_OK;
}

ad_status copy_out(ad_graph_t g, void *dst, const void *src_dev, size_t bytes) {
    if (bytes == 0) return AD_OK;
    AD_CUDA_TRY(cudaMemcpyAsync(dst, src_dev, bytes, cudaMemcpyDefault, g->stream));
    if (!is_device_ptr(dst)) AD_CUDA_TRY(cudaStreamSynchronize(g->stream));
    return AD_OK;
}

// caller array -> device pointer (the caller's own if already on the device)
static ad_status stage_in(ad_graph_t g, const void *src, size_t bytes, DevBuf &tmp, const void **out) {
    if (is_device_ptr(src)) { *out = src; return AD_OK; }
    AD_TRY(ensure(g, tmp, bytes));
    AD_TRY(copy_in(g, tmp.ptr, src, bytes));
    *out = tmp.ptr;
    return AD_OK;
}

static void destroy_graph(ad_graph_t g);

}  // namespace ad

using namespace ad;

// ----------------------------------------------------------------------------
// Library
// ----------------------------------------------------------------------------
extern "C" const char *ad_version(void) { return "0.1.0"; }

extern "C" const char *ad_status_string(ad_status s) {
    switch (s) {
        case AD_OK: return "AD_OK";
        case AD_ERR_INVALID_ARG: return "AD_ERR_INVALID_ARG";
        case AD_ERR_NOT_SYMMETRIC: return "AD_ERR_NOT_SYMMETRIC";
        case AD_ERR_SELF_LOOP: return "AD_ERR_SELF_LOOP";
        case AD_ERR_DUPLICATE_EDGE: return "AD_ERR_DUPLICATE_EDGE";
        case AD_ERR_BAD_WEIGHT: return "AD_ERR_BAD_WEIGHT";
        case AD_ERR_OOM: return "AD_ERR_OOM";
        case AD_ERR_CUDA: return "AD_ERR_CUDA";
        case AD_ERR_TIMEOUT: return "AD_ERR_TIMEOUT";
        case AD_ERR_STATE: return "AD_ERR_STATE";
        case AD_ERR_BAD_CSR: return "AD_ERR_BAD_CSR";
    }
    return "AD_ERR_UNKNOWN";
}

extern "C" const char *ad_last_error(void) { return t_err.c_str(); }

extern "C" ad_status ad_set_allocator(ad_alloc_fn alloc, ad_free_fn rel, void *ctx) {
    if ((alloc == nullptr) != (rel == nullptr)) return fail(AD_ERR_INVALID_ARG, "alloc and release must both be set or both be NULL");
    std::lock_guard<std::mutex> lk(g_alloc_mu);
    g_alloc.alloc = alloc;
    g_alloc.release = rel;
    g_alloc.ctx = ctx;
    return AD_OK;
}

extern "C" uint64_t ad_kernel_launch_count(void) { return g_launches.load(); }

extern "C" ad_status ad_graph_set_profiling(ad_graph_t g, int32_t enable) {
    if (!g) return fail(AD_ERR_INVALID_ARG, "NULL graph");
    if (enable && !g->ev0) {
        AD_CUDA_TRY(cudaEventCreate(&g->ev0));
        AD_CUDA_TRY(cudaEventCreate(&g->ev1));
    }
    g->profiling = enable != 0;
    return AD_OK;
}

extern "C" ad_status ad_graph_phase_time(ad_graph_t g, const char *phase, double *total_ms, int64_t *launches,
                                         int32_t reset) {
    if (!g || !phase) return fail(AD_ERR_INVALID_ARG, "NULL argument");
    double *ms = nullptr;
    int64_t *cnt = nullptr;
    if (!strcmp(phase, "init")) { ms = &g->init_ms; cnt = &g->init_launches; }
    else if (!strcmp(phase, "sweep")) { ms = &g->sweep_ms; cnt = &g->sweep_launches; }
    else if (!strcmp(phase, "distance")) { ms = &g->dist_ms; cnt = &g->dist_launches; }
    else if (!strcmp(phase, "select")) { ms = &g->select_ms; cnt = &g->select_launches; }
    else return fail(AD_ERR_INVALID_ARG, std::string("unknown phase ") + phase);
    if (total_ms) *total_ms = *ms;
    if (launches) *launches = *cnt;
    if (reset) { *ms = 0; *cnt = 0; }
    return AD_OK;
}

// ----------------------------------------------------------------------------
// Graphs
// ----------------------------------------------------------------------------
namespace ad {
static void drop_replay(ad_graph_t g) {
    if (g->replay.exec) cudaGraphExecDestroy(g->replay.exec);
    g->replay = ad_graph_s::Replay();
}

static void destroy_graph(ad_graph_t g) {
    if (!g) return;
    drop_replay(g);
    if (g->saved) free_saved(g);
    free_sel_cache(g);
    for (auto &b : g->owned) release(g, b);
    g->owned.clear();
    cudaStreamSynchronize(g->stream);
    if (g->ev0) cudaEventDestroy(g->ev0);
    if (g->ev1) cudaEventDestroy(g->ev1);
    delete g;
}

ad_status create_impl(int32_t G, const int64_t *voff, int64_t n, const int64_t *row_ptr, const int32_t *col,
                      const float *weight, int32_t flags, void *stream, ad_graph_t *out) {
    if (!out) return fail(AD_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    if (n < 0 || n > INT32_MAX) return fail(AD_ERR_INVALID_ARG, "n must be in [0, 2^31)");
    if (G < 1 || !voff) return fail(AD_ERR_INVALID_ARG, "need at least one graph");
    if (!row_ptr) return fail(AD_ERR_INVALID_ARG, "row_ptr is NULL");
    if (voff[0] != 0 || voff[G] != n) return fail(AD_ERR_INVALID_ARG, "vertex offsets must run from 0 to n");
    for (int32_t k = 0; k < G; ++k)
        if (voff[k + 1] < voff[k]) return fail(AD_ERR_INVALID_ARG, "vertex offsets must not decrease");
    ad_graph_t g = new ad_graph_s();
    g->n = n;
    g->G = G;
    g->stream = (cudaStream_t)stream;
    g->allocator = current_allocator();
    cudaGetDevice(&g->device);
    cudaDeviceGetAttribute(&g->num_sms, cudaDevAttrMultiProcessorCount, g->device);
    if (g->num_sms <= 0) g->num_sms = kNumSMs;
    g->voff_h.assign(voff, voff + G + 1);
    ad_status st = AD_OK;
    do {
        int64_t nnz = 0;
        st = copy_out(g, &nnz, row_ptr + n, sizeof(int64_t));
        if (st != AD_OK) break;
        if (nnz < 0) { st = fail(AD_ERR_BAD_CSR, "row_ptr[n] < 0"); break; }
        if (nnz > 0 && !col) { st = fail(AD_ERR_INVALID_ARG, "col is NULL"); break; }
        g->nnz = nnz;
        if ((st = dalloc_t(g, n + 1, &g->rp)) != AD_OK) break;
        if ((st = dalloc_t(g, nnz + 1, &g->col)) != AD_OK) break;
        if ((st = copy_in(g, g->rp, row_ptr, (n + 1) * sizeof(int64_t))) != AD_OK) break;
        if ((st = copy_in(g, g->col, col, nnz * sizeof(int32_t))) != AD_OK) break;
        if (weight) {
            if ((st = dalloc_t(g, nnz + 1, &g->w)) != AD_OK) break;
            if ((st = copy_in(g, g->w, weight, nnz * sizeof(float))) != AD_OK) break;
        }
        if ((st = dalloc_t(g, G + 1, &g->voff)) != AD_OK) break;
        if ((st = copy_in(g, g->voff, voff, (G + 1) * sizeof(int64_t))) != AD_OK) break;
        if ((st = graph_setup(g, flags)) != AD_OK) break;
        cudaError_t e = cudaStreamSynchronize(g->stream);
        if (e != cudaSuccess) { st = fail(AD_ERR_CUDA, cudaGetErrorString(e)); break; }
    } while (0);
    if (st != AD_OK) {
        std::string keep = t_err;
        destroy_graph(g);
        t_err = keep;
        return st;
    }
    *out = g;
    return AD_OK;
}
ad_status create_like(ad_graph_t parent, int64_t n, const int64_t *rp_dev, const int32_t *col_dev, const float *w_dev,
                      ad_graph_t *out) {
    const int64_t voff[2] = {0, n};
    return create_impl(1, voff, n, rp_dev, col_dev, w_dev, AD_CREATE_SKIP_VALIDATION, (void *)parent->stream, out);
}
}  // namespace ad

extern "C" ad_status ad_graph_create(int64_t n, const int64_t *row_ptr, const int32_t *col, const float *weight,
                                     int32_t flags, void *stream, ad_graph_t *out) {
    const int64_t voff[2] = {0, n};
    return create_impl(1, voff, n, row_ptr, col, weight, flags, stream, out);
}

extern "C" ad_status ad_graph_create_batched(int32_t n_graphs, const int64_t *vertex_offset, int64_t n,
                                             const int64_t *row_ptr, const int32_t *col, const float *weight,
                                             int32_t flags, void *stream, ad_graph_t *out) {
    if (vertex_offset && is_device_ptr(vertex_offset))
        return fail(AD_ERR_INVALID_ARG, "vertex_offset must be a host array");
    return create_impl(n_graphs, vertex_offset, n, row_ptr, col, weight, flags, stream, out);
}

extern "C" ad_status ad_graph_destroy(ad_graph_t g) {
    destroy_graph(g);
    return AD_OK;
}

extern "C" ad_status ad_graph_info(ad_graph_t g, int64_t *n, int64_t *m, int64_t *nnz, int64_t *n_active,
                                   int32_t *n_graphs) {
    if (!g) return fail(AD_ERR_INVALID_ARG, "NULL graph");
    if (n) *n = g->n;
    if (m) *m = g->m;
    if (nnz) *nnz = g->nnz;
    if (n_active) *n_active = g->n_active;
    if (n_graphs) *n_graphs = g->G;
    return AD_OK;
}

extern "C" ad_status ad_graph_export(ad_graph_t g, int64_t *row_ptr, int32_t *col, float *weight,
                                     int32_t *has_weight) {
    if (!g) return fail(AD_ERR_INVALID_ARG, "NULL graph");
    if (row_ptr) AD_TRY(copy_out(g, row_ptr, g->rp, (g->n + 1) * sizeof(int64_t)));
    if (col) AD_TRY(copy_out(g, col, g->col, g->nnz * sizeof(int32_t)));
    if (weight && g->w) AD_TRY(copy_out(g, weight, g->w, g->nnz * sizeof(float)));
    if (has_weight) *has_weight = g->w ? 1 : 0;
    AD_CUDA_TRY(cudaStreamSynchronize(g->stream));
    return AD_OK;
}

extern "C" ad_status ad_graph_edge_offsets(ad_graph_t g, int64_t *edge_offset) {
    if (!g || !edge_offset) return fail(AD_ERR_INVALID_ARG, "NULL argument");
    memcpy(edge_offset, g->eoff_h.data(), sizeof(int64_t) * (g->G + 1));
    return AD_OK;
}

namespace ad {
__global__ void k_scatter_edge_weights(const int64_t *eid, int64_t nnz, const float *we, float *w,
                                       unsigned long long *bad) {
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < nnz; p += (int64_t)gridDim.x * blockDim.x) {
        const int64_t e = eid[p];
        const float x = we[e];
        if (!(x > 0.f) || !isfinite(x)) atomicMin(bad, (unsigned long long)e);
        w[p] = x;
    }
}
}  // namespace ad

extern "C" ad_status ad_graph_set_edge_weights(ad_graph_t g, const float *w_edge) {
    if (!g || (!w_edge && g->m > 0)) return fail(AD_ERR_INVALID_ARG, "NULL argument");
    AD_TRY(ensure_mirror(g));
    if (!g->w) AD_TRY(dalloc_t(g, g->nnz + 1, &g->w));
    DevBuf tmp;
    const void *src = nullptr;
    AD_TRY(stage_in(g, w_edge, g->m * sizeof(float), tmp, &src));
    unsigned long long *bad = nullptr;
    AD_TRY(dalloc_t(g, 1, &bad));
    AD_CUDA_TRY(cudaMemsetAsync(bad, 0xff, sizeof(unsigned long long), g->stream));
    if (g->nnz > 0)
        AD_LAUNCH(k_scatter_edge_weights, g->num_sms * 16, 256, 0, g->stream, g->eid, g->nnz, (const float *)src, g->w,
                  bad);
    unsigned long long b = 0;
    AD_TRY(copy_out(g, &b, bad, sizeof(b)));
    dfree(g, bad);
    if (tmp.ptr) dfree(g, tmp.ptr);
    if (b != ~0ull) return fail(AD_ERR_BAD_WEIGHT, "edge weight " + std::to_string(b) + " not positive and finite");
    AD_TRY(recompute_degrees(g));
    g->have_rho = false;
    g->rho_version++;
    return AD_OK;
}

// ----------------------------------------------------------------------------
// Algebraic distance
// ----------------------------------------------------------------------------
// A call that repeats the previous one (same parameters, same scratch
// buffers) replays the launch sequence recorded from it as a CUDA graph: one
// graph launch instead of 2k + 3 kernel launches, which is what bounds small
// graphs.  The first call of a kind runs (and sizes every buffer) directly,
// the second is captured, later ones replay.  Streams that cannot be captured
// (the legacy default stream) and profiled handles always run directly.
static void replay_ptrs(ad_graph_t g, const void **p) {
    p[0] = g->x0.ptr; p[1] = g->x1.ptr; p[2] = g->mm.ptr; p[3] = g->ac.ptr; p[4] = g->part.ptr; p[5] = g->rho;
    p[6] = g->sweep_plans.empty() ? nullptr : (const void *)&g->sweep_plans.front();
}

static ad_status distance_replayed(ad_graph_t g, int32_t R, int32_t k, double omega, uint64_t seed,
                                   uint32_t stream_id, ad_storage storage, int32_t flags) {
    auto &rp = g->replay;
    if (g->profiling)   // per-phase events need the direct launches
        return algebraic_distance(g, R, k, omega, seed, stream_id, storage, flags, g->rho);
    const void *now[7];
    replay_ptrs(g, now);
    const bool same = rp.have_key && rp.R == R && rp.k == k && rp.omega == omega && rp.seed == seed &&
                      rp.stream_id == stream_id && rp.storage == (int32_t)storage && rp.flags == flags &&
                      std::equal(now, now + 7, rp.ptrs);
    const bool capturable = g->stream != nullptr && g->stream != cudaStreamLegacy;
    if (same && rp.exec) {
        AD_CUDA_TRY(cudaGraphLaunch(rp.exec, g->stream));
        g_launches.fetch_add(rp.launches, std::memory_order_relaxed);
        return AD_OK;
    }
    if (same && capturable) {
        cudaGraph_t graph = nullptr;
        const uint64_t l0 = g_launches.load();
        AD_CUDA_TRY(cudaStreamBeginCapture(g->stream, cudaStreamCaptureModeThreadLocal));
        const ad_status st = algebraic_distance(g, R, k, omega, seed, stream_id, storage, flags, g->rho);
        const cudaError_t ce = cudaStreamEndCapture(g->stream, &graph);
        cudaGetLastError();
        const void *after[7];
        replay_ptrs(g, after);
        cudaGraphExec_t exec = nullptr;
        if (st == AD_OK && ce == cudaSuccess && graph && std::equal(after, after + 7, now) &&
            cudaGraphInstantiate(&exec, graph, 0) == cudaSuccess) {
            cudaGraphDestroy(graph);
            rp.exec = exec;
            rp.launches = g_launches.load() - l0;
            g_launches.fetch_sub(rp.launches, std::memory_order_relaxed);   // counted when they run
            AD_CUDA_TRY(cudaGraphLaunch(rp.exec, g->stream));
            g_launches.fetch_add(rp.launches, std::memory_order_relaxed);
            return AD_OK;
        }
        if (graph) cudaGraphDestroy(graph);
        cudaGetLastError();
        drop_replay(g);      // could not record it: run it directly
    }
    if (rp.exec) drop_replay(g);
    AD_TRY(algebraic_distance(g, R, k, omega, seed, stream_id, storage, flags, g->rho));
    rp.have_key = true;
    rp.R = R; rp.k = k; rp.omega = omega; rp.seed = seed; rp.stream_id = stream_id;
    rp.storage = (int32_t)storage; rp.flags = flags;
    replay_ptrs(g, rp.ptrs);
    return AD_OK;
}
extern "C" ad_status ad_algebraic_distance(ad_graph_t g, int32_t R, int32_t k, double omega, uint64_t seed,
                                           uint32_t stream_id, ad_storage storage, int32_t flags, float *rho_out) {
    if (!g) return fail(AD_ERR_INVALID_ARG, "NULL graph");
    if (R < 1 || R > 256) return fail(AD_ERR_INVALID_ARG, "R must be in [1, 256]");
    if (k < 0) return fail(AD_ERR_INVALID_ARG, "k must be >= 0");
    if (!(omega > 0.0 && omega <= 1.0)) return fail(AD_ERR_INVALID_ARG, "omega must be in (0, 1]");
    if (storage < AD_STORAGE_FP32 || storage > AD_STORAGE_Q16) return fail(AD_ERR_INVALID_ARG, "bad storage");
    if (flags & ~(AD_DIST_NORMALIZE | AD_DIST_KEEP_STATE | AD_DIST_PERSISTENT | AD_DIST_SQRT_CHECKPOINTS))
        return fail(AD_ERR_INVALID_ARG, "unknown flags");
    if ((flags & AD_DIST_KEEP_STATE) && (storage != AD_STORAGE_FP32 || (flags & AD_DIST_NORMALIZE)))
        return fail(AD_ERR_INVALID_ARG, "kept state needs FP32 storage and no normalisation");
    if (!g->rho) AD_TRY(dalloc_t(g, g->m + 1, &g->rho));
    g->have_rho = false;
    g->rho_version++;
    if (flags & AD_DIST_KEEP_STATE)
        AD_TRY(algebraic_distance_keep(g, R, k, omega, seed, stream_id, g->rho, (flags & AD_DIST_SQRT_CHECKPOINTS) != 0));
    else AD_TRY(distance_replayed(g, R, k, omega, seed, stream_id, storage, flags));
    g->have_rho = true;
    g->rho_version++;
    if (rho_out) AD_TRY(copy_out(g, rho_out, g->rho, g->m * sizeof(float)));
    return AD_OK;
}

// ----------------------------------------------------------------------------
// Autotuning of the sweep shape
// ----------------------------------------------------------------------------
extern "C" ad_status ad_graph_autotune(ad_graph_t g, int32_t R, ad_storage storage, int32_t *lanes_per_row,
                                       int32_t *chunks_per_lane, int32_t *ctas_per_sm) {
    if (!g) return fail(AD_ERR_INVALID_ARG, "NULL graph");
    if (R < 1 || R > 256) return fail(AD_ERR_INVALID_ARG, "R must be in [1, 256]");
    if (storage < AD_STORAGE_FP32 || storage > AD_STORAGE_Q16) return fail(AD_ERR_INVALID_ARG, "bad storage");
    drop_replay(g);   // a recorded launch sequence holds the old shape
    auto &tv = g->tuned;
    tv.erase(std::remove_if(tv.begin(), tv.end(),
                            [&](const ad_graph_s::Tuned &t) { return t.R == R && t.storage == (int32_t)storage; }),
             tv.end());
    int nat_lpr = 1, nat_cpl = 1;
    natural_shape(R, storage, &nat_lpr, &nat_cpl);
    struct Cand { int lpr, cpl, per_sm; };
    std::vector<Cand> cands;
    std::vector<std::pair<int, int>> shapes = {{nat_lpr, nat_cpl}};
    if (nat_lpr >= 2 && nat_cpl == 1) shapes.push_back({nat_lpr / 2, 2});
    for (const auto &sh : shapes)
        for (int per_sm : {0, 5, 4}) cands.push_back({sh.first, sh.second, per_sm});
    int best = 0;
    float best_ms = 0.f;
    if (g->m > 0) {
        float *rho = nullptr;
        AD_TRY(dalloc_t(g, g->m + 1, &rho));
        cudaEvent_t e0, e1;
        AD_CUDA_TRY(cudaEventCreate(&e0));
        AD_CUDA_TRY(cudaEventCreate(&e1));
        const bool prof = g->profiling;
        g->profiling = false;
        ad_status st = AD_OK;
        for (size_t c = 0; c < cands.size() && st == AD_OK; ++c) {
            tv.push_back({R, (int32_t)storage, cands[c].lpr, cands[c].cpl, cands[c].per_sm});
            float t_best = 0.f;
            for (int rep = 0; rep < 3 && st == AD_OK; ++rep) {   // the first run builds the row plans
                cudaEventRecord(e0, g->stream);
                st = algebraic_distance(g, R, 4, 0.5, 1, 0, storage, 0, rho);
                cudaEventRecord(e1, g->stream);
                if (cudaEventSynchronize(e1) != cudaSuccess) st = fail(AD_ERR_CUDA, "autotune timing");
                float ms = 0.f;
                cudaEventElapsedTime(&ms, e0, e1);
                if (rep > 0 && (rep == 1 || ms < t_best)) t_best = ms;
            }
            tv.pop_back();
            if (st == AD_OK && (c == 0 || t_best < best_ms)) {
                best = (int)c;
                best_ms = t_best;
            }
        }
        g->profiling = prof;
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        dfree(g, rho);
        AD_TRY(st);
    }
    tv.push_back({R, (int32_t)storage, cands[best].lpr, cands[best].cpl, cands[best].per_sm});
    if (lanes_per_row) *lanes_per_row = cands[best].lpr;
    if (chunks_per_lane) *chunks_per_lane = cands[best].cpl;
    if (ctas_per_sm) *ctas_per_sm = cands[best].per_sm;
    return AD_OK;
}

// ----------------------------------------------------------------------------
// Ranking and sampling
// ----------------------------------------------------------------------------
namespace ad {
static ad_status sparsify_impl(ad_graph_t g, const float *score_dev, double fraction, ad_mode mode, ad_scope scope,
                               uint8_t *keep_out, int64_t *n_kept, double *e_used) {
    if (!(fraction >= 0.0 && fraction <= 1.0)) return fail(AD_ERR_INVALID_ARG, "fraction must be in [0, 1]");
    if (mode != AD_MODE_LOCAL && mode != AD_MODE_GLOBAL) return fail(AD_ERR_INVALID_ARG, "bad mode");
    if (scope != AD_SCOPE_PER_NODE && scope != AD_SCOPE_WHOLE_GRAPH) return fail(AD_ERR_INVALID_ARG, "bad scope");
    if (!keep_out && g->m > 0) return fail(AD_ERR_INVALID_ARG, "keep_out is NULL");
    const bool dev_out = is_device_ptr(keep_out);
    uint8_t *kd = keep_out;
    DevBuf tmp;
    if (!dev_out) {
        AD_TRY(ensure(g, tmp, g->m + 16));
        kd = static_cast<uint8_t *>(tmp.ptr);
    }
    if (g->profiling) cudaEventRecord(g->ev0, g->stream);
    int64_t kept = 0;
    double e = -1.0;
    if (scope == AD_SCOPE_WHOLE_GRAPH) AD_TRY(select_whole_graph(g, score_dev, fraction, mode, kd, &kept));
    else AD_TRY(select_per_node_fit(g, score_dev, fraction, mode, kd, &kept, &e));
    if (g->profiling) {
        cudaEventRecord(g->ev1, g->stream);
        cudaEventSynchronize(g->ev1);
        float ms = 0;
        cudaEventElapsedTime(&ms, g->ev0, g->ev1);
        g->select_ms += ms;
        g->select_launches += 1;
    }
    if (!dev_out) AD_TRY(copy_out(g, keep_out, kd, g->m));
    if (tmp.ptr) dfree(g, tmp.ptr);
    if (n_kept) *n_kept = kept;
    if (e_used) *e_used = e;
    return AD_OK;
}
}  // namespace ad

extern "C" ad_status ad_sparsify(ad_graph_t g, double fraction, ad_mode mode, ad_scope scope, uint8_t *keep_out,
                                 int64_t *n_kept, double *e_used) {
    if (!g) return fail(AD_ERR_INVALID_ARG, "NULL graph");
    if (!g->have_rho) return fail(AD_ERR_STATE, "no distances: call ad_algebraic_distance first");
    return sparsify_impl(g, g->rho, fraction, mode, scope, keep_out, n_kept, e_used);
}

extern "C" ad_status ad_sparsify_local_global(ad_graph_t g, double fraction, uint8_t *keep_local,
                                              uint8_t *keep_global, int64_t *n_kept, double *e_used) {
    if (!g) return fail(AD_ERR_INVALID_ARG, "NULL graph");
    if (!g->have_rho) return fail(AD_ERR_STATE, "no distances: call ad_algebraic_distance first");
    if (!(fraction >= 0.0 && fraction <= 1.0)) return fail(AD_ERR_INVALID_ARG, "fraction must be in [0, 1]");
    if ((!keep_local || !keep_global) && g->m > 0) return fail(AD_ERR_INVALID_ARG, "keep_local or keep_global is NULL");
    uint8_t *out[2] = {keep_local, keep_global}, *kd[2] = {keep_local, keep_global};
    DevBuf tmp[2];
    ad_status st = AD_OK;
    for (int s = 0; s < 2 && st == AD_OK; ++s)
        if (g->m > 0 && !is_device_ptr(out[s])) {
            st = ensure(g, tmp[s], g->m + 16);
            kd[s] = static_cast<uint8_t *>(tmp[s].ptr);
        }
    int64_t kept[2] = {0, 0};
    double e[2] = {-1.0, -1.0};
    if (g->profiling) cudaEventRecord(g->ev0, g->stream);
    if (st == AD_OK) st = select_per_node_fit_both(g, g->rho, fraction, kd[0], kd[1], kept, e);
    if (st == AD_OK && g->profiling) {
        cudaEventRecord(g->ev1, g->stream);
        cudaEventSynchronize(g->ev1);
        float ms = 0;
        cudaEventElapsedTime(&ms, g->ev0, g->ev1);
        g->select_ms += ms;
        g->select_launches += 1;
    }
    for (int s = 0; s < 2 && st == AD_OK; ++s)
        if (kd[s] != out[s]) st = copy_out(g, out[s], kd[s], g->m);
    for (DevBuf &b : tmp)
        if (b.ptr) dfree(g, b.ptr);
    if (st != AD_OK) return st;
    for (int s = 0; s < 2; ++s) {
        if (n_kept) n_kept[s] = kept[s];
        if (e_used) e_used[s] = e[s];
    }
    return AD_OK;
}

extern "C" ad_status ad_sparsify_scores(ad_graph_t g, const float *score, double fraction, ad_mode mode,
                                        ad_scope scope, uint8_t *keep_out, int64_t *n_kept, double *e_used) {
    if (!g) return fail(AD_ERR_INVALID_ARG, "NULL graph");
    if (!score && g->m > 0) return fail(AD_ERR_INVALID_ARG, "score is NULL");
    DevBuf tmp;
    const void *sd = nullptr;
    AD_TRY(stage_in(g, score, g->m * sizeof(float), tmp, &sd));
    ad_status st = check_scores(g, (const float *)sd);
    if (st == AD_OK) st = sparsify_impl(g, (const float *)sd, fraction, mode, scope, keep_out, n_kept, e_used);
    if (tmp.ptr) dfree(g, tmp.ptr);
    return st;
}

extern "C" ad_status ad_sparsify_binned(ad_graph_t g, const float *score, double fraction, uint64_t seed,
                                        uint8_t *keep_out, int64_t *n_kept, double *e_used) {
    if (!g) return fail(AD_ERR_INVALID_ARG, "NULL graph");
    if (!(fraction >= 0.0 && fraction <= 1.0)) return fail(AD_ERR_INVALID_ARG, "fraction must be in [0, 1]");
    if (!keep_out && g->m > 0) return fail(AD_ERR_INVALID_ARG, "keep_out is NULL");
    DevBuf tmp_s, tmp_k, ranks;
    const float *sd = g->rho;
    if (score) {
        const void *p = nullptr;
        AD_TRY(stage_in(g, score, g->m * sizeof(float), tmp_s, &p));
        sd = static_cast<const float *>(p);
        AD_TRY(check_scores(g, sd));
    } else if (!g->have_rho) {
        return fail(AD_ERR_STATE, "no distances: call ad_algebraic_distance first or pass scores");
    }
    const bool dev_out = is_device_ptr(keep_out);
    uint8_t *kd = keep_out;
    if (!dev_out) {
        AD_TRY(ensure(g, tmp_k, g->m + 16));
        kd = static_cast<uint8_t *>(tmp_k.ptr);
    }
    int64_t kept = 0;
    double e = -1.0;
    ad_status st = ensure(g, ranks, sizeof(uint32_t) * (g->nnz + 1));
    if (st == AD_OK) st = binned_ranks(g, sd, seed, static_cast<uint32_t *>(ranks.ptr));
    if (st == AD_OK) st = select_per_node_fit_ranked(g, static_cast<const uint32_t *>(ranks.ptr), fraction, kd, &kept, &e);
    if (st == AD_OK && !dev_out) st = copy_out(g, keep_out, kd, g->m);
    for (DevBuf *b : {&tmp_s, &tmp_k, &ranks})
        if (b->ptr) dfree(g, b->ptr);
    if (st != AD_OK) return st;
    if (n_kept) *n_kept = kept;
    if (e_used) *e_used = e;
    return AD_OK;
}

extern "C" ad_status ad_binned_ranks(ad_graph_t g, const float *score, uint64_t seed, uint32_t *rank_out,
                                     uint32_t *bin_out) {
    if (!g) return fail(AD_ERR_INVALID_ARG, "NULL graph");
    if (!rank_out && g->nnz > 0) return fail(AD_ERR_INVALID_ARG, "rank_out is NULL");
    if (g->nnz == 0) return AD_OK;
    DevBuf tmp_s, ranks, bins;
    const float *sd = g->rho;
    if (score) {
        const void *p = nullptr;
        AD_TRY(stage_in(g, score, g->m * sizeof(float), tmp_s, &p));
        sd = static_cast<const float *>(p);
        AD_TRY(check_scores(g, sd));
    } else if (!g->have_rho) {
        return fail(AD_ERR_STATE, "no distances: call ad_algebraic_distance first or pass scores");
    }
    const size_t bytes = sizeof(uint32_t) * g->nnz;
    ad_status st = ensure(g, ranks, bytes + 16);
    if (st == AD_OK && bin_out) st = ensure(g, bins, bytes + 16);
    if (st == AD_OK)
        st = binned_ranks(g, sd, seed, static_cast<uint32_t *>(ranks.ptr),
                          bin_out ? static_cast<uint32_t *>(bins.ptr) : nullptr);
    if (st == AD_OK) st = copy_out(g, rank_out, ranks.ptr, bytes);
    if (st == AD_OK && bin_out) st = copy_out(g, bin_out, bins.ptr, bytes);
    for (DevBuf *b : {&tmp_s, &ranks, &bins})
        if (b->ptr) dfree(g, b->ptr);
    return st;
}

extern "C" ad_status ad_sparsify_local_degree(ad_graph_t g, double fraction, uint8_t *keep_out, int64_t *n_kept,
                                              double *e_used) {
    if (!g) return fail(AD_ERR_INVALID_ARG, "NULL graph");
    if (!(fraction >= 0.0 && fraction <= 1.0)) return fail(AD_ERR_INVALID_ARG, "fraction must be in [0, 1]");
    if (!keep_out && g->m > 0) return fail(AD_ERR_INVALID_ARG, "keep_out is NULL");
    const bool dev_out = is_device_ptr(keep_out);
    DevBuf tmp;
    uint8_t *kd = keep_out;
    if (!dev_out) {
        AD_TRY(ensure(g, tmp, g->m + 16));
        kd = static_cast<uint8_t *>(tmp.ptr);
    }
    int64_t kept = 0;
    double e = -1.0;
    ad_status st = select_local_degree(g, fraction, kd, &kept, &e);
    if (st == AD_OK && !dev_out) st = copy_out(g, keep_out, kd, g->m);
    if (tmp.ptr) dfree(g, tmp.ptr);
    if (st != AD_OK) return st;
    if (n_kept) *n_kept = kept;
    if (e_used) *e_used = e;
    return AD_OK;
}

extern "C" ad_status ad_select_per_node(ad_graph_t g, const float *score, double e, ad_mode mode, uint8_t *keep_out,
                                        int64_t *n_kept) {
    if (!g) return fail(AD_ERR_INVALID_ARG, "NULL graph");
    if (!(e >= 0.0 && e <= 1.0)) return fail(AD_ERR_INVALID_ARG, "e must be in [0, 1]");
    if (mode != AD_MODE_LOCAL && mode != AD_MODE_GLOBAL) return fail(AD_ERR_INVALID_ARG, "bad mode");
    DevBuf tmp_s, tmp_k;
    const float *sd = g->rho;
    if (score) {
        const void *p = nullptr;
        AD_TRY(stage_in(g, score, g->m * sizeof(float), tmp_s, &p));
        sd = (const float *)p;
        AD_TRY(check_scores(g, sd));
    } else if (!g->have_rho) {
        return fail(AD_ERR_STATE, "no distances: call ad_algebraic_distance first or pass scores");
    }
    uint8_t *kd = keep_out;
    const bool dev_out = keep_out && is_device_ptr(keep_out);
    if (!dev_out) {
        AD_TRY(ensure(g, tmp_k, g->m + 16));
        kd = static_cast<uint8_t *>(tmp_k.ptr);
    }
    int64_t kept = 0;
    AD_TRY(select_per_node_at(g, sd, e, mode, kd, &kept));
    if (keep_out && !dev_out) AD_TRY(copy_out(g, keep_out, kd, g->m));
    if (tmp_s.ptr) dfree(g, tmp_s.ptr);
    if (tmp_k.ptr) dfree(g, tmp_k.ptr);
    if (n_kept) *n_kept = kept;
    return AD_OK;
}
