// ad_internal.cuh -- shared declarations of the sm_103a library (device helpers,
// handle layout, kernel entry points).  Not part of the public ABI (include/ad.h).
#pragma once

#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <stdint.h>

#include <atomic>
#include <string>
#include <vector>

#include "../../include/ad.h"

// ----------------------------------------------------------------------------
// Errors
// ----------------------------------------------------------------------------
namespace ad {

void set_error(const std::string &msg);
ad_status fail(ad_status s, const std::string &msg);

extern std::atomic<uint64_t> g_launches;

}  // namespace ad

#define AD_CUDA_TRY(expr)                                                                  \
    do {                                                                                   \
        cudaError_t _e = (expr);                                                           \
        if (_e != cudaSuccess)                                                             \
            return ::ad::fail(_e == cudaErrorMemoryAllocation ? AD_ERR_OOM : AD_ERR_CUDA,  \
                              std::string(#expr) + ": " + cudaGetErrorString(_e));         \
    } while (0)

#define AD_TRY(expr)                        \
    do {                                    \
        ad_status _s = (expr);              \
        if (_s != AD_OK) return _s;         \
    } while (0)

// Launch helper: counts launches and checks the launch error.
#define AD_LAUNCH(kernel, grid, block, smem, stream, ...)                                  \
    do {                                                                                   \
        ::ad::g_launches.fetch_add(1, std::memory_order_relaxed);                          \
        kernel<<<(grid), (block), (smem), (stream)>>>(__VA_ARGS__);                        \
        cudaError_t _le = cudaGetLastError();                                              \
        if (_le != cudaSuccess)                                                            \
            return ::ad::fail(AD_ERR_CUDA, std::string("launch " #kernel ": ") +           \
                                               cudaGetErrorString(_le));                   \
    } while (0)

namespace ad {

constexpr int kNumSMs = 152;  // GB300; the runtime value is queried, this is a default
// single graphs with at most this many CSR entries are relaxed in one persistent launch
// without being asked (AD_DIST_PERSISTENT).  Measured on GB300, per-sweep launches
// replayed as a CUDA graph are faster for every size tried (the persistent kernel
// must read the vectors past L1), so none are by default.
#ifndef AD_PERSIST_MAX_NNZ
#define AD_PERSIST_MAX_NNZ 0
#endif
constexpr int64_t kPersistMaxNnz = AD_PERSIST_MAX_NNZ;

// ----------------------------------------------------------------------------
// Device helpers
// ----------------------------------------------------------------------------

// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11): ten rounds; each round
// multiplies counter words 0 and 2 by the two round multipliers, swaps the
// halves and xors in the key, which is advanced by the Weyl increments.
__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint2 k) {
#pragma unroll
    for (int round = 0; round < 10; ++round) {
        const uint32_t lo0 = 0xD2511F53u * c.x;
        const uint32_t hi0 = __umulhi(0xD2511F53u, c.x);
        const uint32_t lo1 = 0xCD9E8D57u * c.z;
        const uint32_t hi1 = __umulhi(0xCD9E8D57u, c.z);
        c = make_uint4(hi1 ^ c.y ^ k.x, lo1, hi0 ^ c.w ^ k.y, lo0);
        k.x += 0x9E3779B9u;
        k.y += 0xBB67AE85u;
    }
    return c;
}

// rand(-0.5, 0.5) of Alg. 1: top 24 bits of a Philox word on the 2^-24 grid.
__device__ __forceinline__ float unit_centered(uint32_t u) {
    return __uint2float_rn(u >> 8) * 5.9604644775390625e-8f - 0.5f;
}

// Order-preserving map float -> uint32 (for atomic min/max on floats).
__device__ __forceinline__ uint32_t f2ord(float f) {
    uint32_t b = __float_as_uint(f);
    return (b & 0x80000000u) ? ~b : (b | 0x80000000u);
}
__host__ __device__ __forceinline__ float ord2f(uint32_t o) {
    uint32_t b = (o & 0x80000000u) ? (o & 0x7fffffffu) : ~o;
#ifdef __CUDA_ARCH__
    return __uint_as_float(b);
#else
    float f;
    memcpy(&f, &b, 4);
    return f;
#endif
}

// Storage type traits: 16-byte chunk of V elements <-> V floats.
template <typename T> struct Store;
template <> struct Store<float> {
    static constexpr int V = 4;
    __device__ __forceinline__ static void unpack(const uint4 &q, float *f) {
        f[0] = __uint_as_float(q.x); f[1] = __uint_as_float(q.y);
        f[2] = __uint_as_float(q.z); f[3] = __uint_as_float(q.w);
    }
    __device__ __forceinline__ static uint4 pack(const float *f) {
        return make_uint4(__float_as_uint(f[0]), __float_as_uint(f[1]), __float_as_uint(f[2]),
                          __float_as_uint(f[3]));
    }
    // value as stored (identity for FP32)
    __device__ __forceinline__ static float round(float f) { return f; }
};
template <> struct Store<__nv_bfloat16> {
    static constexpr int V = 8;
    __device__ __forceinline__ static void unpack2(uint32_t w, float &lo, float &hi) {
        lo = __uint_as_float(w << 16);
        hi = __uint_as_float(w & 0xffff0000u);
    }
    __device__ __forceinline__ static void unpack(const uint4 &q, float *f) {
        unpack2(q.x, f[0], f[1]); unpack2(q.y, f[2], f[3]);
        unpack2(q.z, f[4], f[5]); unpack2(q.w, f[6], f[7]);
    }
    __device__ __forceinline__ static uint32_t pack2(float lo, float hi) {
        __nv_bfloat162 h = __floats2bfloat162_rn(lo, hi);   // round to nearest even
        return *reinterpret_cast<uint32_t *>(&h);
    }
    __device__ __forceinline__ static uint4 pack(const float *f) {
        return make_uint4(pack2(f[0], f[1]), pack2(f[2], f[3]), pack2(f[4], f[5]), pack2(f[6], f[7]));
    }
    __device__ __forceinline__ static float round(float f) {
        return __bfloat162float(__float2bfloat16_rn(f));
    }
};

template <> struct Store<__half> {
    static constexpr int V = 8;
    __device__ __forceinline__ static void unpack2(uint32_t w, float &lo, float &hi) {
        const float2 f = __half22float2(*reinterpret_cast<const __half2 *>(&w));
        lo = f.x;
        hi = f.y;
    }
    __device__ __forceinline__ static void unpack(const uint4 &q, float *f) {
        unpack2(q.x, f[0], f[1]); unpack2(q.y, f[2], f[3]);
        unpack2(q.z, f[4], f[5]); unpack2(q.w, f[6], f[7]);
    }
    __device__ __forceinline__ static uint32_t pack2(float lo, float hi) {
        __half2 h = __floats2half2_rn(lo, hi);
        return *reinterpret_cast<uint32_t *>(&h);
    }
    __device__ __forceinline__ static uint4 pack(const float *f) {
        return make_uint4(pack2(f[0], f[1]), pack2(f[2], f[3]), pack2(f[4], f[5]), pack2(f[6], f[7]));
    }
    __device__ __forceinline__ static float round(float f) { return __half2float(__float2half_rn(f)); }
};

// 16-bit fixed point: q in [-32768, 32767] stands for q * 2^-15 (covers [-1, 1);
// every stored value of a sweep lies in [-1, 1]).
struct Q16 {
    int16_t q;
};
template <> struct Store<Q16> {
    static constexpr int V = 8;
    static constexpr float kStep = 3.0517578125e-5f;   // 2^-15
    __device__ __forceinline__ static void unpack2(uint32_t w, float &lo, float &hi) {
        lo = (float)((int32_t)(w << 16) >> 16) * kStep;
        hi = (float)((int32_t)w >> 16) * kStep;
    }
    __device__ __forceinline__ static void unpack(const uint4 &q, float *f) {
        unpack2(q.x, f[0], f[1]); unpack2(q.y, f[2], f[3]);
        unpack2(q.z, f[4], f[5]); unpack2(q.w, f[6], f[7]);
    }
    __device__ __forceinline__ static int32_t code(float f) {
        const int32_t c = __float2int_rn(f * 32768.0f);
        return c < -32768 ? -32768 : (c > 32767 ? 32767 : c);
    }
    __device__ __forceinline__ static uint32_t pack2(float lo, float hi) {
        return ((uint32_t)code(lo) & 0xffffu) | ((uint32_t)code(hi) << 16);
    }
    __device__ __forceinline__ static uint4 pack(const float *f) {
        return make_uint4(pack2(f[0], f[1]), pack2(f[2], f[3]), pack2(f[4], f[5]), pack2(f[6], f[7]));
    }
    __device__ __forceinline__ static float round(float f) { return (float)code(f) * kStep; }
};

// ----------------------------------------------------------------------------
// Device memory owned by a handle
// ----------------------------------------------------------------------------
struct Allocator {
    ad_alloc_fn alloc = nullptr;
    ad_free_fn release = nullptr;
    void *ctx = nullptr;
};
Allocator current_allocator();

struct DevBuf {
    void *ptr = nullptr;
    size_t bytes = 0;
};

// ----------------------------------------------------------------------------
// Work plan of the row-parallel kernels (sweep, distance).  Rows of degree
// > 0 are split into three task kinds processed by one warp each:
//   big    a chunk of <= kChunk neighbours of a row of degree > kBig; the
//          chunks of one row are consecutive tasks and the last one to finish
//          combines their partial sums (fixed order) and writes the row;
//   medium one row of degree in (small_max, kBig];
//   small  `groups` rows of degree <= small_max, one per lane group.
// Big tasks come first, then medium rows by decreasing degree class, then
// small rows, so that warps striding over the task list meet similar work.
// ----------------------------------------------------------------------------
#ifndef AD_CHUNK
#define AD_CHUNK 512
#endif
constexpr int kChunk = AD_CHUNK;
constexpr int kBig = AD_CHUNK;

struct RowPlan {
    int small_max = 0;          // degree bound of the small class
    int groups = 0;             // lane groups per warp the plan was built for
    int64_t n_big = 0;          // big chunk tasks
    int64_t n_medium = 0;
    int64_t n_small_rows = 0;
    int32_t *big_row = nullptr;     // [n_big]
    int32_t *big_chunk = nullptr;   // [n_big]
    int32_t *medium_row = nullptr;  // [n_medium]
    int32_t *small_row = nullptr;   // [n_small_rows]
    uint32_t *big_counter = nullptr;  // [n_big], zero between launches
    bool upper_only = false;
    int64_t tasks() const {
        return n_big + n_medium + (n_small_rows + groups - 1) / (groups > 0 ? groups : 1);
    }
};

}  // namespace ad

struct ad_graph_s {
    int64_t n = 0, nnz = 0, m = 0, n_active = 0;
    int32_t G = 1;
    cudaStream_t stream = nullptr;
    int device = 0;
    int num_sms = ad::kNumSMs;
    ad::Allocator allocator;
    std::vector<ad::DevBuf> owned;

    // CSR on the device
    int64_t *rp = nullptr;
    int32_t *col = nullptr;
    float *w = nullptr;          // nullptr = unit weights
    double *D = nullptr;         // weighted degree (FP64)
    uint8_t *dexact = nullptr;   // [n] weighted graphs: 1 where every partial sum of the row's weights is exact in FP64
    float *Dinv = nullptr;       // 1 / D (0 for isolated vertices)
    int64_t *upos = nullptr;     // first CSR position of row i with col > i
    int64_t *eoff = nullptr;     // edge id of that position; eoff[n] = m
    int64_t *mirror = nullptr;   // [nnz] position of the reverse entry (built lazily)
    int32_t *erow = nullptr;     // [nnz] row of each entry (built lazily)
    int64_t *eid = nullptr;      // [nnz] edge id of each entry (built lazily)
    int32_t *deg_class = nullptr;  // [n] index of the row's degree among distinct degrees (lazy)
    int32_t n_deg_classes = 0;
    std::vector<int64_t> distinct_degrees;  // host copy, ascending

    // batches
    std::vector<int64_t> voff_h, eoff_h;   // vertex / edge offsets per graph (host)
    int64_t *voff = nullptr;               // device copies
    int32_t *anchor = nullptr;             // [G] vertex of largest weighted degree of each graph
    int64_t *goff_e = nullptr;

    // work plans keyed by lane-group count
    std::vector<ad::RowPlan> sweep_plans, dist_plans;

    // scores of the last ad_algebraic_distance call
    float *rho = nullptr;
    bool have_rho = false;
    uint64_t rho_version = 0;    // bumped whenever rho is recomputed

    // cached scratch
    ad::DevBuf x0, x1, part, mm, ws, ac, relax_sync;

    // profiling
    bool profiling = false;
    double sweep_ms = 0, dist_ms = 0, init_ms = 0, select_ms = 0;
    int64_t sweep_launches = 0, dist_launches = 0, init_launches = 0, select_launches = 0;
    cudaEvent_t ev0 = nullptr, ev1 = nullptr;

    // state kept for the backward pass
    struct Saved;
    Saved *saved = nullptr;

    // cached selection workspace (select.cu) and scan workspace (graph.cu)
    struct SelCache;
    SelCache *sel = nullptr;
    ad::DevBuf scan_ws;

    // sweep shapes chosen by ad_graph_autotune, per (R, storage)
    struct Tuned {
        int32_t R, storage, lpr, cpl, per_sm;
    };
    std::vector<Tuned> tuned;

    // CUDA graph of the launch sequence of a repeated ad_algebraic_distance call
    struct Replay {
        bool have_key = false;      // key / ptrs describe the last call
        int32_t R = 0, k = 0, flags = 0;
        double omega = 0;
        uint64_t seed = 0;
        uint32_t stream_id = 0;
        int32_t storage = 0;
        const void *ptrs[7] = {};   // scratch the launches read or write (x0, x1, mm, ac, part, rho, plans)
        cudaGraphExec_t exec = nullptr;
        uint64_t launches = 0;      // kernels in the graph
    } replay;
};

namespace ad {

// memory helpers (graph-owned allocations are released by ad_graph_destroy)
ad_status dalloc(ad_graph_t g, size_t bytes, void **out);
template <typename T> ad_status dalloc_t(ad_graph_t g, size_t count, T **out) {
    void *p = nullptr;
    ad_status s = dalloc(g, count * sizeof(T) + 16, &p);
    *out = static_cast<T *>(p);
    return s;
}
void dfree(ad_graph_t g, void *p);
ad_status ensure(ad_graph_t g, DevBuf &b, size_t bytes);

// pointer classification
bool is_device_ptr(const void *p);

// copy helpers between caller memory (host or device) and device buffers
ad_status copy_in(ad_graph_t g, void *dst_dev, const void *src, size_t bytes);
ad_status copy_out(ad_graph_t g, void *dst, const void *src_dev, size_t bytes);

// scans
ad_status exclusive_scan_i64(ad_graph_t g, const int64_t *in, int64_t *out, int64_t n, int64_t *total_host);

// graph setup (graph.cu)
ad_status graph_setup(ad_graph_t g, int32_t flags);
ad_status build_row_plan(ad_graph_t g, int groups, int small_max, bool upper_only, RowPlan &plan);
ad_status ensure_mirror(ad_graph_t g);   // also builds erow and eid
ad_status ensure_degree_classes(ad_graph_t g);
ad_status partition_by_class(ad_graph_t g, const int8_t *cls, int64_t n, int nclasses, int32_t *order,
                             std::vector<int64_t> &start);
ad_status recompute_degrees(ad_graph_t g);

// algebraic distance (sweep.cu).  With keep: the stored vectors after sweep
// t = 0, every, 2 every, ... are copied to keep->ckpt[t / every] (as many as
// given) and the min/max slots of all sweeps to keep->mm_copy.
struct KeepSpec {
    int every = 1;
    std::vector<void *> ckpt;
    uint32_t *mm_copy = nullptr;
};
ad_status algebraic_distance(ad_graph_t g, int32_t R, int32_t k, double omega, uint64_t seed,
                             uint32_t stream_id, ad_storage storage, int32_t flags, float *rho_dev,
                             const KeepSpec *keep = nullptr);
ad_status sweep_step(ad_graph_t g, ad_storage storage, int32_t R, double omega, const void *x_in, void *x_out,
                     const uint32_t *pmin, const uint32_t *pmax, uint32_t *mn, uint32_t *mx);
ad_status get_row_plan(ad_graph_t g, int groups, bool upper, RowPlan **out);
void natural_shape(int R, ad_storage storage, int *lanes_per_row, int *chunks_per_lane);   // sweep.cu

// selection (select.cu)
ad_status select_whole_graph(ad_graph_t g, const float *score_dev, double fraction, ad_mode mode,
                             uint8_t *keep_dev, int64_t *n_kept);
ad_status select_per_node_fit(ad_graph_t g, const float *score_dev, double fraction, ad_mode mode,
                              uint8_t *keep_dev, int64_t *n_kept, double *e_used);
ad_status select_per_node_fit_both(ad_graph_t g, const float *score, double fraction, uint8_t *keep_local,
                                   uint8_t *keep_global, int64_t *n_kept, double *e_used);
ad_status select_per_node_at(ad_graph_t g, const float *score_dev, double e, ad_mode mode,
                             uint8_t *keep_dev, int64_t *n_kept);
ad_status select_per_node_fit_ranked(ad_graph_t g, const uint32_t *rank_dev, double fraction, uint8_t *keep_dev,
                                     int64_t *n_kept, double *e_used);
ad_status select_local_degree(ad_graph_t g, double fraction, uint8_t *keep_dev, int64_t *n_kept, double *e_used);
ad_status row_ranks(ad_graph_t g, const uint32_t *ekey, uint32_t *rank_out, uint32_t *desc_scratch);
constexpr int64_t kLongRowDegree = 512;   // long_rows(): the rows of degree above this
ad_status long_rows(ad_graph_t g, const int64_t **rows, int64_t *count);

// SparsifyB order (binned.cu)
ad_status binned_ranks(ad_graph_t g, const float *score_dev, uint64_t seed, uint32_t *rank_dev,
                       uint32_t *bin_dev = nullptr);

ad_status check_scores(ad_graph_t g, const float *score);
void free_sel_cache(ad_graph_t g);

// sorting and compaction (sort.cu)
ad_status radix_sort_pairs(ad_graph_t g, uint64_t *keys, int64_t *vals, int64_t n, const std::vector<int> &shifts);
ad_status compact_flags(ad_graph_t g, const uint8_t *flag, int64_t n, int64_t **idx_out, int64_t *count);

// graph creation shared by the ABI and the multilevel code (api.cu)
ad_status create_impl(int32_t G, const int64_t *voff, int64_t n, const int64_t *row_ptr, const int32_t *col,
                      const float *weight, int32_t flags, void *stream, ad_graph_t *out);
ad_status create_like(ad_graph_t parent, int64_t n, const int64_t *rp_dev, const int32_t *col_dev, const float *w_dev,
                      ad_graph_t *out);

// reverse mode (grad.cu)
ad_status algebraic_distance_keep(ad_graph_t g, int32_t R, int32_t k, double omega, uint64_t seed,
                                  uint32_t stream_id, float *rho_dev, bool sqrt_checkpoints);
void free_saved(ad_graph_t g);

// host-side exact degree target of Alg. 2 (same formula as the documented reading)
int64_t degree_target(int64_t d, double e);

}  // namespace ad
