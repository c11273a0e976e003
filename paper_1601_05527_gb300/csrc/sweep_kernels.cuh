// sweep_kernels.cuh -- kernels of ComputeAlgDist (Alg. 1) on sm_103a: Philox
// init, JOR sweeps with the per-sweep rescale fused into the epilogue, and the
// per-edge distance.  Instantiated once per storage type (sweep_<type>.cu).
//
// Data layout: the R test vectors of vertex i form row i of X[n][stride]
// (stride = lanes_per_row * chunks_per_lane * V elements, 16-byte chunks,
// V = 4 FP32 or 8 16-bit values).  A lane group of LPR lanes owns one row at a
// time; lane gl of the group holds chunks gl, gl + LPR, ... of the row.
//
// Stored frame.  The iterate of Alg. 1 after sweep t is x_t = rescale(M x_{t-1}),
// M = (1-omega) I + omega D^-1 W, rescale mapping [min, max] of each vector
// onto [-1/2, 1/2].  M commutes with adding a constant vector and with scaling,
// and rescale ignores both, so the kernels store
//     s_t = a_{t-1} (M s_{t-1} - s_{t-1}[anchor]),   a_{t-1} = 1 / (max - min)(s_{t-1}),
// which differs from x_t by a per-vector shift only: the same rescaled values,
// the same distances rho = a_t |s_i - s_j|.  The anchor is the vertex of
// largest weighted degree of each graph.  Its value lies inside the bulk of
// the smoothed vector, so the stored values are deviations around zero instead
// of a common offset plus small deviations -- which is what lets 16-bit
// storage resolve the small distances of well-mixed graphs.  Each sweep
// reduces min/max of what it stores; the next launch turns them into a.
#pragma once
#include "ad_internal.cuh"

#include <cmath>
#include <cstring>

// Tuning parameters (compile-time; the defaults are the measured choice on GB300).
#ifndef AD_SWEEP_UB
#define AD_SWEEP_UB 4          // independent row loads in flight per lane of the distance pass
#endif
#ifndef AD_STREAM_U32
#define AD_STREAM_U32 8        // row loads in flight per lane of the streaming sweep, FP32 rows
#endif
#ifndef AD_STREAM_U16
#define AD_STREAM_U16 4        // ... 16-bit rows
#endif
#ifndef AD_STREAM_MINB
#define AD_STREAM_MINB 3       // resident CTAs per SM requested from ptxas for the streaming sweep
#endif
#ifndef AD_DIST_MINB
#define AD_DIST_MINB 4         // ... for the distance pass
#endif
#ifndef AD_MAX_LPR
#define AD_MAX_LPR 32          // most lanes that share one row (more chunks go to each lane beyond it)
#endif
#ifndef AD_COL_STREAM
#define AD_COL_STREAM 1        // 1: read column indices with the streaming (evict-first) hint
#endif

namespace ad {

template <typename T>
__device__ __forceinline__ T ld_stream(const T *p) {
#if AD_COL_STREAM
    return __ldcs(p);
#else
    return __ldg(p);
#endif
}

struct SweepArgs {
    const int64_t *rp;
    const int32_t *col;
    const float *w;        // nullable
    const float *Dinv;
    const double *D;
    const int64_t *upos;   // distance: first upper entry
    const int64_t *eoff;   // distance: edge id of that entry
    const void *x_in;
    void *x_out;
    const uint32_t *mm_prev_min, *mm_prev_max;  // nullptr at t = 0
    uint32_t *mm_min, *mm_max;                  // this sweep's min/max
    float *rho;            // distance output
    // plan
    const int32_t *big_row, *big_chunk, *medium_row, *small_row;
    uint32_t *big_counter;
    int64_t n_big, n_medium, n_small_rows;
    int64_t n_tasks;
    int32_t stride;        // elements per row
    int32_t nchunks;       // valid 16-byte chunks per row (ceil(R / V))
    int32_t R;
    float omega;
    int32_t normalize;
    // batches: graph gph owns rows [voff[gph], voff[gph+1]); min/max slots are
    // [G][stride] per sweep.  Batched launches give each warp a contiguous
    // block of tasks so that consecutive rows mostly share one graph.
    const int64_t *voff;
    int32_t G;
    int32_t blocked;
    const int32_t *anchor;   // [G] vertex whose previous value is subtracted (the stored frame's centre)
    float *ac;               // [G][2][stride]: scale a and centre c of this sweep (k_scale_center)
    // streaming sweep (k_sweep_stream).  Long rows (degree > kShortMax): their
    // entries, row after row, form a sequence [0, nnz_long) cut into S ranges of
    // equal length, range s = [s nnz_long / S, (s + 1) nnz_long / S).  Short rows:
    // a list of (row, CSR begin, degree).
    const int32_t *lrow;     // [n_long] long rows in increasing order
    const int32_t *lbeg;     // [n_long + 1] sequence position of each long row's first entry
    const int32_t *lcsr;     // [n_long] CSR position of each long row's first entry
    const int4 *srows;       // [n_short] short rows: (row, CSR begin, degree, 0)
    const int32_t *k0;       // [S] long row holding the first entry of each range
    uint32_t *counter;       // [S] pieces finished of the split row that starts in range s (zero between launches)
    float *spart;            // [2 S][stride] partial sums: 2s = the row continued from before range s, 2s + 1 = the row continuing after it
    int32_t n_long;
    int32_t n_short;
    int32_t S;
    int32_t nnz_long;
};

__device__ __forceinline__ int graph_of(const int64_t *voff, int G, int64_t row) {
    int lo = 0, hi = G;
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (__ldg(voff + mid) <= row) lo = mid; else hi = mid;
    }
    return lo;
}

// task index range of warp `wid` among `W` warps: [t, t_end) stepping `step`
struct TaskIter {
    int64_t t, t_end, step;
};
__device__ __forceinline__ TaskIter task_iter(int64_t n_tasks, int64_t wid, int64_t W, int blocked) {
    TaskIter it;
    if (blocked) {
        const int64_t per = (n_tasks + W - 1) / W;
        it.t = wid * per;
        it.t_end = min(n_tasks, it.t + per);
        it.step = 1;
    } else {
        it.t = wid;
        it.t_end = n_tasks;
        it.step = W;
    }
    return it;
}

// ----------------------------------------------------------------------------
// Init: x[i][r] = rand(-0.5, 0.5) from Philox, counter (i, r/4, stream), i the
// vertex id inside its graph.  One thread per (row, quad of vectors); rows of
// degree 0 are skipped.
// ----------------------------------------------------------------------------
template <typename T>
__global__ void k_init(const int64_t *__restrict__ rp, int64_t n, int32_t stride, uint32_t seed_lo,
                       uint32_t seed_hi, uint32_t stream_id, const int64_t *voff, int G, T *__restrict__ x) {
    const int32_t quads = stride / 4;
    const int64_t total = n * quads;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total;
         t += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = t / quads;
        const int32_t q = (int32_t)(t - i * quads);
        if (rp[i + 1] == rp[i]) continue;
        const int64_t li = G > 1 ? i - voff[graph_of(voff, G, i)] : i;   // id inside its graph
        uint4 c = make_uint4((uint32_t)((uint64_t)li), (uint32_t)((uint64_t)li >> 32), (uint32_t)q, stream_id);
        uint4 u = philox4x32_10(c, make_uint2(seed_lo, seed_hi));
        float v[4] = {unit_centered(u.x), unit_centered(u.y), unit_centered(u.z), unit_centered(u.w)};
        T *dst = x + i * stride + 4 * q;
        if constexpr (sizeof(T) == 4) {
            *reinterpret_cast<float4 *>(dst) = make_float4(v[0], v[1], v[2], v[3]);
        } else {
            uint2 p = make_uint2(Store<T>::pack2(v[0], v[1]), Store<T>::pack2(v[2], v[3]));
            *reinterpret_cast<uint2 *>(dst) = p;
        }
    }
}

// ----------------------------------------------------------------------------
// Helpers for the lane-group kernels
// ----------------------------------------------------------------------------
template <typename T, int LPR, int CPL>
struct Lane {
    static constexpr int V = Store<T>::V;
    static constexpr int E = CPL * V;       // elements held by one lane
    static constexpr int G = 32 / LPR;      // groups per warp
};

// Sum over the G groups of a warp (butterfly: every group ends with the total).
template <int LPR, int E>
__device__ __forceinline__ void reduce_groups(float (&acc)[E]) {
#pragma unroll
    for (int off = LPR; off < 32; off <<= 1)
#pragma unroll
        for (int e = 0; e < E; ++e) acc[e] += __shfl_xor_sync(0xffffffffu, acc[e], off);
}

// Epilogue of a row: z = (1-omega) s_i + omega Dinv_i S, store a (z - c), track min/max.
template <typename T, int LPR, int CPL>
__device__ __forceinline__ void load_own(const SweepArgs &a, int64_t row, int gl, uint4 (&own)[CPL]) {
    const uint4 *X = reinterpret_cast<const uint4 *>(a.x_in);
    const int64_t row_q = a.stride / Store<T>::V;
#pragma unroll
    for (int c = 0; c < CPL; ++c) {
        const int q = gl + c * LPR;
        own[c] = q < a.nchunks ? __ldg(X + row * row_q + q) : make_uint4(0, 0, 0, 0);
    }
}

// Scale a = 1 / (max - min) of the previous sweep's stored values for the
// lane's elements (1 before the first sweep, 0 for a vector with max == min).
template <typename T, int LPR, int CPL>
__device__ __forceinline__ void load_scale(const uint32_t *pmin, const uint32_t *pmax, int gl,
                                           float (&A)[CPL * Store<T>::V]) {
    // pmin / pmax point at the slots of the row's graph (nullptr: no rescale yet)
    constexpr int V = Store<T>::V;
#pragma unroll
    for (int c = 0; c < CPL; ++c)
#pragma unroll
        for (int e = 0; e < V; ++e) {
            const int r = (gl + c * LPR) * V + e;
            float av = 1.f;
            if (pmin) {   // FP32 on purpose: FP64 division runs on a very narrow pipe on this part
                const float lo = ord2f(pmin[r]), hi = ord2f(pmax[r]);
                av = hi > lo ? 1.f / (hi - lo) : 0.f;
            }
            A[c * V + e] = av;
        }
}

// Scale a = 1 / (max - min) of the previous sweep's stored values (1 before the
// first sweep, 0 for a vector with max == min) and centre c of the stored frame
// (the previous values of the graph's anchor vertex), once per graph and sweep,
// so that the sweep reads them from one cached line instead of holding them in
// registers.  Block g, one thread per 16-byte chunk.
template <typename T>
__global__ void k_scale_center(const uint32_t *pmin, const uint32_t *pmax, const void *x_in, const int32_t *anchor,
                               int32_t stride, float *ac) {
    constexpr int V = Store<T>::V;
    const int g = blockIdx.x;
    float *A = ac + (size_t)g * 2 * stride, *C = A + stride;
    const uint4 *xa = reinterpret_cast<const uint4 *>(x_in) + (int64_t)anchor[g] * (stride / V);
    for (int q = threadIdx.x; q < stride / V; q += blockDim.x) {
        float f[V];
        Store<T>::unpack(xa[q], f);
#pragma unroll
        for (int e = 0; e < V; ++e) {
            const int r = q * V + e;
            float av = 1.f;
            if (pmin) {   // FP32 on purpose: FP64 division runs on a very narrow pipe on this part
                const float lo = ord2f(pmin[(size_t)g * stride + r]), hi = ord2f(pmax[(size_t)g * stride + r]);
                av = hi > lo ? 1.f / (hi - lo) : 0.f;
            }
            A[r] = av;
            C[r] = f[e];
        }
    }
}

// ----------------------------------------------------------------------------
// Running min/max of the values a lane stores, for the graph `cg` of the rows
// it handled last; flushed with atomics when the lane moves to another graph.
// ----------------------------------------------------------------------------
template <typename T, int LPR, int CPL>
struct LaneStats {
    static constexpr int V = Store<T>::V, E = CPL * V;
    float mn[E], mx[E];
    int cg = -1;
    const float *acg = nullptr;   // scale and centre of graph cg

    __device__ __forceinline__ void flush(const SweepArgs &a, int gl) {
        if (cg < 0) return;
#pragma unroll
        for (int c = 0; c < CPL; ++c)
#pragma unroll
            for (int e = 0; e < V; ++e) {
                const int r = (gl + c * LPR) * V + e;
                if ((gl + c * LPR) < a.nchunks && mn[c * V + e] <= mx[c * V + e]) {
                    atomicMin(a.mm_min + (size_t)cg * a.stride + r, f2ord(mn[c * V + e]));
                    atomicMax(a.mm_max + (size_t)cg * a.stride + r, f2ord(mx[c * V + e]));
                }
            }
    }
    // make the lane's state describe graph `g`
    __device__ __forceinline__ void enter(const SweepArgs &a, int gl, int g, bool flush_old) {
        if (g == cg) return;
        if (flush_old) flush(a, gl);
        cg = g;
        acg = a.ac + (size_t)g * 2 * a.stride;
#pragma unroll
        for (int e = 0; e < E; ++e) { mn[e] = INFINITY; mx[e] = -INFINITY; }
    }
};

template <typename T>
constexpr int stream_minb() { return AD_STREAM_MINB; }

// ----------------------------------------------------------------------------
// Streaming JOR sweep (Alg. 1 inner loop), two phases in one launch.
//
// Long rows (degree > kShortMax).  Their entries, row after row, form one
// sequence; it is cut into S ranges of equal length and lane group s walks
// range s, U entries per batch: the column indices (and weights) of the next
// batch are loaded while the current batch's U neighbour rows are in flight,
// so every group keeps U row loads outstanding.  A long row has more entries
// than a batch, so a batch holds at most one row change: entries before it
// add to the finishing row, the rest to the next one, and the finishing row is
// written after the batch.  A row that lies inside one range is summed by its
// group in CSR order; a row cut by range ends ("split") leaves one partial sum
// per range it touches, and the last piece to finish adds them in range order
// and writes the row, so the result does not depend on timing.
//
// Short rows (degree 1 .. kShortMax).  One lane group per row, the row's
// column indices in one load, all of its neighbour rows in flight at once, the
// sum in CSR order; the groups of a warp take consecutive rows of the list and
// warps stride over it.
//
// The groups of a warp run in lock step (every shuffle sees all lanes); row
// changes are handled in a branch that the whole warp enters when any of its
// groups needs it.
// ----------------------------------------------------------------------------
constexpr int kShortMax = 8;   // rows of degree <= kShortMax take the short-row phase (>= every batch size U)

__device__ __forceinline__ int32_t range_of(int64_t p, int32_t S, int32_t len) {
    // largest s with floor(s len / S) <= p
    return (int32_t)(((p + 1) * (int64_t)S + len - 1) / len - 1);
}

template <typename T, int LPR, int CPL, int U>
struct StreamLane {
    static constexpr int V = Store<T>::V, E = CPL * V, G = 32 / LPR;
    static constexpr int CU = (U + LPR - 1) / LPR;            // column registers per lane per batch
    static constexpr int CS = (kShortMax + LPR - 1) / LPR;    // ... per short row
    static constexpr int MPL = LPR >= 8 ? 1 : 8 / LPR;        // row-metadata registers per lane per window
    static constexpr int W = LPR * MPL;                       // rows per metadata window
    static_assert(U <= kShortMax, "a batch must be shorter than every long row");
};

// lrow / lbeg / lcsr of long rows kb + gl + c LPR (past the end: no row, a position never reached)
template <int LPR, int MPL>
__device__ __forceinline__ void stream_window(const SweepArgs &a, int64_t kb, int gl, int32_t (&wr)[MPL],
                                              int32_t (&wb)[MPL], int32_t (&wc)[MPL]) {
#pragma unroll
    for (int c = 0; c < MPL; ++c) {
        const int64_t k = kb + gl + c * LPR;
        wr[c] = k < a.n_long ? __ldg(a.lrow + k) : 0;
        wb[c] = k <= a.n_long ? __ldg(a.lbeg + k) : 0x7fffffff;
        wc[c] = k < a.n_long ? __ldg(a.lcsr + k) : 0;
    }
}

template <typename T, int LPR, int CPL, int U, bool WT, bool BATCH>
__device__ __forceinline__ void sweep_stream_body(const SweepArgs &a, float *sm) {
    using SL = StreamLane<T, LPR, CPL, U>;
    constexpr int V = SL::V, E = SL::E, G = SL::G, CU = SL::CU, CS = SL::CS, MPL = SL::MPL, W = SL::W;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
    const int grp = lane / LPR, gl = lane % LPR;
    const unsigned gmask = LPR == 32 ? 0xffffffffu : (((1u << LPR) - 1u) << (grp * LPR));
    const int32_t gwarp = (int32_t)((int64_t)blockIdx.x * nwarps + warp);
    const int32_t gid = gwarp * G + grp;
    const uint4 *X = reinterpret_cast<const uint4 *>(a.x_in);
    const int32_t row_q = a.stride / V;

    LaneStats<T, LPR, CPL> ls;
    ls.enter(a, gl, 0, false);
    int32_t gbeg = 0, gend = 0;   // rows of graph ls.cg (batches only)
    if (BATCH) gend = (int32_t)__ldg(a.voff + 1);

    // row r's output: z = (1-omega) s_r + omega Dinv_r S, stored as a (z - c), min/max tracked
    auto epilogue = [&](int32_t r, const uint4 (&ow)[CPL], float di, const float (&S)[E]) {
        if (BATCH && (r >= gend || r < gbeg)) {
            ls.enter(a, gl, graph_of(a.voff, a.G, r), true);
            gbeg = (int32_t)__ldg(a.voff + ls.cg);
            gend = (int32_t)__ldg(a.voff + ls.cg + 1);
        }
        uint4 *Y = reinterpret_cast<uint4 *>(a.x_out);
        const float om = a.omega, om1 = 1.f - a.omega;
#pragma unroll
        for (int c = 0; c < CPL; ++c) {
            const int q = gl + c * LPR;
            if (q < a.nchunks) {
                float y[V], o[V];
                Store<T>::unpack(ow[c], y);
#pragma unroll
                for (int e4 = 0; e4 < V / 4; ++e4) {
                    const float4 av = __ldg(reinterpret_cast<const float4 *>(ls.acg + q * V) + e4);
                    const float4 cv = __ldg(reinterpret_cast<const float4 *>(ls.acg + a.stride + q * V) + e4);
                    const float A[4] = {av.x, av.y, av.z, av.w}, C[4] = {cv.x, cv.y, cv.z, cv.w};
#pragma unroll
                    for (int i = 0; i < 4; ++i) {
                        const int e = 4 * e4 + i;
                        const float z = fmaf(om1, y[e], om * (S[c * V + e] * di));
                        o[e] = Store<T>::round(A[i] * (z - C[i]));
                        ls.mn[c * V + e] = fminf(ls.mn[c * V + e], o[e]);
                        ls.mx[c * V + e] = fmaxf(ls.mx[c * V + e], o[e]);
                    }
                }
                Y[(int64_t)r * row_q + q] = Store<T>::pack(o);
            }
        }
    };
    auto add = [&](float (&dst)[E], const uint4 (&vu)[CPL], float w) {
#pragma unroll
        for (int c = 0; c < CPL; ++c) {
            float f[V];
            Store<T>::unpack(vu[c], f);
#pragma unroll
            for (int e = 0; e < V; ++e) dst[c * V + e] = WT ? fmaf(w, f[e], dst[c * V + e]) : dst[c * V + e] + f[e];
        }
    };

    // ======================= long rows =======================
    if (a.n_long > 0) {
        const bool has = gid < a.S;
        const int32_t s0 = has ? (int32_t)((int64_t)gid * a.nnz_long / a.S) : 0;
        const int32_t s1 = has ? (int32_t)(((int64_t)gid + 1) * a.nnz_long / a.S) : 0;
        // k: current long row; row = lrow[k]; sequence [rs, re); CSR begins cs (row k), cn (k + 1), cn2 (k + 2);
        // rn2 = end of row k + 1.  Rows kb .. kb + 2W - 1 are held in the window.
        int64_t k = has ? __ldg(a.k0 + gid) : 0;
        int64_t kb = k;
        int32_t wr[MPL], wb[MPL], wc[MPL], nr[MPL], nb2[MPL], nc[MPL];
        stream_window<LPR, MPL>(a, kb, gl, wr, wb, wc);
        stream_window<LPR, MPL>(a, kb + W, gl, nr, nb2, nc);
        auto fetch = [&](int64_t kk, int32_t &r_out, int32_t &b_out, int32_t &c_out) {
            const int rel = (int)(kk - kb);
            const int src = grp * LPR + rel % LPR, slot = (rel % W) / LPR;
            const bool second = rel >= W;
#pragma unroll
            for (int c = 0; c < MPL; ++c) {
                const int32_t tr = __shfl_sync(0xffffffffu, second ? nr[c] : wr[c], src);
                const int32_t tb = __shfl_sync(0xffffffffu, second ? nb2[c] : wb[c], src);
                const int32_t tc = __shfl_sync(0xffffffffu, second ? nc[c] : wc[c], src);
                if (c == slot) { r_out = tr; b_out = tb; c_out = tc; }
            }
        };
        int32_t row = 0, rs = 0, re = 0, rn2 = 0, cs = 0, cn = 0, cn2 = 0, tmp = 0;
        fetch(k, row, rs, cs);
        fetch(k + 1, tmp, re, cn);
        fetch(k + 2, tmp, rn2, cn2);
        if (!has) { re = 0x7fffffff; rn2 = 0x7fffffff; }

        uint4 own[CPL];
        float dinv = 0.f;
        if (has) {
            load_own<T, LPR, CPL>(a, row, gl, own);
            dinv = __ldg(a.Dinv + row);
        }
        float acc[E];
#pragma unroll
        for (int e = 0; e < E; ++e) acc[e] = 0.f;

        // A split row whose last piece this group finished: combined after the batch.
        int32_t pend_row = -1, pend_r0 = 0, pend_r1 = 0;
        auto finish = [&]() {
            if (rs >= s0 && re <= s1) {   // the whole row lies in this range
                epilogue(row, own, dinv, acc);
                return;
            }
            const int64_t slot = 2 * (int64_t)gid + (rs < s0 ? 0 : 1);
            float *pp = a.spart + slot * a.stride;
#pragma unroll
            for (int c = 0; c < CPL; ++c) {
                const int q = gl + c * LPR;
                if (q < a.nchunks) {
#pragma unroll
                    for (int e4 = 0; e4 < V / 4; ++e4)
                        __stcg(reinterpret_cast<float4 *>(pp + q * V) + e4,
                               make_float4(acc[c * V + 4 * e4], acc[c * V + 4 * e4 + 1], acc[c * V + 4 * e4 + 2],
                                           acc[c * V + 4 * e4 + 3]));
                }
            }
            __threadfence();
            __syncwarp(gmask);
            const int32_t r0 = range_of(rs, a.S, a.nnz_long), r1 = range_of((int64_t)re - 1, a.S, a.nnz_long);
            uint32_t old = 0;
            if (gl == 0) old = atomicAdd(a.counter + r0, 1u);
            old = __shfl_sync(gmask, old, grp * LPR);
            if (old == (uint32_t)(r1 - r0)) { pend_row = row; pend_r0 = r0; pend_r1 = r1; }
        };
        // partials of a split row in range order (a few loads in flight), then its output
        auto combine = [&]() {
            __threadfence();
            uint4 ow[CPL];
            load_own<T, LPR, CPL>(a, pend_row, gl, ow);
            const float di = __ldg(a.Dinv + pend_row);
            float S[E];
#pragma unroll
            for (int e = 0; e < E; ++e) S[e] = 0.f;
            constexpr int UC = 4;
            for (int32_t rb = pend_r0; rb <= pend_r1; rb += UC) {
                float4 f[UC][E / 4];
#pragma unroll
                for (int u = 0; u < UC; ++u) {
                    const int32_t rr = rb + u;
                    const int64_t sl = rr == pend_r0 ? 2 * (int64_t)rr + 1 : 2 * (int64_t)rr;
#pragma unroll
                    for (int c = 0; c < CPL; ++c) {
                        const int q = gl + c * LPR;
#pragma unroll
                        for (int e4 = 0; e4 < V / 4; ++e4)
                            f[u][c * (V / 4) + e4] = (rr <= pend_r1 && q < a.nchunks)
                                ? __ldcg(reinterpret_cast<const float4 *>(a.spart + sl * a.stride + q * V) + e4)
                                : make_float4(0.f, 0.f, 0.f, 0.f);
                    }
                }
#pragma unroll
                for (int u = 0; u < UC; ++u)
#pragma unroll
                    for (int i = 0; i < E / 4; ++i) {
                        S[4 * i + 0] += f[u][i].x;
                        S[4 * i + 1] += f[u][i].y;
                        S[4 * i + 2] += f[u][i].z;
                        S[4 * i + 3] += f[u][i].w;
                    }
            }
            epilogue(pend_row, ow, di, S);
            if (gl == 0) a.counter[pend_r0] = 0u;
            pend_row = -1;
        };
        // the row change of the groups with `ends`, the next row's sum starting from carry
        auto next_row = [&](bool ends, const float (&carry)[E]) {
            if (ends) {
                finish();
                ++k;
                if (k - kb == W) {   // into the second half of the window; load the one after it
                    kb += W;
#pragma unroll
                    for (int c = 0; c < MPL; ++c) { wr[c] = nr[c]; wb[c] = nb2[c]; wc[c] = nc[c]; }
                    stream_window<LPR, MPL>(a, kb + W, gl, nr, nb2, nc);
                }
            }
            int32_t nrow = 0, b2 = 0, c2 = 0;
            fetch(k, nrow, tmp, tmp);
            fetch(k + 2, tmp, b2, c2);
            if (ends) {
                row = nrow;
                rs = re; re = rn2; rn2 = b2;
                cs = cn; cn = cn2; cn2 = c2;
                load_own<T, LPR, CPL>(a, row, gl, own);
                dinv = __ldg(a.Dinv + row);
#pragma unroll
                for (int e = 0; e < E; ++e) acc[e] = carry[e];
            }
        };
        // CSR position of sequence position q (q in rows k .. k + 2)
        auto csr_of = [&](int64_t q) -> int64_t {
            return q < re ? cs + (q - rs) : (q < rn2 ? cn + (q - re) : cn2 + (q - rn2));
        };
        auto load_cols = [&](int64_t p, int32_t (&cj)[CU], float (&cw)[CU]) {
#pragma unroll
            for (int c = 0; c < CU; ++c) {
                const int64_t q = p + gl + c * LPR;
                const bool ok = gl + c * LPR < U && q < s1;
                const int64_t pos = csr_of(q);
                cj[c] = ok ? ld_stream(a.col + pos) : 0;
                if (WT) cw[c] = ok ? ld_stream(a.w + pos) : 0.f;
            }
        };

        const int32_t len = s1 - s0;
        const int nbt = __reduce_max_sync(0xffffffffu, (len + U - 1) / U);
        int32_t cj[CU], cjn[CU];
        float cw[CU], cwn[CU];
        load_cols(s0, cj, cw);
        for (int b = 0; b < nbt; ++b) {
            const int32_t p = s0 + b * U;
            uint4 v[U][CPL];
            float wt[U];
#pragma unroll
            for (int u = 0; u < U; ++u) {
                const int src = grp * LPR + u % LPR;
                const int32_t j = __shfl_sync(0xffffffffu, cj[u / LPR], src);
                wt[u] = WT ? __shfl_sync(0xffffffffu, cw[u / LPR], src) : 1.f;
#pragma unroll
                for (int c = 0; c < CPL; ++c) {
                    const int q = gl + c * LPR;
                    v[u][c] = (p + u < s1 && q < a.nchunks) ? __ldg(X + (int64_t)j * row_q + q)
                                                            : make_uint4(0, 0, 0, 0);
                }
            }
            load_cols(p + U, cjn, cwn);
            const bool end_in = re < min(p + U, s1);   // the group's row ends inside the batch (at most once)
            if (!__any_sync(0xffffffffu, end_in)) {
#pragma unroll
                for (int u = 0; u < U; ++u) add(acc, v[u], wt[u]);
            } else {
                float acc2[E];
#pragma unroll
                for (int e = 0; e < E; ++e) acc2[e] = 0.f;
#pragma unroll
                for (int u = 0; u < U; ++u) {
                    if (p + u < re) add(acc, v[u], wt[u]);
                    else add(acc2, v[u], wt[u]);
                }
                next_row(end_in, acc2);
                if (__any_sync(0xffffffffu, pend_row >= 0)) {
                    if (pend_row >= 0) combine();
                }
            }
#pragma unroll
            for (int c = 0; c < CU; ++c) { cj[c] = cjn[c]; if (WT) cw[c] = cwn[c]; }
        }
        if (has && len > 0) finish();   // the row holding the range's last entry
        if (pend_row >= 0) combine();
    }

    // ======================= short rows =======================
    {
        const int32_t total_warps = (int32_t)(gridDim.x * nwarps);
        const int32_t n_tasks = (a.n_short + G - 1) / G;
        for (int32_t t = gwarp; t < n_tasks; t += total_warps) {
            const int32_t sk = t * G + grp;
            const int4 sr = sk < a.n_short ? __ldg(a.srows + sk) : make_int4(0, 0, 0, 0);
            const int32_t row = sr.x, beg = sr.y, deg = sr.z;
            int32_t cj[CS];
            float cw[CS];
#pragma unroll
            for (int c = 0; c < CS; ++c) {
                const int u = gl + c * LPR;
                const bool ok = u < deg;
                cj[c] = ok ? ld_stream(a.col + beg + u) : 0;
                if (WT) cw[c] = ok ? ld_stream(a.w + beg + u) : 0.f;
            }
            uint4 own[CPL];
            float dinv = 0.f;
            if (deg > 0) {
                load_own<T, LPR, CPL>(a, row, gl, own);
                dinv = __ldg(a.Dinv + row);
            }
            uint4 v[kShortMax][CPL];
            float wt[kShortMax];
#pragma unroll
            for (int u = 0; u < kShortMax; ++u) {
                const int src = grp * LPR + u % LPR;
                const int32_t j = __shfl_sync(0xffffffffu, cj[u / LPR], src);
                wt[u] = WT ? __shfl_sync(0xffffffffu, cw[u / LPR], src) : 1.f;
#pragma unroll
                for (int c = 0; c < CPL; ++c) {
                    const int q = gl + c * LPR;
                    v[u][c] = (u < deg && q < a.nchunks) ? __ldg(X + (int64_t)j * row_q + q) : make_uint4(0, 0, 0, 0);
                }
            }
            float acc[E];
#pragma unroll
            for (int e = 0; e < E; ++e) acc[e] = 0.f;
#pragma unroll
            for (int u = 0; u < kShortMax; ++u)
                if (u < deg) add(acc, v[u], wt[u]);
            if (deg > 0) epilogue(row, own, dinv, acc);
        }
    }

    // ---- min/max of what this CTA stored -> atomics
    if (BATCH) {
        const bool same = __all_sync(0xffffffffu, ls.cg == __shfl_sync(0xffffffffu, ls.cg, 0));
        if (same) {
#pragma unroll
            for (int off = LPR; off < 32; off <<= 1)
#pragma unroll
                for (int e = 0; e < E; ++e) {
                    ls.mn[e] = fminf(ls.mn[e], __shfl_xor_sync(0xffffffffu, ls.mn[e], off));
                    ls.mx[e] = fmaxf(ls.mx[e], __shfl_xor_sync(0xffffffffu, ls.mx[e], off));
                }
            if (grp == 0) ls.flush(a, gl);
        } else {
            ls.flush(a, gl);
        }
        return;
    }
#pragma unroll
    for (int off = LPR; off < 32; off <<= 1)
#pragma unroll
        for (int e = 0; e < E; ++e) {
            ls.mn[e] = fminf(ls.mn[e], __shfl_xor_sync(0xffffffffu, ls.mn[e], off));
            ls.mx[e] = fmaxf(ls.mx[e], __shfl_xor_sync(0xffffffffu, ls.mx[e], off));
        }
    float *smn = sm, *smx = sm + nwarps * a.stride;
    if (grp == 0) {
#pragma unroll
        for (int c = 0; c < CPL; ++c)
#pragma unroll
            for (int e = 0; e < V; ++e) {
                const int r = (gl + c * LPR) * V + e;
                smn[warp * a.stride + r] = ls.mn[c * V + e];
                smx[warp * a.stride + r] = ls.mx[c * V + e];
            }
    }
    __syncthreads();
    for (int r = threadIdx.x; r < a.nchunks * V; r += blockDim.x) {
        float lo = INFINITY, hi = -INFINITY;
        for (int wi = 0; wi < nwarps; ++wi) {
            lo = fminf(lo, smn[wi * a.stride + r]);
            hi = fmaxf(hi, smx[wi * a.stride + r]);
        }
        if (lo <= hi) {
            atomicMin(a.mm_min + r, f2ord(lo));
            atomicMax(a.mm_max + r, f2ord(hi));
        }
    }
}

// row loads in flight per lane of the streaming sweep: 8 for FP32 rows, 4 for
// 16-bit rows (whose lanes hold twice the values)
template <typename T>
constexpr int stream_u() { return sizeof(T) == 4 ? AD_STREAM_U32 : AD_STREAM_U16; }

template <typename T, int LPR, int CPL, bool BATCH>
__global__ void __launch_bounds__(256, stream_minb<T>()) k_sweep_stream(SweepArgs a) {
    extern __shared__ float sm[];   // [2][warps][stride]
    if (a.w) sweep_stream_body<T, LPR, CPL, stream_u<T>() / CPL, true, BATCH>(a, sm);
    else sweep_stream_body<T, LPR, CPL, stream_u<T>() / CPL, false, BATCH>(a, sm);
}

// ----------------------------------------------------------------------------
// Edge distance: for every upper entry (i, j > i) of the CSR, edge id e =
// eoff[i] + (p - upos[i]), rho_e = sqrt(sum_r a_r^2 (y_i^r - y_j^r)^2).
// A lane group handles one edge; its lanes hold different chunks of R.
// ----------------------------------------------------------------------------
// Sums of K values over the LPR lanes of a group, transposed: each exchange
// halves the values a lane holds, so K sums take about LPR shuffles in total
// instead of K * log2(LPR).  Afterwards lane gl holds in s[0 .. NH) the sums of
// values which .. which + NH - 1 (NH = max(1, K / LPR)); when LPR > K the lanes
// that differ only in their low bits hold the same sums.
template <int LPR, int K>
__device__ __forceinline__ void group_sums(float (&s)[K], int gl, unsigned gmask, int &which) {
    static_assert(K >= 1 && (K & (K - 1)) == 0, "the transposed sums halve K: K must be a power of two");
    which = 0;
#pragma unroll
    for (int o = LPR / 2, c = K; o >= 1; o >>= 1) {
        if (c > 1) {
            const bool upper = (gl & o) != 0;
#pragma unroll
            for (int i = 0; i < K / 2; ++i) {
                if (i < c / 2) {
                    const float send = upper ? s[i] : s[i + c / 2];
                    const float keep = upper ? s[i + c / 2] : s[i];
                    s[i] = keep + __shfl_xor_sync(gmask, send, o);
                }
            }
            if (upper) which += c / 2;
            c >>= 1;
        } else {
            s[0] += __shfl_xor_sync(gmask, s[0], o);
        }
    }
}

template <typename T, int LPR, int CPL>
__device__ __forceinline__ void edge_rows(const SweepArgs &a, int64_t row, int64_t p0, int64_t p1, int step,
                                          int first, int gl, unsigned gmask, const float (&A2)[CPL * Store<T>::V]) {
    constexpr int V = Store<T>::V, E = CPL * V;
    // edges of one group in flight: the largest power of two <= AD_SWEEP_UB (group_sums halves it)
    constexpr int UB = AD_SWEEP_UB >= 8 ? 8 : AD_SWEEP_UB >= 4 ? 4 : AD_SWEEP_UB >= 2 ? 2 : 1;
    const uint4 *X = reinterpret_cast<const uint4 *>(a.x_in);
    const int64_t row_q = a.stride / V;
    float yi[E];
#pragma unroll
    for (int c = 0; c < CPL; ++c) {
        const int q = gl + c * LPR;
        if (q < a.nchunks) Store<T>::unpack(__ldg(X + row * row_q + q), yi + c * V);
        else {
#pragma unroll
            for (int e = 0; e < V; ++e) yi[c * V + e] = 0.f;
        }
    }
    const int64_t ebase = a.eoff[row] - a.upos[row];
    const double Di = a.normalize ? a.D[row] : 0.0;
    // the lanes of one group share p, so the group-masked reduction below is uniform
    for (int64_t pb = p0 + first; pb < p1; pb += (int64_t)step * UB) {
        int32_t jn[UB];
        uint4 v[UB][CPL];
#pragma unroll
        for (int u = 0; u < UB; ++u) {
            const int64_t p = pb + (int64_t)u * step;
            jn[u] = p < p1 ? ld_stream(a.col + p) : 0;
        }
#pragma unroll
        for (int u = 0; u < UB; ++u)
#pragma unroll
            for (int c = 0; c < CPL; ++c) {
                const int q = gl + c * LPR;
                v[u][c] = (pb + (int64_t)u * step < p1 && q < a.nchunks) ? __ldg(X + (int64_t)jn[u] * row_q + q)
                                                                          : make_uint4(0, 0, 0, 0);
            }
        float s[UB];
#pragma unroll
        for (int u = 0; u < UB; ++u) {
            s[u] = 0.f;
#pragma unroll
            for (int c = 0; c < CPL; ++c) {
                float yj[V];
                Store<T>::unpack(v[u][c], yj);
#pragma unroll
                for (int e = 0; e < V; ++e) {
                    const float d = yi[c * V + e] - yj[e];
                    s[u] = fmaf(A2[c * V + e] * d, d, s[u]);
                }
            }
        }
        int which = 0;
        group_sums<LPR, UB>(s, gl, gmask, which);
        constexpr int NH = UB / LPR > 0 ? UB / LPR : 1;
        const bool writer = (LPR <= UB) || (gl % (LPR / UB) == 0);
#pragma unroll
        for (int i = 0; i < NH; ++i) {
            int32_t jw = 0;
#pragma unroll
            for (int u = 0; u < UB; ++u) jw = (u == which + i) ? jn[u] : jw;
            const int64_t p = pb + (int64_t)(which + i) * step;
            if (writer && p < p1) {
                float rho = sqrtf(s[i]);
                if (a.normalize) rho = (float)((double)rho * sqrt(Di * a.D[jw]));
                a.rho[ebase + p] = rho;
            }
        }
    }
}

template <typename T, int LPR, int CPL>
__global__ void __launch_bounds__(256, AD_DIST_MINB) k_distance(SweepArgs a) {
    using L = Lane<T, LPR, CPL>;
    constexpr int V = L::V, E = L::E, G = L::G;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
    const int grp = lane / LPR, gl = lane % LPR;
    const unsigned gmask = LPR == 32 ? 0xffffffffu : (((1u << LPR) - 1u) << (grp * LPR));
    float A[E], A2[E];
    int cg = -1;
    // squared scale of the last rescale of graph g; padded vectors r >= R excluded
    auto enter = [&](int g) {
        if (g == cg) return;
        cg = g;
        load_scale<T, LPR, CPL>(a.mm_prev_min ? a.mm_prev_min + (size_t)g * a.stride : nullptr,
                                a.mm_prev_max ? a.mm_prev_max + (size_t)g * a.stride : nullptr, gl, A);
#pragma unroll
        for (int c = 0; c < CPL; ++c)
#pragma unroll
            for (int e = 0; e < V; ++e) {
                const int r = (gl + c * LPR) * V + e;
                A2[c * V + e] = (r < a.R) ? A[c * V + e] * A[c * V + e] : 0.f;
            }
    };
    auto row_graph = [&](int64_t row) { return a.G > 1 ? graph_of(a.voff, a.G, row) : 0; };
    const int64_t W = (int64_t)gridDim.x * nwarps;
    const TaskIter it = task_iter(a.n_tasks, (int64_t)blockIdx.x * nwarps + warp, W, a.blocked);
    for (int64_t task = it.t; task < it.t_end; task += it.step) {
        if (task < a.n_big) {
            const int64_t row = a.big_row[task];
            const int32_t c = a.big_chunk[task];
            const int64_t ub = a.upos[row], ue = a.rp[row + 1];
            const int64_t p0 = ub + (int64_t)c * kChunk, p1 = min(ue, p0 + kChunk);
            enter(row_graph(row));
            edge_rows<T, LPR, CPL>(a, row, p0, p1, G, grp, gl, gmask, A2);
        } else if (task < a.n_big + a.n_medium) {
            const int64_t row = a.medium_row[task - a.n_big];
            enter(row_graph(row));
            edge_rows<T, LPR, CPL>(a, row, a.upos[row], a.rp[row + 1], G, grp, gl, gmask, A2);
        } else {
            const int64_t si = (task - a.n_big - a.n_medium) * G + grp;
            if (si < a.n_small_rows) {
                const int64_t row = a.small_row[si];
                enter(row_graph(row));
                edge_rows<T, LPR, CPL>(a, row, a.upos[row], a.rp[row + 1], 1, 0, gl, gmask, A2);
            }
        }
    }
}

struct Config {
    int lpr, cpl, V, stride, nchunks;
    int per_sm = 0;   // sweep CTAs per SM (0: as many as fit)
};


// One streaming sweep: ranges sized so that every resident lane group of the
// launch walks one range (fewer, of >= 32 entries each, on small graphs).
template <typename T, int LPR, int CPL>
ad_status launch_sweep_stream(ad_graph_t g, const SweepArgs &a, int per_sm_cap, size_t smem) {
    if (g->nnz > (int64_t)0x7fffffff - 256)   // positions and batch ends are 32-bit in the kernel
        return fail(AD_ERR_INVALID_ARG, "too many CSR entries for the streaming sweep");
    const bool batch = a.G > 1;
    int per_sm = 0;
    if (batch) cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_sweep_stream<T, LPR, CPL, true>, 256, smem);
    else cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_sweep_stream<T, LPR, CPL, false>, 256, smem);
    if (per_sm < 1) per_sm = 1;
    if (per_sm_cap > 0 && per_sm_cap < per_sm) per_sm = per_sm_cap;
    const int64_t groups_per_block = 8 * (32 / LPR);
    int64_t S = (int64_t)per_sm * g->num_sms * groups_per_block;

    StreamPlan *sp = nullptr;
    AD_TRY(get_stream_plan(g, (int32_t)S, &sp));
    S = sp->S;
    AD_TRY(ensure(g, g->part, (size_t)2 * S * a.stride * sizeof(float)));
    SweepArgs b = a;
    b.lrow = g->lrow;
    b.lbeg = g->lbeg;
    b.lcsr = g->lcsr;
    b.srows = reinterpret_cast<const int4 *>(g->srows);
    b.k0 = sp->k0;
    b.counter = sp->counter;
    b.spart = static_cast<float *>(g->part.ptr);
    b.n_long = (int32_t)g->n_long;
    b.n_short = (int32_t)g->n_short;
    b.S = (int32_t)S;
    b.nnz_long = (int32_t)g->nnz_long;
    // every resident group walks one range (fewer ranges, of >= 32 entries, on small graphs),
    // and up to one group per short row
    int64_t need = std::max<int64_t>(S, g->n_short);
    const int64_t cap = (int64_t)per_sm * g->num_sms * groups_per_block;
    if (need > cap) need = cap;
    const int blocks = (int)std::max<int64_t>(1, (need + groups_per_block - 1) / groups_per_block);
    AD_LAUNCH(k_scale_center<T>, a.G, 32, 0, g->stream, a.mm_prev_min, a.mm_prev_max, a.x_in, a.anchor, a.stride,
              a.ac);
    if (batch) AD_LAUNCH((k_sweep_stream<T, LPR, CPL, true>), blocks, 256, smem, g->stream, b);
    else AD_LAUNCH((k_sweep_stream<T, LPR, CPL, false>), blocks, 256, smem, g->stream, b);
    return AD_OK;
}
template <typename T, int LPR, int CPL>
ad_status launch_distance(ad_graph_t g, const SweepArgs &a, int blocks) {
    AD_LAUNCH((k_distance<T, LPR, CPL>), blocks, 256, 0, g->stream, a);
    return AD_OK;
}
template <typename T, int LPR, int CPL>
int distance_blocks_per_sm() {
    int per_sm = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_distance<T, LPR, CPL>, 256, 0);
    return per_sm > 0 ? per_sm : 1;
}

template <typename T>
ad_status dispatch(ad_graph_t g, const Config &cf, bool sweep, const SweepArgs &a, int64_t n_tasks,
                          size_t smem) {
    // persistent grid: every SM full, but no more warps than tasks
    auto run = [&](auto lpr_c, auto cpl_c) -> ad_status {
        constexpr int LPR = decltype(lpr_c)::value, CPL = decltype(cpl_c)::value;
        if (sweep) return launch_sweep_stream<T, LPR, CPL>(g, a, cf.per_sm, smem);
        int64_t blocks = (int64_t)distance_blocks_per_sm<T, LPR, CPL>() * g->num_sms;
        const int64_t need = (n_tasks + 7) / 8;
        if (blocks > need) blocks = need > 0 ? need : 1;
        return launch_distance<T, LPR, CPL>(g, a, (int)blocks);
    };
    using std::integral_constant;
    switch (cf.lpr * 100 + cf.cpl) {
        case 101: return run(integral_constant<int, 1>{}, integral_constant<int, 1>{});
        case 201: return run(integral_constant<int, 2>{}, integral_constant<int, 1>{});
        case 401: return run(integral_constant<int, 4>{}, integral_constant<int, 1>{});
        case 801: return run(integral_constant<int, 8>{}, integral_constant<int, 1>{});
        case 1601: return run(integral_constant<int, 16>{}, integral_constant<int, 1>{});
        case 3201: return run(integral_constant<int, 32>{}, integral_constant<int, 1>{});
        case 3202: return run(integral_constant<int, 32>{}, integral_constant<int, 2>{});
        default: return fail(AD_ERR_INVALID_ARG, "unsupported R / storage combination");
    }
}


// one instantiation per storage type, each in its own translation unit
ad_status dispatch_f32(ad_graph_t g, const Config &cf, bool sweep, const SweepArgs &a, int64_t n_tasks, size_t smem);
ad_status dispatch_bf16(ad_graph_t g, const Config &cf, bool sweep, const SweepArgs &a, int64_t n_tasks, size_t smem);
ad_status dispatch_f16(ad_graph_t g, const Config &cf, bool sweep, const SweepArgs &a, int64_t n_tasks, size_t smem);
ad_status dispatch_q16(ad_graph_t g, const Config &cf, bool sweep, const SweepArgs &a, int64_t n_tasks, size_t smem);
ad_status launch_init(ad_graph_t g, ad_storage storage, int blocks, int32_t stride, uint64_t seed, uint32_t stream_id,
                      void *x);

}  // namespace ad
