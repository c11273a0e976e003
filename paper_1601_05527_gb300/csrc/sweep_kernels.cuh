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

#include <algorithm>
#include <cmath>
#include <cstring>

// Tuning parameters (compile-time; the defaults are the measured choice on GB300).
#ifndef AD_SWEEP_UB
#define AD_SWEEP_UB 4          // independent row loads in flight per lane
#endif
#ifndef AD_SWEEP_MINB
#define AD_SWEEP_MINB 6        // resident CTAs per SM requested from ptxas for the FP32 sweep
#endif
#ifndef AD_SWEEP_MINB16
#define AD_SWEEP_MINB16 5      // ... for the 16-bit storage formats
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
    float *part;           // [n_big][stride] partial sums of big rows
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
};

__device__ __forceinline__ int graph_of(const int64_t *voff, int G, int64_t row) {
    int lo = 0, hi = G;
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (__ldg(voff + mid) <= row) lo = mid; else hi = mid;
    }
    return lo;
}

// graph_of with the vertex range of the last graph found kept: the rows a
// lane group visits in a batch mostly lie in one graph, so most lookups are
// one comparison instead of a binary search
struct GraphCache {
    int64_t lo = 0, hi = -1;
    int g = 0;
    __device__ __forceinline__ int of(const int64_t *voff, int G, int64_t row) {
        if (row >= lo && row < hi) return g;
        g = graph_of(voff, G, row);
        lo = __ldg(voff + g);
        hi = __ldg(voff + g + 1);
        return g;
    }
};

// task index range of warp `wid` among `W` warps: [t, t_end) stepping `step`
struct TaskIter {
    int64_t t, t_end, step;
};
__device__ __forceinline__ TaskIter task_iter(int64_t n_tasks, int64_t wid, int64_t W, int blocked) {
    TaskIter it;
    if (blocked) {
        // a contiguous range of tasks per CTA, the CTA's warps interleaved inside
        // it: a batch's lanes then meet few graphs (each change of graph flushes
        // the lane's min/max), and the CTA's warps share neighbouring rows
        const int nw = blockDim.x >> 5;
        const int64_t ncta = W / nw, cta = wid / nw;
        const int64_t per = (n_tasks + ncta - 1) / ncta;
        it.t = cta * per + wid % nw;
        it.t_end = min(n_tasks, cta * per + per);
        it.step = nw;
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
__device__ __forceinline__ void init_rows(const int64_t *__restrict__ rp, int64_t n, int32_t stride, uint32_t seed_lo,
                                          uint32_t seed_hi, uint32_t stream_id, const int64_t *voff, int G,
                                          T *__restrict__ x) {
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

template <typename T>
__global__ void k_init(const int64_t *__restrict__ rp, int64_t n, int32_t stride, uint32_t seed_lo,
                       uint32_t seed_hi, uint32_t stream_id, const int64_t *voff, int G, T *__restrict__ x) {
    init_rows<T>(rp, n, stride, seed_lo, seed_hi, stream_id, voff, G, x);
}

// ----------------------------------------------------------------------------
// Helpers for the lane-group kernels
// ----------------------------------------------------------------------------
// Two FP32 additions (or fused multiply-adds) in one packed instruction; each
// half is rounded as the scalar operation would be, so sums are unchanged.
__device__ __forceinline__ void add_f32x2(float &a0, float &a1, float b0, float b1) {
    asm("{\n\t.reg .b64 x, y, z;\n\tmov.b64 x, {%0, %1};\n\tmov.b64 y, {%2, %3};\n\t"
        "add.rn.f32x2 z, x, y;\n\tmov.b64 {%0, %1}, z;\n\t}"
        : "+f"(a0), "+f"(a1) : "f"(b0), "f"(b1));
}
__device__ __forceinline__ void fma_f32x2(float &a0, float &a1, float w, float b0, float b1) {
    asm("{\n\t.reg .b64 x, y, z;\n\tmov.b64 x, {%0, %1};\n\tmov.b64 y, {%2, %3};\n\tmov.b64 z, {%4, %4};\n\t"
        "fma.rn.f32x2 x, z, y, x;\n\tmov.b64 {%0, %1}, x;\n\t}"
        : "+f"(a0), "+f"(a1) : "f"(b0), "f"(b1), "f"(w));
}
// acc[e] += f[e] (W: acc[e] = fmaf(w, f[e], acc[e])) for an even count of values
template <int N, bool W>
__device__ __forceinline__ void accumulate(float *acc, const float *f, float w) {
#pragma unroll
    for (int e = 0; e < N; e += 2) {
        if (W) fma_f32x2(acc[e], acc[e + 1], w, f[e], f[e + 1]);
        else add_f32x2(acc[e], acc[e + 1], f[e], f[e + 1]);
    }
}
// Loads of the test-vector block.  Separate launches read it through the
// read-only path; a persistent launch (k_relax) rewrites it between sweeps, so
// there it is read coherently from L2, and the per-sweep scale and centre come
// from shared memory.
template <bool P>
__device__ __forceinline__ uint4 ldx(const uint4 *p) { return P ? __ldcg(p) : __ldg(p); }
template <bool P>
__device__ __forceinline__ float4 ldac(const float *p) {
    return P ? *reinterpret_cast<const float4 *>(p) : __ldg(reinterpret_cast<const float4 *>(p));
}

template <typename T, int LPR, int CPL>
struct Lane {
    static constexpr int V = Store<T>::V;
    static constexpr int E = CPL * V;       // elements held by one lane
    static constexpr int G = 32 / LPR;      // groups per warp
};

// Gather-accumulate rows col[p] for p in [p0, p1) with the whole warp: group
// grp takes every G-th neighbour.  Column indices (and weights) are read 32 at
// a time, coalesced, and broadcast with shuffles; the next 32 are loaded
// before the current ones are used, so their latency overlaps the row loads.
// Each lane issues up to UB independent 16-byte row loads before it consumes
// any of them, so that enough requests are in flight to cover the L2 latency.
// W: edge weights present; without them no weight is read or broadcast and
// the rows are plainly added (the same sums as fmaf with weight 1).
template <typename T, int LPR, int CPL, bool W, bool P>
__device__ __forceinline__ void warp_gather_w(const SweepArgs &a, int64_t p0, int64_t p1, int lane, int grp,
                                              int gl, float (&acc)[CPL * Store<T>::V]) {
    using L = Lane<T, LPR, CPL>;
    constexpr int V = L::V, G = L::G;
    constexpr int U = 32 / G;                       // neighbours per group per batch of 32
    constexpr int UBc = AD_SWEEP_UB / CPL > 0 ? AD_SWEEP_UB / CPL : 1;
    constexpr int UB = UBc < U ? UBc : U;          // loads in flight per chunk slot
    const uint4 *X = reinterpret_cast<const uint4 *>(a.x_in);
    const int64_t row_q = a.stride / V;   // 16-byte chunks per row
    int32_t cjn = 0;
    float wjn = 0.f;
    if (p0 + lane < p1) {
        cjn = ld_stream(a.col + p0 + lane);
        if (W) wjn = ld_stream(a.w + p0 + lane);
    }
    for (int64_t base = p0; base < p1; base += 32) {
        const int32_t cj = cjn;
        const float wj = wjn;
        const int64_t pn = base + 32 + lane;
        if (pn < p1) {
            cjn = ld_stream(a.col + pn);
            if (W) wjn = ld_stream(a.w + pn);
        }
        const int cnt = (int)(p1 - base < 32 ? p1 - base : 32);
#pragma unroll
        for (int u0 = 0; u0 < U; u0 += UB) {
            if (u0 * G >= cnt) break;
            uint4 v[UB][CPL];
            float wt[UB];
#pragma unroll
            for (int u = 0; u < UB; ++u) {
                const int src = (u0 + u) * G + grp;
                const int32_t nb = __shfl_sync(0xffffffffu, cj, src);
                if (W) wt[u] = __shfl_sync(0xffffffffu, wj, src);
#pragma unroll
                for (int c = 0; c < CPL; ++c) {
                    const int q = gl + c * LPR;
                    v[u][c] = (src < cnt && q < a.nchunks) ? ldx<P>(X + (int64_t)nb * row_q + q) : make_uint4(0, 0, 0, 0);
                }
            }
#pragma unroll
            for (int u = 0; u < UB; ++u)
#pragma unroll
                for (int c = 0; c < CPL; ++c) {
                    float f[V];
                    Store<T>::unpack(v[u][c], f);
                    accumulate<V, W>(acc + c * V, f, W ? wt[u] : 1.f);
                }
        }
    }
}

template <typename T, int LPR, int CPL, bool P>
__device__ __forceinline__ void warp_gather(const SweepArgs &a, int64_t p0, int64_t p1, int lane, int grp,
                                            int gl, float (&acc)[CPL * Store<T>::V]) {
    if (!a.w) {   // the weighted loop reads a.w: it is reached only with weights present
        warp_gather_w<T, LPR, CPL, false, P>(a, p0, p1, lane, grp, gl, acc);
        return;
    }
    warp_gather_w<T, LPR, CPL, true, P>(a, p0, p1, lane, grp, gl, acc);
}

// Gather-accumulate a short row (<= kSmallUnroll entries per round) with one
// lane group: all of its column indices, then all row loads, then the sums.
constexpr int kSmallUnroll = AD_SWEEP_UB;
template <typename T, int LPR, int CPL, bool W, bool P>
__device__ __forceinline__ void group_gather_w(const SweepArgs &a, int64_t p0, int64_t p1, int gl,
                                               float (&acc)[CPL * Store<T>::V]) {
    constexpr int V = Store<T>::V;
    constexpr int UB = (kSmallUnroll / CPL) > 0 ? (kSmallUnroll / CPL) : 1;
    const uint4 *X = reinterpret_cast<const uint4 *>(a.x_in);
    const int64_t row_q = a.stride / V;
    for (int64_t base = p0; base < p1; base += UB) {
        int32_t nb[UB];
        float wt[UB];
#pragma unroll
        for (int u = 0; u < UB; ++u) {
            const bool ok = base + u < p1;
            nb[u] = ok ? ld_stream(a.col + base + u) : 0;
            if (W) wt[u] = ok ? ld_stream(a.w + base + u) : 0.f;
        }
        uint4 v[UB][CPL];
#pragma unroll
        for (int u = 0; u < UB; ++u)
#pragma unroll
            for (int c = 0; c < CPL; ++c) {
                const int q = gl + c * LPR;
                v[u][c] = (base + u < p1 && q < a.nchunks) ? ldx<P>(X + (int64_t)nb[u] * row_q + q) : make_uint4(0, 0, 0, 0);
            }
#pragma unroll
        for (int u = 0; u < UB; ++u)
#pragma unroll
            for (int c = 0; c < CPL; ++c) {
                float f[V];
                Store<T>::unpack(v[u][c], f);
                accumulate<V, W>(acc + c * V, f, W ? wt[u] : 1.f);
            }
    }
}

template <typename T, int LPR, int CPL, bool P>
__device__ __forceinline__ void group_gather(const SweepArgs &a, int64_t p0, int64_t p1, int gl,
                                             float (&acc)[CPL * Store<T>::V]) {
    if (!a.w) {   // the weighted loop reads a.w: it is reached only with weights present
        group_gather_w<T, LPR, CPL, false, P>(a, p0, p1, gl, acc);
        return;
    }
    group_gather_w<T, LPR, CPL, true, P>(a, p0, p1, gl, acc);
}

// Sum over the G groups of a warp (butterfly: every group ends with the total).
template <int LPR, int E>
__device__ __forceinline__ void reduce_groups(float (&acc)[E]) {
#pragma unroll
    for (int off = LPR; off < 32; off <<= 1)
#pragma unroll
        for (int e = 0; e < E; ++e) acc[e] += __shfl_xor_sync(0xffffffffu, acc[e], off);
}

// Epilogue of a row: z = (1-omega) s_i + omega Dinv_i S, store a (z - c), track min/max.
template <typename T, int LPR, int CPL, bool P = false>
__device__ __forceinline__ void load_own(const SweepArgs &a, int64_t row, int gl, uint4 (&own)[CPL]) {
    const uint4 *X = reinterpret_cast<const uint4 *>(a.x_in);
    const int64_t row_q = a.stride / Store<T>::V;
#pragma unroll
    for (int c = 0; c < CPL; ++c) {
        const int q = gl + c * LPR;
        own[c] = q < a.nchunks ? ldx<P>(X + row * row_q + q) : make_uint4(0, 0, 0, 0);
    }
}

template <typename T, int LPR, int CPL, bool P = false>
__device__ __forceinline__ void row_epilogue(const SweepArgs &a, int64_t row, int gl, const uint4 (&own)[CPL],
                                             const float (&S)[CPL * Store<T>::V], const float *acg,
                                             float (&mn)[CPL * Store<T>::V], float (&mx)[CPL * Store<T>::V]) {
    constexpr int V = Store<T>::V;
    uint4 *Y = reinterpret_cast<uint4 *>(a.x_out);
    const int64_t row_q = a.stride / V;
    const float dinv = __ldg(a.Dinv + row);
    const float om = a.omega, om1 = 1.f - a.omega;
#pragma unroll
    for (int c = 0; c < CPL; ++c) {
        const int q = gl + c * LPR;
        if (q < a.nchunks) {
            float y[V], o[V], A[V], C[V];
            Store<T>::unpack(own[c], y);
#pragma unroll
            for (int e4 = 0; e4 < V / 4; ++e4) {   // scale and centre of the row's graph (the same line for every row)
                const float4 av = ldac<P>(acg + q * V + 4 * e4);
                const float4 cv = ldac<P>(acg + a.stride + q * V + 4 * e4);
                A[4 * e4] = av.x; A[4 * e4 + 1] = av.y; A[4 * e4 + 2] = av.z; A[4 * e4 + 3] = av.w;
                C[4 * e4] = cv.x; C[4 * e4 + 1] = cv.y; C[4 * e4 + 2] = cv.z; C[4 * e4 + 3] = cv.w;
            }
#pragma unroll
            for (int e = 0; e < V; ++e) {
                const float z = fmaf(om1, y[e], om * (S[c * V + e] * dinv));
                o[e] = Store<T>::round(A[e] * (z - C[e]));
                mn[c * V + e] = fminf(mn[c * V + e], o[e]);
                mx[c * V + e] = fmaxf(mx[c * V + e], o[e]);
            }
            Y[row * row_q + q] = Store<T>::pack(o);
        }
    }
}

// Scale a = 1 / (max - min) of the previous sweep's stored values for the
// lane's elements (1 before the first sweep, 0 for a vector with max == min).
template <typename T, int LPR, int CPL, bool P = false>
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
                const float lo = ord2f(P ? __ldcg(pmin + r) : pmin[r]), hi = ord2f(P ? __ldcg(pmax + r) : pmax[r]);
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

// ----------------------------------------------------------------------------
// One JOR sweep (Alg. 1 inner loop) over all rows of degree > 0.
// ----------------------------------------------------------------------------
// Sum of the partial rows of one high-degree row (its chunks t0 .. t0 +
// nchunk - 1): group g adds partials g, g + G, ... in order, then the groups'
// sums are added (once per high-degree row).
template <typename T, int LPR, int CPL>
__device__ __forceinline__ void sum_partials(const SweepArgs &a, int64_t t0, int32_t nchunk, int grp, int gl, float (&S)[CPL * Store<T>::V]) {
    constexpr int V = Store<T>::V, E = CPL * V, G = 32 / LPR;
#pragma unroll
    for (int e = 0; e < E; ++e) S[e] = 0.f;
    for (int32_t cc2 = grp; cc2 < nchunk; cc2 += G) {
        const float4 *pp = reinterpret_cast<const float4 *>(a.part + (t0 + cc2) * (int64_t)a.stride);
#pragma unroll
        for (int cc = 0; cc < CPL; ++cc) {
            const int q = gl + cc * LPR;
            if (q < a.nchunks) {
#pragma unroll
                for (int e4 = 0; e4 < V / 4; ++e4) {
                    const float4 f = __ldcg(pp + (q * V) / 4 + e4);
                    S[cc * V + 4 * e4 + 0] += f.x;
                    S[cc * V + 4 * e4 + 1] += f.y;
                    S[cc * V + 4 * e4 + 2] += f.z;
                    S[cc * V + 4 * e4 + 3] += f.w;
                }
            }
        }
    }
    reduce_groups<LPR, E>(S);
}

// More warps per SM hide more of the gather latency even at the cost of a few
// spilled registers: measured best at 6 CTAs (FP32) and 5 (16-bit) per SM.
template <typename T>
constexpr int sweep_minb() { return sizeof(T) == 4 ? AD_SWEEP_MINB : AD_SWEEP_MINB16; }

// The tasks of one sweep on this CTA, then the CTA's min/max to the sweep's
// slots.  P: inside the persistent launch (acs = the scale and centre of the
// single graph in shared memory).
template <typename T, int LPR, int CPL, bool P>
__device__ __forceinline__ void sweep_tasks(const SweepArgs &a, float *sm, const float *acs) {
    using L = Lane<T, LPR, CPL>;
    constexpr int V = L::V, E = L::E, G = L::G;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
    const int grp = lane / LPR, gl = lane % LPR;

    LaneStats<T, LPR, CPL> ls;
    ls.enter(a, gl, 0, false);
    if (P) ls.acg = acs;
    GraphCache gcache;
    auto row_graph = [&](int64_t row) { return a.G > 1 ? gcache.of(a.voff, a.G, row) : 0; };

    const int64_t W = (int64_t)gridDim.x * nwarps;
    const TaskIter it = task_iter(a.n_tasks, (int64_t)blockIdx.x * nwarps + warp, W, a.blocked);
    for (int64_t task = it.t; task < it.t_end; task += it.step) {
        float acc[E];
#pragma unroll
        for (int e = 0; e < E; ++e) acc[e] = 0.f;
        if (task < a.n_big) {
            // ---- a chunk of a high-degree row; the last chunk combines
            const int64_t row = a.big_row[task];
            const int32_t c = a.big_chunk[task];
            const int64_t rb = a.rp[row], re = a.rp[row + 1];
            const int64_t p0 = rb + (int64_t)c * kChunk, p1 = min(re, p0 + kChunk);
            warp_gather<T, LPR, CPL, P>(a, p0, p1, lane, grp, gl, acc);
            reduce_groups<LPR, E>(acc);
            float *part = a.part + task * (int64_t)a.stride;
            if (grp == 0) {
#pragma unroll
                for (int cc = 0; cc < CPL; ++cc) {
                    const int q = gl + cc * LPR;
                    if (q < a.nchunks) {
#pragma unroll
                        for (int e = 0; e < V; ++e) __stcg(part + q * V + e, acc[cc * V + e]);
                    }
                }
                __threadfence();
            }
            __syncwarp();
            const int64_t t0 = task - c;
            const int32_t nchunk = (int32_t)((re - rb + kChunk - 1) / kChunk);
            uint32_t old = 0;
            if (lane == 0) old = atomicAdd(a.big_counter + t0, 1u);
            old = __shfl_sync(0xffffffffu, old, 0);
            if (old == (uint32_t)(nchunk - 1)) {
                __threadfence();
                // group g sums partials g, g + G, ... (fixed order); then the groups' sums are added
                uint4 own[CPL];
                load_own<T, LPR, CPL, P>(a, row, gl, own);
                float S[E];
                sum_partials<T, LPR, CPL>(a, t0, nchunk, grp, gl, S);
                if (grp == 0) {
                    ls.enter(a, gl, row_graph(row), true);
                    row_epilogue<T, LPR, CPL, P>(a, row, gl, own, S, ls.acg, ls.mn, ls.mx);
                }
                if (lane == 0) a.big_counter[t0] = 0u;
            }
        } else if (task < a.n_big + a.n_medium) {
            // ---- one row, whole warp
            const int64_t row = a.medium_row[task - a.n_big];
            uint4 own[CPL];
            load_own<T, LPR, CPL, P>(a, row, gl, own);
            warp_gather<T, LPR, CPL, P>(a, a.rp[row], a.rp[row + 1], lane, grp, gl, acc);
            reduce_groups<LPR, E>(acc);
            if (grp == 0) {
                ls.enter(a, gl, row_graph(row), true);
                row_epilogue<T, LPR, CPL, P>(a, row, gl, own, acc, ls.acg, ls.mn, ls.mx);
            }
        } else {
            // ---- G low-degree rows, one per lane group
            const int64_t si = (task - a.n_big - a.n_medium) * G + grp;
            if (si < a.n_small_rows) {
                const int64_t row = a.small_row[si];
                uint4 own[CPL];
                load_own<T, LPR, CPL, P>(a, row, gl, own);
                group_gather<T, LPR, CPL, P>(a, a.rp[row], a.rp[row + 1], gl, acc);
                ls.enter(a, gl, row_graph(row), true);
                row_epilogue<T, LPR, CPL, P>(a, row, gl, own, acc, ls.acg, ls.mn, ls.mx);
            }
        }
    }

    // ---- min/max of what this CTA stored -> atomics
    if (a.G > 1) {
        // lanes of a warp that share one graph are reduced first
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

template <typename T, int LPR, int CPL>
__global__ void __launch_bounds__(256, sweep_minb<T>()) k_sweep(SweepArgs a) {
    extern __shared__ float sm[];   // [2][warps][stride]
    sweep_tasks<T, LPR, CPL, false>(a, sm, nullptr);
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

template <typename T, int LPR, int CPL, bool P>
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
        if (q < a.nchunks) Store<T>::unpack(ldx<P>(X + row * row_q + q), yi + c * V);
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
                v[u][c] = (pb + (int64_t)u * step < p1 && q < a.nchunks) ? ldx<P>(X + (int64_t)jn[u] * row_q + q)
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
        constexpr int WS = LPR > UB ? LPR / UB : 1;   // lanes per edge that hold the same sum
        const bool writer = gl % WS == 0;
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

template <typename T, int LPR, int CPL, bool P>
__device__ __forceinline__ void distance_tasks(const SweepArgs &a) {
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
        load_scale<T, LPR, CPL, P>(a.mm_prev_min ? a.mm_prev_min + (size_t)g * a.stride : nullptr,
                                a.mm_prev_max ? a.mm_prev_max + (size_t)g * a.stride : nullptr, gl, A);
#pragma unroll
        for (int c = 0; c < CPL; ++c)
#pragma unroll
            for (int e = 0; e < V; ++e) {
                const int r = (gl + c * LPR) * V + e;
                A2[c * V + e] = (r < a.R) ? A[c * V + e] * A[c * V + e] : 0.f;
            }
    };
    GraphCache gcache;
    auto row_graph = [&](int64_t row) { return a.G > 1 ? gcache.of(a.voff, a.G, row) : 0; };
    const int64_t W = (int64_t)gridDim.x * nwarps;
    const TaskIter it = task_iter(a.n_tasks, (int64_t)blockIdx.x * nwarps + warp, W, a.blocked);
    for (int64_t task = it.t; task < it.t_end; task += it.step) {
        if (task < a.n_big) {
            const int64_t row = a.big_row[task];
            const int32_t c = a.big_chunk[task];
            const int64_t ub = a.upos[row], ue = a.rp[row + 1];
            const int64_t p0 = ub + (int64_t)c * kChunk, p1 = min(ue, p0 + kChunk);
            enter(row_graph(row));
            edge_rows<T, LPR, CPL, P>(a, row, p0, p1, G, grp, gl, gmask, A2);
        } else if (task < a.n_big + a.n_medium) {
            const int64_t row = a.medium_row[task - a.n_big];
            enter(row_graph(row));
            edge_rows<T, LPR, CPL, P>(a, row, a.upos[row], a.rp[row + 1], G, grp, gl, gmask, A2);
        } else {
            const int64_t si = (task - a.n_big - a.n_medium) * G + grp;
            if (si < a.n_small_rows) {
                const int64_t row = a.small_row[si];
                enter(row_graph(row));
                edge_rows<T, LPR, CPL, P>(a, row, a.upos[row], a.rp[row + 1], 1, 0, gl, gmask, A2);
            }
        }
    }
}

template <typename T, int LPR, int CPL>
__global__ void __launch_bounds__(256, AD_DIST_MINB) k_distance(SweepArgs a) {
    distance_tasks<T, LPR, CPL, false>(a);
}

// ----------------------------------------------------------------------------
// Persistent relaxation: the whole of Alg. 1 for a single graph in one
// cooperative launch -- init, k sweeps, each followed by a grid-wide barrier
// (the next sweep's rescale needs every CTA's min/max), and the distances.
// The barrier is a counter that every CTA increments and then polls with an
// acquire load, at most kBarrierPolls times; a CTA that runs out writes
// AD_ERR_TIMEOUT to *err and returns, and the others stop at their next
// barrier once they see the error.
// ----------------------------------------------------------------------------
#ifndef AD_BARRIER_POLLS
#define AD_BARRIER_POLLS (1u << 25)   // with the 32 ns back-off and the loads: a few seconds
#endif

struct RelaxArgs {
    SweepArgs s;            // sweep plan and constant fields (x_in / x_out / slots set per sweep)
    SweepArgs d;            // distance plan
    int64_t n;              // vertices
    int32_t k;
    void *x0, *x1;
    uint32_t *mm_min, *mm_max;   // [k][stride]
    uint32_t seed_lo, seed_hi, stream_id;
    unsigned int *bar;      // [kBarrierSlots] arrival counters, zero before the launch
    int *err;               // zero before the launch
    unsigned int polls;     // barrier poll limit
    unsigned int extra;     // arrivals the barrier waits for beyond the grid (0; > 0 only to test the limit)
};

__device__ __forceinline__ unsigned int ld_acquire_u32(const unsigned int *p) {
    unsigned int v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void red_release_add_u32(unsigned int *p, unsigned int v) {
    asm volatile("red.release.gpu.global.add.u32 [%0], %1;" :: "l"(p), "r"(v) : "memory");
}

// Arrivals are spread over kBarrierSlots counters (CTA b adds to slot b mod
// kBarrierSlots) so that they do not queue on one address; warp 0 of every
// CTA sums the slots with acquire loads until the total reaches the target.
constexpr int kBarrierSlots = 32;

// false: the barrier timed out here or elsewhere (every thread of the CTA gets the same answer)
__device__ __forceinline__ bool grid_barrier(const RelaxArgs &r, unsigned int phase) {
    __syncthreads();
    __shared__ int ok_s;
    if (threadIdx.x < 32) {
        const int lane = threadIdx.x;
        if (lane == 0) red_release_add_u32(r.bar + (blockIdx.x % kBarrierSlots), 1u);
        const unsigned int target = (gridDim.x + r.extra) * phase;
        int ok = 1;
        unsigned int polls = 0;
        for (;;) {
            unsigned int v = ld_acquire_u32(r.bar + lane);
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
            if (v >= target) break;
            if (*(volatile int *)r.err != 0) { ok = 0; break; }
            if (++polls > r.polls) {
                if (lane == 0) atomicCAS(r.err, 0, (int)AD_ERR_TIMEOUT);
                ok = 0;
                break;
            }
            __nanosleep(32);
        }
        if (lane == 0) ok_s = ok;
    }
    __syncthreads();
    return ok_s != 0;
}

template <typename T, int LPR, int CPL>
__global__ void __launch_bounds__(256, sweep_minb<T>()) k_relax(RelaxArgs r) {
    constexpr int V = Store<T>::V;
    extern __shared__ float sm[];   // [2][warps][stride] min/max, then [2][stride] scale and centre
    float *acs = sm + 2 * (blockDim.x >> 5) * r.s.stride;
    // x0 <- rand(-0.5, 0.5) on every row of degree > 0
    init_rows<T>(r.s.rp, r.n, r.s.stride, r.seed_lo, r.seed_hi, r.stream_id, r.s.voff, 1, static_cast<T *>(r.x0));
    if (!grid_barrier(r, 1)) return;
    for (int32_t t = 0; t < r.k; ++t) {
        SweepArgs a = r.s;
        a.x_in = (t & 1) ? r.x1 : r.x0;
        a.x_out = (t & 1) ? r.x0 : r.x1;
        a.mm_prev_min = t > 0 ? r.mm_min + (size_t)(t - 1) * a.stride : nullptr;
        a.mm_prev_max = t > 0 ? r.mm_max + (size_t)(t - 1) * a.stride : nullptr;
        a.mm_min = r.mm_min + (size_t)t * a.stride;
        a.mm_max = r.mm_max + (size_t)t * a.stride;
        // scale and centre of this sweep (what k_scale_center computes), per CTA
        const uint4 *xa = reinterpret_cast<const uint4 *>(a.x_in) + (int64_t)__ldg(a.anchor) * (a.stride / V);
        for (int q = threadIdx.x; q < a.stride / V; q += blockDim.x) {
            float f[V];
            Store<T>::unpack(__ldcg(xa + q), f);
#pragma unroll
            for (int e = 0; e < V; ++e) {
                const int rr = q * V + e;
                float av = 1.f;
                if (a.mm_prev_min) {
                    const float lo = ord2f(__ldcg(a.mm_prev_min + rr)), hi = ord2f(__ldcg(a.mm_prev_max + rr));
                    av = hi > lo ? 1.f / (hi - lo) : 0.f;
                }
                acs[rr] = av;
                acs[a.stride + rr] = f[e];
            }
        }
        __syncthreads();
        sweep_tasks<T, LPR, CPL, true>(a, sm, acs);
        if (!grid_barrier(r, (unsigned int)t + 2)) return;
    }
    SweepArgs d = r.d;
    d.x_in = (r.k & 1) ? r.x1 : r.x0;
    d.mm_prev_min = r.k > 0 ? r.mm_min + (size_t)(r.k - 1) * d.stride : nullptr;
    d.mm_prev_max = r.k > 0 ? r.mm_max + (size_t)(r.k - 1) * d.stride : nullptr;
    distance_tasks<T, LPR, CPL, true>(d);
}

struct Config {
    int lpr, cpl, V, stride, nchunks;
    int per_sm = 0;   // sweep CTAs per SM (0: as many as fit)
};


template <typename T, int LPR, int CPL>
ad_status launch_sweep(ad_graph_t g, const SweepArgs &a, int blocks, size_t smem) {
    AD_LAUNCH(k_scale_center<T>, a.G, 32, 0, g->stream, a.mm_prev_min, a.mm_prev_max, a.x_in, a.anchor, a.stride,
              a.ac);
    AD_LAUNCH((k_sweep<T, LPR, CPL>), blocks, 256, smem, g->stream, a);
    return AD_OK;
}
template <typename T, int LPR, int CPL>
ad_status launch_distance(ad_graph_t g, const SweepArgs &a, int blocks) {
    AD_LAUNCH((k_distance<T, LPR, CPL>), blocks, 256, 0, g->stream, a);
    return AD_OK;
}
template <typename T, int LPR, int CPL>
int blocks_for(bool sweep, size_t smem) {
    int per_sm = 0;
    if (sweep)
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_sweep<T, LPR, CPL>, 256, smem);
    else
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_distance<T, LPR, CPL>, 256, 0);
    return per_sm > 0 ? per_sm : 1;
}

template <typename T>
ad_status dispatch(ad_graph_t g, const Config &cf, bool sweep, const SweepArgs &a, int64_t n_tasks,
                          size_t smem) {
    // persistent grid: every SM full, but no more warps than tasks
    auto run = [&](auto lpr_c, auto cpl_c) -> ad_status {
        constexpr int LPR = decltype(lpr_c)::value, CPL = decltype(cpl_c)::value;
        int per_sm = blocks_for<T, LPR, CPL>(sweep, smem);
        if (sweep && cf.per_sm > 0 && cf.per_sm < per_sm) per_sm = cf.per_sm;
        int64_t blocks = (int64_t)per_sm * g->num_sms;
        const int64_t need = (n_tasks + 7) / 8;
        if (blocks > need) blocks = need > 0 ? need : 1;
        return sweep ? launch_sweep<T, LPR, CPL>(g, a, (int)blocks, smem)
                     : launch_distance<T, LPR, CPL>(g, a, (int)blocks);
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
        // fewer lanes per row, more chunks per lane: the alternative shapes the autotuner tries
        case 102: return run(integral_constant<int, 1>{}, integral_constant<int, 2>{});
        case 202: return run(integral_constant<int, 2>{}, integral_constant<int, 2>{});
        case 402: return run(integral_constant<int, 4>{}, integral_constant<int, 2>{});
        case 802: return run(integral_constant<int, 8>{}, integral_constant<int, 2>{});
        case 1602: return run(integral_constant<int, 16>{}, integral_constant<int, 2>{});
        default: return fail(AD_ERR_INVALID_ARG, "unsupported R / storage combination");
    }
}


// Persistent launch of k_relax: every CTA co-resident (cooperative launch),
// as many as fit or as the larger of the two plans can use.
template <typename T, int LPR, int CPL>
ad_status launch_relax(ad_graph_t g, const Config &cf, RelaxArgs &r) {
    const size_t smem = (2 * 8 + 2) * (size_t)r.s.stride * sizeof(float);
    int per_sm = 0;
    AD_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_relax<T, LPR, CPL>, 256, smem));
    if (per_sm < 1) return fail(AD_ERR_CUDA, "the persistent relaxation kernel does not fit on an SM");
    if (cf.per_sm > 0 && cf.per_sm < per_sm) per_sm = cf.per_sm;
    int64_t blocks = (int64_t)per_sm * g->num_sms;
    const int64_t need = (std::max(r.s.n_tasks, r.d.n_tasks) + 7) / 8;
    if (blocks > need) blocks = need > 0 ? need : 1;
    void *args[] = {&r};
    ::ad::g_launches.fetch_add(1, std::memory_order_relaxed);
    AD_CUDA_TRY(cudaLaunchCooperativeKernel((const void *)k_relax<T, LPR, CPL>, dim3((unsigned)blocks), dim3(256), args,
                                            smem, g->stream));
    return AD_OK;
}

template <typename T>
ad_status relax_dispatch(ad_graph_t g, const Config &cf, RelaxArgs &r) {
    using std::integral_constant;
    auto run = [&](auto lpr_c, auto cpl_c) -> ad_status {
        return launch_relax<T, decltype(lpr_c)::value, decltype(cpl_c)::value>(g, cf, r);
    };
    switch (cf.lpr * 100 + cf.cpl) {
        case 101: return run(integral_constant<int, 1>{}, integral_constant<int, 1>{});
        case 201: return run(integral_constant<int, 2>{}, integral_constant<int, 1>{});
        case 401: return run(integral_constant<int, 4>{}, integral_constant<int, 1>{});
        case 801: return run(integral_constant<int, 8>{}, integral_constant<int, 1>{});
        case 1601: return run(integral_constant<int, 16>{}, integral_constant<int, 1>{});
        case 3201: return run(integral_constant<int, 32>{}, integral_constant<int, 1>{});
        case 3202: return run(integral_constant<int, 32>{}, integral_constant<int, 2>{});
        default: return fail(AD_ERR_INVALID_ARG, "the persistent relaxation takes the natural lane shapes only");
    }
}

// one instantiation per storage type, each in its own translation unit
ad_status dispatch_f32(ad_graph_t g, const Config &cf, bool sweep, const SweepArgs &a, int64_t n_tasks, size_t smem);
ad_status dispatch_bf16(ad_graph_t g, const Config &cf, bool sweep, const SweepArgs &a, int64_t n_tasks, size_t smem);
ad_status dispatch_f16(ad_graph_t g, const Config &cf, bool sweep, const SweepArgs &a, int64_t n_tasks, size_t smem);
ad_status dispatch_q16(ad_graph_t g, const Config &cf, bool sweep, const SweepArgs &a, int64_t n_tasks, size_t smem);
ad_status relax_f32(ad_graph_t g, const Config &cf, RelaxArgs &r);
ad_status relax_bf16(ad_graph_t g, const Config &cf, RelaxArgs &r);
ad_status relax_f16(ad_graph_t g, const Config &cf, RelaxArgs &r);
ad_status relax_q16(ad_graph_t g, const Config &cf, RelaxArgs &r);
ad_status launch_init(ad_graph_t g, ad_storage storage, int blocks, int32_t stride, uint64_t seed, uint32_t stream_id,
                      void *x);

}  // namespace ad
