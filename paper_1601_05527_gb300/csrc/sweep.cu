// sweep.cu -- ComputeAlgDist (Alg. 1) on sm_103a: Philox init, JOR sweeps with
// the per-sweep rescale fused into the epilogue, and the per-edge distance.
//
// Data layout: the R test vectors of vertex i form row i of X[n][stride]
// (stride = lanes_per_row * chunks_per_lane * V elements, 16-byte chunks,
// V = 4 FP32 or 8 BF16 values).  A lane group of LPR lanes owns one row at a
// time; lane gl of the group holds chunks gl, gl + LPR, ... of the row.
//
// Rescale.  Sweep t stores the raw update z = (1-omega) y_i + omega D_i^-1 sum_j
// w_ij y_j applied to the stored values y of sweep t-1, mapped through the
// affine x = a y + b that rescales sweep t-1 to [-1/2, 1/2]:
//     sum_j w_ij (a y_j + b) = a sum_j w_ij y_j + b D_i,
// so the stored value of sweep t is a z + b (the JOR operator commutes with
// per-vector affine maps).  Each sweep reduces min/max of what it stores; the
// next launch turns them into (a, b).  The distance of Alg. 1 uses the last
// affine: rho = sqrt(sum_r a_r^2 (y_i^r - y_j^r)^2).
#include "ad_internal.cuh"

#include <cmath>
#include <cstring>

namespace ad {

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
            uint2 p = make_uint2(Store<__nv_bfloat16>::pack2(v[0], v[1]), Store<__nv_bfloat16>::pack2(v[2], v[3]));
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

// Gather-accumulate rows col[p] for p in [p0, p1) with the whole warp: group
// grp takes every G-th neighbour.  Column indices (and weights) are read 32 at
// a time, coalesced, and broadcast with shuffles.
template <typename T, int LPR, int CPL>
__device__ __forceinline__ void warp_gather(const SweepArgs &a, int64_t p0, int64_t p1, int lane, int grp,
                                            int gl, float (&acc)[CPL * Store<T>::V]) {
    using L = Lane<T, LPR, CPL>;
    constexpr int V = L::V, G = L::G;
    const uint4 *X = reinterpret_cast<const uint4 *>(a.x_in);
    const int64_t row_q = a.stride / V;   // 16-byte chunks per row
    for (int64_t base = p0; base < p1; base += 32) {
        const int64_t p = base + lane;
        int32_t cj = -1;
        float wj = 0.f;
        if (p < p1) {
            cj = __ldg(a.col + p);
            wj = a.w ? __ldg(a.w + p) : 1.f;
        }
        const int cnt = (int)(p1 - base < 32 ? p1 - base : 32);
#pragma unroll 4
        for (int j = 0; j < 32; j += G) {
            if (j >= cnt) break;
            const int src = j + grp;
            const int32_t nb = __shfl_sync(0xffffffffu, cj, src);
            const float wt = __shfl_sync(0xffffffffu, wj, src);
            if (src < cnt) {
#pragma unroll
                for (int c = 0; c < CPL; ++c) {
                    const int q = gl + c * LPR;
                    if (q < a.nchunks) {
                        uint4 v = __ldg(X + (int64_t)nb * row_q + q);
                        float f[V];
                        Store<T>::unpack(v, f);
#pragma unroll
                        for (int e = 0; e < V; ++e) acc[c * V + e] = fmaf(wt, f[e], acc[c * V + e]);
                    }
                }
            }
        }
    }
}

// Sum over the G groups of a warp (butterfly: every group ends with the total).
template <int LPR, int E>
__device__ __forceinline__ void reduce_groups(float (&acc)[E]) {
#pragma unroll
    for (int off = LPR; off < 32; off <<= 1)
#pragma unroll
        for (int e = 0; e < E; ++e) acc[e] += __shfl_xor_sync(0xffffffffu, acc[e], off);
}

// Epilogue of a row: z = (1-omega) y_i + omega Dinv_i S, store a z + b, track min/max.
template <typename T, int LPR, int CPL>
__device__ __forceinline__ void row_epilogue(const SweepArgs &a, int64_t row, int gl,
                                             const float (&S)[CPL * Store<T>::V],
                                             const float (&A)[CPL * Store<T>::V],
                                             const float (&B)[CPL * Store<T>::V],
                                             float (&mn)[CPL * Store<T>::V], float (&mx)[CPL * Store<T>::V]) {
    constexpr int V = Store<T>::V;
    const uint4 *X = reinterpret_cast<const uint4 *>(a.x_in);
    uint4 *Y = reinterpret_cast<uint4 *>(a.x_out);
    const int64_t row_q = a.stride / V;
    const float dinv = __ldg(a.Dinv + row);
    const float om = a.omega, om1 = 1.f - a.omega;
#pragma unroll
    for (int c = 0; c < CPL; ++c) {
        const int q = gl + c * LPR;
        if (q < a.nchunks) {
            float y[V], o[V];
            Store<T>::unpack(__ldg(X + row * row_q + q), y);
#pragma unroll
            for (int e = 0; e < V; ++e) {
                const float z = fmaf(om1, y[e], om * (S[c * V + e] * dinv));
                o[e] = Store<T>::round(fmaf(A[c * V + e], z, B[c * V + e]));
                mn[c * V + e] = fminf(mn[c * V + e], o[e]);
                mx[c * V + e] = fmaxf(mx[c * V + e], o[e]);
            }
            Y[row * row_q + q] = Store<T>::pack(o);
        }
    }
}

// Affine (a, b) of the previous sweep's rescale for the lane's elements.
template <typename T, int LPR, int CPL>
__device__ __forceinline__ void load_affine(const uint32_t *pmin, const uint32_t *pmax, int gl,
                                            float (&A)[CPL * Store<T>::V], float (&B)[CPL * Store<T>::V]) {
    // pmin / pmax point at the slots of the row's graph (nullptr: no rescale yet)
    constexpr int V = Store<T>::V;
#pragma unroll
    for (int c = 0; c < CPL; ++c)
#pragma unroll
        for (int e = 0; e < V; ++e) {
            const int r = (gl + c * LPR) * V + e;
            float av = 1.f, bv = 0.f;
            if (pmin) {
                const double lo = ord2f(pmin[r]), hi = ord2f(pmax[r]);
                if (hi > lo) {
                    const double s = 1.0 / (hi - lo);
                    av = (float)s;
                    bv = (float)(-lo * s - 0.5);
                } else {
                    av = 0.f;
                    bv = 0.f;
                }
            }
            A[c * V + e] = av;
            B[c * V + e] = bv;
        }
}

// ----------------------------------------------------------------------------
// Running min/max of the values a lane stores, for the graph `cg` of the rows
// it handled last; flushed with atomics when the lane moves to another graph.
// ----------------------------------------------------------------------------
template <typename T, int LPR, int CPL>
struct LaneStats {
    static constexpr int V = Store<T>::V, E = CPL * V;
    float A[E], B[E], mn[E], mx[E];
    int cg = -1;

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
    // make the lane's state describe graph `g` (affine of its previous sweep)
    __device__ __forceinline__ void enter(const SweepArgs &a, int gl, int g, bool flush_old) {
        if (g == cg) return;
        if (flush_old) flush(a, gl);
        cg = g;
        load_affine<T, LPR, CPL>(a.mm_prev_min ? a.mm_prev_min + (size_t)g * a.stride : nullptr,
                                 a.mm_prev_max ? a.mm_prev_max + (size_t)g * a.stride : nullptr, gl, A, B);
#pragma unroll
        for (int e = 0; e < E; ++e) { mn[e] = INFINITY; mx[e] = -INFINITY; }
    }
};

// ----------------------------------------------------------------------------
// One JOR sweep (Alg. 1 inner loop) over all rows of degree > 0.
// ----------------------------------------------------------------------------
template <typename T, int LPR, int CPL>
__global__ void __launch_bounds__(256) k_sweep(SweepArgs a) {
    using L = Lane<T, LPR, CPL>;
    constexpr int V = L::V, E = L::E, G = L::G;
    extern __shared__ float sm[];   // [2][warps][stride]
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
    const int grp = lane / LPR, gl = lane % LPR;

    LaneStats<T, LPR, CPL> ls;
    ls.enter(a, gl, 0, false);
    auto row_graph = [&](int64_t row) { return a.G > 1 ? graph_of(a.voff, a.G, row) : 0; };

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
            warp_gather<T, LPR, CPL>(a, p0, p1, lane, grp, gl, acc);
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
                if (grp == 0) {
                    float S[E];
#pragma unroll
                    for (int e = 0; e < E; ++e) S[e] = 0.f;
                    for (int32_t cc2 = 0; cc2 < nchunk; ++cc2) {
                        const float *pp = a.part + (t0 + cc2) * (int64_t)a.stride;
#pragma unroll
                        for (int cc = 0; cc < CPL; ++cc) {
                            const int q = gl + cc * LPR;
                            if (q < a.nchunks) {
#pragma unroll
                                for (int e = 0; e < V; ++e) S[cc * V + e] += __ldcg(pp + q * V + e);
                            }
                        }
                    }
                    ls.enter(a, gl, row_graph(row), true);
                    row_epilogue<T, LPR, CPL>(a, row, gl, S, ls.A, ls.B, ls.mn, ls.mx);
                }
                if (lane == 0) a.big_counter[t0] = 0u;
            }
        } else if (task < a.n_big + a.n_medium) {
            // ---- one row, whole warp
            const int64_t row = a.medium_row[task - a.n_big];
            warp_gather<T, LPR, CPL>(a, a.rp[row], a.rp[row + 1], lane, grp, gl, acc);
            reduce_groups<LPR, E>(acc);
            if (grp == 0) {
                ls.enter(a, gl, row_graph(row), true);
                row_epilogue<T, LPR, CPL>(a, row, gl, acc, ls.A, ls.B, ls.mn, ls.mx);
            }
        } else {
            // ---- G low-degree rows, one per lane group
            const int64_t si = (task - a.n_big - a.n_medium) * G + grp;
            if (si < a.n_small_rows) {
                const int64_t row = a.small_row[si];
                const int64_t p0 = a.rp[row], p1 = a.rp[row + 1];
                const uint4 *X = reinterpret_cast<const uint4 *>(a.x_in);
                const int64_t row_q = a.stride / V;
                for (int64_t p = p0; p < p1; ++p) {
                    const int32_t nb = __ldg(a.col + p);
                    const float wt = a.w ? __ldg(a.w + p) : 1.f;
#pragma unroll
                    for (int c = 0; c < CPL; ++c) {
                        const int q = gl + c * LPR;
                        if (q < a.nchunks) {
                            float f[V];
                            Store<T>::unpack(__ldg(X + (int64_t)nb * row_q + q), f);
#pragma unroll
                            for (int e = 0; e < V; ++e) acc[c * V + e] = fmaf(wt, f[e], acc[c * V + e]);
                        }
                    }
                }
                ls.enter(a, gl, row_graph(row), true);
                row_epilogue<T, LPR, CPL>(a, row, gl, acc, ls.A, ls.B, ls.mn, ls.mx);
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

// ----------------------------------------------------------------------------
// Edge distance: for every upper entry (i, j > i) of the CSR, edge id e =
// eoff[i] + (p - upos[i]), rho_e = sqrt(sum_r a_r^2 (y_i^r - y_j^r)^2).
// A lane group handles one edge; its lanes hold different chunks of R.
// ----------------------------------------------------------------------------
template <typename T, int LPR, int CPL>
__device__ __forceinline__ void edge_rows(const SweepArgs &a, int64_t row, int64_t p0, int64_t p1, int step,
                                          int first, int gl, unsigned gmask, const float (&A2)[CPL * Store<T>::V]) {
    constexpr int V = Store<T>::V, E = CPL * V;
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
    for (int64_t p = p0 + first; p < p1; p += step) {
        const int32_t j = __ldg(a.col + p);
        float s = 0.f;
#pragma unroll
        for (int c = 0; c < CPL; ++c) {
            const int q = gl + c * LPR;
            if (q < a.nchunks) {
                float yj[V];
                Store<T>::unpack(__ldg(X + (int64_t)j * row_q + q), yj);
#pragma unroll
                for (int e = 0; e < V; ++e) {
                    const float d = yi[c * V + e] - yj[e];
                    s = fmaf(A2[c * V + e] * d, d, s);
                }
            }
        }
#pragma unroll
        for (int off = 1; off < LPR; off <<= 1) s += __shfl_xor_sync(gmask, s, off);
        if (gl == 0) {
            float rho = sqrtf(s);
            if (a.normalize) rho = (float)((double)rho * sqrt(Di * a.D[j]));
            a.rho[ebase + p] = rho;
        }
    }
}

template <typename T, int LPR, int CPL>
__global__ void __launch_bounds__(256) k_distance(SweepArgs a) {
    using L = Lane<T, LPR, CPL>;
    constexpr int V = L::V, E = L::E, G = L::G;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
    const int grp = lane / LPR, gl = lane % LPR;
    const unsigned gmask = LPR == 32 ? 0xffffffffu : (((1u << LPR) - 1u) << (grp * LPR));
    float A[E], B[E], A2[E];
    int cg = -1;
    // squared scale of the last rescale of graph g; padded vectors r >= R excluded
    auto enter = [&](int g) {
        if (g == cg) return;
        cg = g;
        load_affine<T, LPR, CPL>(a.mm_prev_min ? a.mm_prev_min + (size_t)g * a.stride : nullptr,
                                 a.mm_prev_max ? a.mm_prev_max + (size_t)g * a.stride : nullptr, gl, A, B);
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

// ----------------------------------------------------------------------------
// Host side
// ----------------------------------------------------------------------------
struct Config {
    int lpr, cpl, V, stride, nchunks;
};

static Config pick_config(int R, ad_storage storage) {
    Config c;
    c.V = storage == AD_STORAGE_BF16 ? 8 : 4;
    c.nchunks = (R + c.V - 1) / c.V;
    int p2 = 1;
    while (p2 < c.nchunks) p2 <<= 1;
    c.lpr = p2 < 32 ? p2 : 32;
    c.cpl = p2 / c.lpr;
    c.stride = p2 * c.V;
    return c;
}

// Degree bound of the group-per-row class: a group walks its row alone, so keep
// it to rows whose gathers fit a few rounds of one warp-wide pass.
static int small_max_for(int groups) { return groups >= 4 ? 2 * groups : 0; }

template <typename T, int LPR, int CPL>
static ad_status launch_sweep(ad_graph_t g, const SweepArgs &a, int blocks, size_t smem) {
    AD_LAUNCH((k_sweep<T, LPR, CPL>), blocks, 256, smem, g->stream, a);
    return AD_OK;
}
template <typename T, int LPR, int CPL>
static ad_status launch_distance(ad_graph_t g, const SweepArgs &a, int blocks) {
    AD_LAUNCH((k_distance<T, LPR, CPL>), blocks, 256, 0, g->stream, a);
    return AD_OK;
}

template <typename T, int LPR, int CPL>
static int blocks_for(bool sweep, size_t smem) {
    int per_sm = 0;
    if (sweep)
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_sweep<T, LPR, CPL>, 256, smem);
    else
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_distance<T, LPR, CPL>, 256, 0);
    return per_sm > 0 ? per_sm : 1;
}

template <typename T>
static ad_status dispatch(ad_graph_t g, const Config &cf, bool sweep, const SweepArgs &a, int64_t n_tasks,
                          size_t smem) {
    // persistent grid: every SM full, but no more warps than tasks
    auto run = [&](auto lpr_c, auto cpl_c) -> ad_status {
        constexpr int LPR = decltype(lpr_c)::value, CPL = decltype(cpl_c)::value;
        int per_sm = blocks_for<T, LPR, CPL>(sweep, smem);
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
        default: return fail(AD_ERR_INVALID_ARG, "unsupported R / storage combination");
    }
}

static ad_status get_plan(ad_graph_t g, int groups, bool upper, RowPlan **out) {
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

ad_status algebraic_distance(ad_graph_t g, int32_t R, int32_t k, double omega, uint64_t seed,
                             uint32_t stream_id, ad_storage storage, int32_t flags, float *rho_dev) {
    const Config cf = pick_config(R, storage);
    const int groups = 32 / cf.lpr;
    const size_t esz = storage == AD_STORAGE_BF16 ? 2 : 4;
    const size_t xbytes = (size_t)g->n * cf.stride * esz + 256;
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

    // init
    {
        const int64_t total = g->n * (cf.stride / 4);
        int64_t blocks = (total + 255) / 256;
        if (blocks > (int64_t)g->num_sms * 16) blocks = (int64_t)g->num_sms * 16;
        if (blocks < 1) blocks = 1;
        ev_begin(g);
        if (storage == AD_STORAGE_BF16) {
            AD_LAUNCH(k_init<__nv_bfloat16>, (int)blocks, 256, 0, g->stream, g->rp, g->n, cf.stride,
                      (uint32_t)seed, (uint32_t)(seed >> 32), stream_id, g->voff, g->G,
                      static_cast<__nv_bfloat16 *>(g->x0.ptr));
        } else {
            AD_LAUNCH(k_init<float>, (int)blocks, 256, 0, g->stream, g->rp, g->n, cf.stride, (uint32_t)seed,
                      (uint32_t)(seed >> 32), stream_id, g->voff, g->G, static_cast<float *>(g->x0.ptr));
        }
        ev_end(g, g->init_ms, g->init_launches);
    }

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

    void *xin = g->x0.ptr, *xout = g->x1.ptr;
    const size_t smem = 2 * 8 * (size_t)cf.stride * sizeof(float);
    fill_plan(a, *sp);
    for (int32_t t = 0; t < k; ++t) {
        a.x_in = xin; a.x_out = xout;
        const size_t slot = (size_t)g->G * cf.stride;
        a.mm_prev_min = t > 0 ? mm_min + (size_t)(t - 1) * slot : nullptr;
        a.mm_prev_max = t > 0 ? mm_max + (size_t)(t - 1) * slot : nullptr;
        a.mm_min = mm_min + (size_t)t * slot;
        a.mm_max = mm_max + (size_t)t * slot;
        ev_begin(g);
        if (storage == AD_STORAGE_BF16) AD_TRY(dispatch<__nv_bfloat16>(g, cf, true, a, a.n_tasks, smem));
        else AD_TRY(dispatch<float>(g, cf, true, a, a.n_tasks, smem));
        ev_end(g, g->sweep_ms, g->sweep_launches);
        void *tmp = xin; xin = xout; xout = tmp;
    }

    fill_plan(a, *dp);
    a.x_in = xin;
    a.mm_prev_min = k > 0 ? mm_min + (size_t)(k - 1) * g->G * cf.stride : nullptr;
    a.mm_prev_max = k > 0 ? mm_max + (size_t)(k - 1) * g->G * cf.stride : nullptr;
    a.rho = rho_dev;
    ev_begin(g);
    if (g->m > 0) {
        if (storage == AD_STORAGE_BF16) AD_TRY(dispatch<__nv_bfloat16>(g, cf, false, a, a.n_tasks, 0));
        else AD_TRY(dispatch<float>(g, cf, false, a, a.n_tasks, 0));
    }
    ev_end(g, g->dist_ms, g->dist_launches);
    return AD_OK;
}

}  // namespace ad
