// grad.cu -- reverse mode of ComputeAlgDist (per-sweep rescale form of Alg. 1)
// with respect to the undirected edge weights.
//
// Forward (sweep_kernels.cuh stores the frame s_t, rescaled iterate
// x_t = a_t s_t + b_t with a_t = 1/(max - min)(s_t), b_t = -a_t min(s_t) - 1/2,
// x_0 = s_0 = the Philox init):
//     y_t = M x_{t-1},  M = (1-omega) I + omega D^-1 W,   x_t = rescale(y_t),
//     rho_e = |x_k,i - x_k,j|.
// Given rhobar = dL/drho, backwards for t = k .. 1:
//     xbar_k,i   = sum_j c_ij (x_k,i - x_k,j),  c_ij = rhobar_e / rho_e (0 if rho_e = 0)
//     ybar_t     = a_t xbar_t + e_argmin a_t A_t - e_argmax a_t B_t,
//                  A_t = sum_i xbar_t,i (x_t,i - 1/2),  B_t = sum_i xbar_t,i (x_t,i + 1/2)
//                  (lowest-index argmin/argmax; ybar = 0 when max == min)
//     xbar_{t-1} = (1-omega) ybar_t + omega W (D^-1 ybar_t)        (W symmetric)
//     dL/dw_ij  += omega ybar_t,i . (x_{t-1,j} - avg_i) / D_i,   avg_i = D_i^-1 sum_l w_il x_{t-1,l}
// and in the stored frame x_{t-1,j} - avg_i = a_{t-1} (s_{t-1,j} - sigma_i) with
// sigma_i = D_i^-1 sum_l w_il s_{t-1,l}.  Per CSR entry p = (i, j) the kernels
// accumulate G_p = sum_t v_i . s_{t-1,j} and per row C_i = sum_t v_i . sigma_i with
// v_i = ybar_t,i * a_{t-1}; then dL/dw_e = omega (G_p - C_i) / D_i + omega (G_q - C_j) / D_j
// for the two entries p = (i, j), q = (j, i) of edge e.  All sums are in a fixed
// order (no floating-point atomics), G and C in FP64.
//
// Memory: the stored vectors after sweeps 0, c, 2c, ... (c = ceil(sqrt k)) are
// kept by the forward; each segment of c sweeps is recomputed from its
// checkpoint when the backward reaches it.
#include "sweep_kernels.cuh"

#include <algorithm>
#include <climits>
#include <cmath>
#include <cstring>

struct ad_graph_s::Saved {
    int32_t R = 0, k = 0, c = 1;
    bool all = false;             // ckpt holds every iterate s_0 .. s_k (c = 1)
    double omega = 0.5;
    int32_t stride = 0, nchunks = 0, lpr = 1, cpl = 1;
    std::vector<void *> ckpt;     // stored vectors after sweep 0, c, 2c, ... (all: after every sweep)
    uint32_t *mm = nullptr;       // [2][k][stride] min then max slots of every sweep
    float *rho = nullptr;         // forward distances
};

namespace ad {

void free_saved(ad_graph_t g) {
    if (!g->saved) return;
    for (void *p : g->saved->ckpt) dfree(g, p);
    if (g->saved->mm) dfree(g, g->saved->mm);
    if (g->saved->rho) dfree(g, g->saved->rho);
    delete g->saved;
    g->saved = nullptr;
}

ad_status algebraic_distance_keep(ad_graph_t g, int32_t R, int32_t k, double omega, uint64_t seed, uint32_t stream_id,
                                  float *rho_dev, bool sqrt_checkpoints) {
    if (g->G != 1) return fail(AD_ERR_INVALID_ARG, "the reverse mode takes a single graph, not a batch");
    free_saved(g);
    auto *sv = new ad_graph_s::Saved();
    g->saved = sv;
    sv->R = R;
    sv->k = k;
    sv->omega = omega;
    const int V = 4;
    const int nch = (R + V - 1) / V;
    int p2 = 1;
    while (p2 < nch) p2 <<= 1;
    sv->nchunks = nch;
    sv->lpr = p2 < 32 ? p2 : 32;
    sv->cpl = p2 / sv->lpr;
    sv->stride = p2 * V;
    const size_t xbytes = ((size_t)g->n + 1) * sv->stride * sizeof(float);
    // every iterate s_0 .. s_k when they fit in half of the free memory (the
    // backward then recomputes nothing), else s_0, s_c, s_2c, ... with c = ceil(sqrt k)
    size_t free_b = 0, total_b = 0;
    const bool all = !sqrt_checkpoints && k > 0 && cudaMemGetInfo(&free_b, &total_b) == cudaSuccess &&
                     (size_t)(k + 1) * xbytes <= free_b / 2;
    int c = 1;
    if (!all)
        while ((int64_t)c * c < k) ++c;
    sv->c = c;
    sv->all = all;
    KeepSpec ks;
    ks.every = c;
    const int nck = all ? k + 1 : k > 0 ? (k + c - 1) / c : 1;
    for (int j = 0; j < nck; ++j) {
        void *p = nullptr;
        AD_TRY(dalloc(g, xbytes, &p));
        sv->ckpt.push_back(p);
    }
    ks.ckpt = sv->ckpt;
    AD_TRY(dalloc_t(g, 2 * (size_t)(k > 0 ? k : 1) * sv->stride, &sv->mm));
    ks.mm_copy = sv->mm;
    AD_TRY(algebraic_distance(g, R, k, omega, seed, stream_id, AD_STORAGE_FP32, 0, rho_dev, &ks));
    AD_TRY(dalloc_t(g, g->m + 1, &sv->rho));
    if (g->m > 0)
        AD_CUDA_TRY(cudaMemcpyAsync(sv->rho, rho_dev, g->m * sizeof(float), cudaMemcpyDeviceToDevice, g->stream));
    return AD_OK;
}

// ----------------------------------------------------------------------------
// Kernels (FP32 stored vectors)
// ----------------------------------------------------------------------------
struct BwArgs {
    const int64_t *rp;
    const int32_t *col;
    const float *w;
    const float *Dinv;
    const int64_t *eid;
    int32_t stride, nchunks, R;
    float omega;
    // distance backward
    const float *rho, *rhobar;
    const float *a_k;            // [stride] per-vector scale of the last iterate (device)
    // sweep backward
    const float *U;              // D^-1 ybar_t
    const float *Sprev;          // stored s_{t-1}
    int32_t gpitch;              // row pitch (floats) of U and Sprev in the adjoint gather
    const float *Ybar;           // ybar_t
    const float *a_prev;         // [stride] a_{t-1} (device; nullptr: 1, for t = 1)
    const float *Sk;             // stored s_k (distance backward input)
    float *xbar_out;
    double *G;                   // [nnz]
    double *C;                   // [n]
    float *part;                 // [n_big][2][stride]
    // plan
    const int32_t *big_row, *big_chunk, *medium_row, *small_row;
    uint32_t *big_counter;
    int64_t n_big, n_medium, n_small_rows, n_tasks;
    int mode;                    // 0: distance backward, 1: sweep backward
};

template <int CPL>
__device__ __forceinline__ void ld4(const float *base, int64_t row, int stride, int q, float *out) {
    const float4 f = __ldg(reinterpret_cast<const float4 *>(base + row * stride) + q);
    out[0] = f.x; out[1] = f.y; out[2] = f.z; out[3] = f.w;
}

template <int LPR, int CPL>
__device__ __forceinline__ void bw_gather_adjoint(const BwArgs &a, int64_t p0, int64_t p1, int first, int gstride,
                                                  int gl, unsigned gmask, const float (&v)[CPL * 4],
                                                  float (&acc_a)[CPL * 4], float (&acc_b)[CPL * 4]);

// One row (or chunk of a row) p in [p0, p1) processed by the warp (G groups
// over neighbours) or by one group (G = 1 group, gstride = 1).
//   mode 0: acc_a = sum c_p s_j, acc_b = sum c_p (scalar in slot 0)
//   mode 1: acc_a = sum w U_j, acc_b = sum w s_j, G_p += v_i . s_j (bw_gather_adjoint)
template <int LPR, int CPL>
__device__ __forceinline__ void bw_gather(const BwArgs &a, int64_t row, int64_t p0, int64_t p1, int first, int gstride,
                                          int gl, unsigned gmask, const float (&v)[CPL * 4], float (&acc_a)[CPL * 4],
                                          float (&acc_b)[CPL * 4]) {
    if (a.mode == 1) {
        bw_gather_adjoint<LPR, CPL>(a, p0, p1, first, gstride, gl, gmask, v, acc_a, acc_b);
        return;
    }
    for (int64_t p = p0 + first; p < p1; p += gstride) {
        const int32_t j = __ldg(a.col + p);
        {
            const int64_t e = a.eid[p];
            const float r = a.rho[e];
            const float cf = r > 0.f ? a.rhobar[e] / r : 0.f;
#pragma unroll
            for (int c = 0; c < CPL; ++c) {
                const int q = gl + c * LPR;
                if (q < a.nchunks) {
                    float s[4];
                    ld4<CPL>(a.Sk, j, a.stride, q, s);
#pragma unroll
                    for (int e4 = 0; e4 < 4; ++e4) acc_a[c * 4 + e4] = fmaf(cf, s[e4], acc_a[c * 4 + e4]);
                }
            }
            acc_b[0] += cf;
        }
    }
}

// mode 1 in batches of kBwUB neighbours per group: all their loads are issued
// before any is used, and the per-entry dots are summed over the group's lanes
// together (group_sums)
#ifndef AD_BW_UB
#define AD_BW_UB 8            // neighbours in flight per group (measured at R-MAT 22: 8 with 3 CTAs per SM fastest)
#endif
#ifndef AD_BW_GPF
#define AD_BW_GPF 1
#endif

constexpr int kBwUB = AD_BW_UB;
template <int LPR, int CPL>
__device__ __forceinline__ void bw_gather_adjoint(const BwArgs &a, int64_t p0, int64_t p1, int first, int gstride,
                                                  int gl, unsigned gmask, const float (&v)[CPL * 4],
                                                  float (&acc_a)[CPL * 4], float (&acc_b)[CPL * 4]) {
    constexpr int UB = kBwUB;
    constexpr int NH = UB / LPR > 0 ? UB / LPR : 1;
    constexpr int WS = LPR > UB ? LPR / UB : 1;   // lanes per entry that hold the same dot
    const bool writer = gl % WS == 0;
    // the entries whose dots this lane will hold after group_sums
    int which = 0;
#pragma unroll
    for (int o = LPR / 2, c = UB; o >= 1; o >>= 1)
        if (c > 1) {
            if (gl & o) which += c / 2;
            c >>= 1;
        }
    for (int64_t pb = p0 + first; pb < p1; pb += (int64_t)gstride * UB) {
        int32_t jn[UB];
        float wt[UB];
#pragma unroll
        for (int u = 0; u < UB; ++u) {
            const int64_t p = pb + (int64_t)u * gstride;
            const bool ok = p < p1;
            jn[u] = ok ? __ldg(a.col + p) : 0;
            wt[u] = ok ? (a.w ? __ldg(a.w + p) : 1.f) : 0.f;
        }
#if AD_BW_GPF
        // the accumulators of those entries, loaded with the rows so that their latency overlaps
        double gold[NH];
#pragma unroll
        for (int i = 0; i < NH; ++i) {
            const int64_t p = pb + (int64_t)(which + i) * gstride;
            gold[i] = (writer && p < p1) ? __ldcg(a.G + p) : 0.0;
        }
#endif
        float4 uu[UB][CPL], ss[UB][CPL];
#pragma unroll
        for (int u = 0; u < UB; ++u)
#pragma unroll
            for (int c = 0; c < CPL; ++c) {
                const int q = gl + c * LPR;
                const bool ok = pb + (int64_t)u * gstride < p1 && q < a.nchunks;
                uu[u][c] = ok ? __ldg(reinterpret_cast<const float4 *>(a.U + (int64_t)jn[u] * a.gpitch) + q)
                              : make_float4(0.f, 0.f, 0.f, 0.f);
                ss[u][c] = ok ? __ldg(reinterpret_cast<const float4 *>(a.Sprev + (int64_t)jn[u] * a.gpitch) + q)
                              : make_float4(0.f, 0.f, 0.f, 0.f);
            }
        float dot[UB];
#pragma unroll
        for (int u = 0; u < UB; ++u) {
            dot[u] = 0.f;
#pragma unroll
            for (int c = 0; c < CPL; ++c) {
                const float uf[4] = {uu[u][c].x, uu[u][c].y, uu[u][c].z, uu[u][c].w};
                const float sf[4] = {ss[u][c].x, ss[u][c].y, ss[u][c].z, ss[u][c].w};
#pragma unroll
                for (int e4 = 0; e4 < 4; ++e4) {
                    acc_a[c * 4 + e4] = fmaf(wt[u], uf[e4], acc_a[c * 4 + e4]);
                    acc_b[c * 4 + e4] = fmaf(wt[u], sf[e4], acc_b[c * 4 + e4]);
                    dot[u] = fmaf(v[c * 4 + e4], sf[e4], dot[u]);
                }
            }
        }
        int w2 = 0;
        group_sums<LPR, UB>(dot, gl, gmask, w2);
#pragma unroll
        for (int i = 0; i < NH; ++i) {
            const int64_t p = pb + (int64_t)(which + i) * gstride;
#if AD_BW_GPF
            if (writer && p < p1) a.G[p] = gold[i] + (double)dot[i];
#else
            if (writer && p < p1) a.G[p] += (double)dot[i];
#endif
        }
    }
}

template <int LPR, int CPL>
__device__ __forceinline__ void bw_finish(const BwArgs &a, int64_t row, int gl, unsigned gmask,
                                          const float (&v)[CPL * 4], const float (&own)[CPL * 4],
                                          const float (&acc_a)[CPL * 4], const float (&acc_b)[CPL * 4]) {
    float *xo = a.xbar_out + row * (int64_t)a.stride;
    if (a.mode == 0) {
        // xbar_k,i = a_k (sum_j c_ij s_i - sum_j c_ij s_j)
        const float csum = acc_b[0];
#pragma unroll
        for (int c = 0; c < CPL; ++c) {
            const int q = gl + c * LPR;
            if (q < a.nchunks) {
#pragma unroll
                for (int e4 = 0; e4 < 4; ++e4) {
                    const int r = q * 4 + e4;
                    xo[r] = (r < a.R ? __ldg(a.a_k + r) : 0.f) * (csum * own[c * 4 + e4] - acc_a[c * 4 + e4]);
                }
            }
        }
        return;
    }
    const float dinv = __ldg(a.Dinv + row);
    const float om = a.omega, om1 = 1.f - a.omega;
    float cdot = 0.f;
#pragma unroll
    for (int c = 0; c < CPL; ++c) {
        const int q = gl + c * LPR;
        if (q < a.nchunks) {
#pragma unroll
            for (int e4 = 0; e4 < 4; ++e4) {
                const int r = q * 4 + e4;
                xo[r] = fmaf(om1, own[c * 4 + e4], om * acc_a[c * 4 + e4]);
                cdot = fmaf(v[c * 4 + e4], dinv * acc_b[c * 4 + e4], cdot);
            }
        }
    }
#pragma unroll
    for (int off = 1; off < LPR; off <<= 1) cdot += __shfl_xor_sync(gmask, cdot, off);
    if (gl == 0) a.C[row] += (double)cdot;
}

// own values of row i: mode 0 -> s_k,i ; mode 1 -> ybar_t,i (v = ybar * a_{t-1})
template <int LPR, int CPL>
__device__ __forceinline__ void bw_own(const BwArgs &a, int64_t row, int gl, float (&own)[CPL * 4], float (&v)[CPL * 4]) {
#pragma unroll
    for (int c = 0; c < CPL; ++c) {
        const int q = gl + c * LPR;
        if (q < a.nchunks) {
            ld4<CPL>(a.mode == 0 ? a.Sk : a.Ybar, row, a.stride, q, own + c * 4);
#pragma unroll
            for (int e4 = 0; e4 < 4; ++e4)
                v[c * 4 + e4] = a.mode == 1 ? own[c * 4 + e4] * (a.a_prev ? __ldg(a.a_prev + q * 4 + e4) : 1.f) : 0.f;
        } else {
#pragma unroll
            for (int e4 = 0; e4 < 4; ++e4) { own[c * 4 + e4] = 0.f; v[c * 4 + e4] = 0.f; }
        }
    }
}

#ifndef AD_BW_MINB
#define AD_BW_MINB 3          // CTAs per SM (measured: 3 with 8 neighbours in flight beat 4-6 with 2 or 4)
#endif
template <int LPR, int CPL>
__global__ void __launch_bounds__(256, AD_BW_MINB) k_bw(BwArgs a) {
    constexpr int E = CPL * 4, G = 32 / LPR;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
    const int grp = lane / LPR, gl = lane % LPR;
    const unsigned gmask = LPR == 32 ? 0xffffffffu : (((1u << LPR) - 1u) << (grp * LPR));
    const int64_t W = (int64_t)gridDim.x * nwarps;
    for (int64_t task = (int64_t)blockIdx.x * nwarps + warp; task < a.n_tasks; task += W) {
        float acc_a[E], acc_b[E], own[E], v[E];
#pragma unroll
        for (int e = 0; e < E; ++e) { acc_a[e] = 0.f; acc_b[e] = 0.f; }
        if (task < a.n_big) {
            const int64_t row = a.big_row[task];
            const int32_t c = a.big_chunk[task];
            const int64_t rb = a.rp[row], re = a.rp[row + 1];
            const int64_t p0 = rb + (int64_t)c * kChunk, p1 = min(re, p0 + kChunk);
            bw_own<LPR, CPL>(a, row, gl, own, v);
            bw_gather<LPR, CPL>(a, row, p0, p1, grp, G, gl, gmask, v, acc_a, acc_b);
            reduce_groups<LPR, E>(acc_a);
            reduce_groups<LPR, E>(acc_b);
            float *part = a.part + task * (int64_t)2 * a.stride;
            if (grp == 0) {
#pragma unroll
                for (int cc = 0; cc < CPL; ++cc) {
                    const int q = gl + cc * LPR;
                    if (q < a.nchunks) {
#pragma unroll
                        for (int e4 = 0; e4 < 4; ++e4) {
                            __stcg(part + q * 4 + e4, acc_a[cc * 4 + e4]);
                            __stcg(part + a.stride + q * 4 + e4, acc_b[cc * 4 + e4]);
                        }
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
                    float sa[E], sb[E];
#pragma unroll
                    for (int e = 0; e < E; ++e) { sa[e] = 0.f; sb[e] = 0.f; }
                    for (int32_t k2 = 0; k2 < nchunk; ++k2) {
                        const float *pp = a.part + (t0 + k2) * (int64_t)2 * a.stride;
#pragma unroll
                        for (int cc = 0; cc < CPL; ++cc) {
                            const int q = gl + cc * LPR;
                            if (q < a.nchunks) {
#pragma unroll
                                for (int e4 = 0; e4 < 4; ++e4) {
                                    sa[cc * 4 + e4] += __ldcg(pp + q * 4 + e4);
                                    sb[cc * 4 + e4] += __ldcg(pp + a.stride + q * 4 + e4);
                                }
                            }
                        }
                    }
                    bw_finish<LPR, CPL>(a, row, gl, gmask, v, own, sa, sb);
                }
                if (lane == 0) a.big_counter[t0] = 0u;
            }
        } else if (task < a.n_big + a.n_medium) {
            const int64_t row = a.medium_row[task - a.n_big];
            bw_own<LPR, CPL>(a, row, gl, own, v);
            bw_gather<LPR, CPL>(a, row, a.rp[row], a.rp[row + 1], grp, G, gl, gmask, v, acc_a, acc_b);
            reduce_groups<LPR, E>(acc_a);
            reduce_groups<LPR, E>(acc_b);
            if (grp == 0) bw_finish<LPR, CPL>(a, row, gl, gmask, v, own, acc_a, acc_b);
        } else {
            const int64_t si = (task - a.n_big - a.n_medium) * G + grp;
            if (si < a.n_small_rows) {
                const int64_t row = a.small_row[si];
                bw_own<LPR, CPL>(a, row, gl, own, v);
                bw_gather<LPR, CPL>(a, row, a.rp[row], a.rp[row + 1], 0, 1, gl, gmask, v, acc_a, acc_b);
                bw_finish<LPR, CPL>(a, row, gl, gmask, v, own, acc_a, acc_b);
            }
        }
    }
}

// per-block partial sums of A = sum xbar (x - 1/2) and B = sum xbar (x + 1/2),
// x = a (s - lo) - 1/2, and the lowest-index argmin / argmax of each vector
// of the stored iterate (active rows).  Products in FP32 (FP64 runs on a very narrow pipe on
// this part), each thread's running sums compensated (Kahan), the threads'
// sums combined in FP64.  B = A + sum xbar.
constexpr int kRedBlocks = 1216;      // 8 per SM: the per-thread sums are latency bound
__device__ __forceinline__ void kahan_add(float &sum, float &comp, float x) {
    const float y = x - comp;
    const float t = sum + y;
    comp = (t - sum) - y;
    sum = t;
}

__global__ void k_bw_partial(const float *xbar, const float *S, const int64_t *rp, int64_t n, int32_t stride, int32_t R,
                             const uint32_t *mn, const uint32_t *mx, const float *a_t, double *partA, double *partB,
                             unsigned long long *amin, unsigned long long *amax) {
    __shared__ double sA[256], sB[256];
    // thread layout: r = threadIdx.x % R, rows strided over the block's R-wide slices
    const int Rp = R;
    const int lanes_per = blockDim.x / Rp > 0 ? blockDim.x / Rp : 1;
    const int r = threadIdx.x % Rp;
    const int sub = threadIdx.x / Rp;
    float accA = 0.f, cA = 0.f, accX = 0.f, cX = 0.f;
    if (sub < lanes_per && threadIdx.x < lanes_per * Rp) {
        const float lo = ord2f(mn[r]), hi = ord2f(mx[r]);
        const float ar = a_t[r];
        for (int64_t i = (int64_t)blockIdx.x * lanes_per + sub; i < n; i += (int64_t)gridDim.x * lanes_per) {
            if (rp[i + 1] == rp[i]) continue;
            const float xb = xbar[i * stride + r];
            const float sv = S[i * stride + r];
            // the lowest-index argmin / argmax of vector r (the rescale's sub-gradient points)
            if (sv == lo) atomicMin(amin + r, (unsigned long long)i);
            if (sv == hi) atomicMin(amax + r, (unsigned long long)i);
            const float xv = ar * (sv - lo) - 0.5f;
            kahan_add(accA, cA, xb * (xv - 0.5f));
            kahan_add(accX, cX, xb);
        }
    }
    sA[threadIdx.x] = (double)accA - (double)cA;
    sB[threadIdx.x] = (double)accX - (double)cX;
    __syncthreads();
    if (threadIdx.x < Rp) {
        double tA = 0.0, tX = 0.0;
        for (int s2 = 0; s2 < lanes_per; ++s2) { tA += sA[s2 * Rp + threadIdx.x]; tX += sB[s2 * Rp + threadIdx.x]; }
        partA[(int64_t)blockIdx.x * Rp + threadIdx.x] = tA;
        partB[(int64_t)blockIdx.x * Rp + threadIdx.x] = tA + tX;
    }
}

// one warp per vector r: the lanes sum every 32nd block's partial, then a butterfly
__global__ void k_bw_reduce(const double *partA, const double *partB, int nblocks, int32_t R, double *A, double *B) {
    const int lane = threadIdx.x & 31;
    for (int r = threadIdx.x >> 5; r < R; r += blockDim.x >> 5) {
        double tA = 0.0, tB = 0.0;
        for (int b = lane; b < nblocks; b += 32) {
            tA += partA[(int64_t)b * R + r];
            tB += partB[(int64_t)b * R + r];
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            tA += __shfl_xor_sync(0xffffffffu, tA, o);
            tB += __shfl_xor_sync(0xffffffffu, tB, o);
        }
        if (lane == 0) {
            A[r] = tA;
            B[r] = tB;
        }
    }
}

// ybar = a xbar (+ a A at the argmin, - a B at the argmax); U = D^-1 ybar, written
// with a copy of s_{t-1} into the rows of Z (the adjoint gather reads both).
// a * xbar in FP32 is the correctly rounded product, i.e. what FP64 then
// rounding gives; FP64 only at the two corrected entries of each vector.
__global__ void k_bw_ybar(const float *xbar, const int64_t *rp, const float *Dinv, int64_t n, int32_t sshift, int32_t R,
                          const float *a_t, const double *A, const double *B, const unsigned long long *amin,
                          const unsigned long long *amax, float *ybar, const float *S, float *Z) {
    const int64_t total = n << sshift;
    const int rmask = (1 << sshift) - 1;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = t >> sshift;
        const int r = (int)(t & rmask);
        float yb = 0.f;
        if (r < R && rp[i + 1] > rp[i]) {
            const float ar = __ldg(a_t + r);
            if (ar > 0.f) {
                const bool lo_i = (unsigned long long)i == amin[r], hi_i = (unsigned long long)i == amax[r];
                if (lo_i || hi_i) {
                    double v = (double)ar * xbar[t];
                    if (lo_i) v += (double)ar * A[r];
                    if (hi_i) v -= (double)ar * B[r];
                    yb = (float)v;
                } else {
                    yb = ar * xbar[t];
                }
            }
        }
        ybar[t] = yb;
        const int64_t z = (i << (sshift + 1)) + r;   // U and s_{t-1} side by side, twice the pitch
        Z[z] = yb * Dinv[i];
        Z[z + (1 << sshift)] = S[t];
    }
}

__global__ void k_scale_from_mm(const uint32_t *mn, const uint32_t *mx, int32_t stride, float *a) {
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= stride) return;
    const float lo = ord2f(mn[r]), hi = ord2f(mx[r]);   // the forward sweeps' scale, bit for bit
    a[r] = hi > lo ? 1.f / (hi - lo) : 0.f;
}

// dL/dw_e from the per-entry and per-row accumulators of both directions of e
__global__ void k_edge_grad(const int64_t *rp, const int32_t *col, const int64_t *upos, const int64_t *eoff,
                            const int64_t *mirror, const int32_t *erow, const double *D, int64_t nnz, const double *G,
                            const double *C, double omega, float *wbar) {
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < nnz; p += (int64_t)gridDim.x * blockDim.x) {
        const int32_t i = erow[p], j = col[p];
        if (j <= i) continue;
        const int64_t q = mirror[p];
        const int64_t e = eoff[i] + (p - upos[i]);
        const double gi = omega * (G[p] - C[i]) / D[i];
        const double gj = q >= 0 ? omega * (G[q] - C[j]) / D[j] : 0.0;
        wbar[e] = (float)(gi + gj);
    }
}

template <int LPR, int CPL>
static ad_status launch_bw(ad_graph_t g, const BwArgs &a) {
    int per_sm = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_bw<LPR, CPL>, 256, 0);
    int64_t blocks = (int64_t)(per_sm > 0 ? per_sm : 1) * g->num_sms;
    const int64_t need = (a.n_tasks + 7) / 8;
    if (blocks > need) blocks = need > 0 ? need : 1;
    AD_LAUNCH((k_bw<LPR, CPL>), (int)blocks, 256, 0, g->stream, a);
    return AD_OK;
}

static ad_status dispatch_bw(ad_graph_t g, int lpr, int cpl, const BwArgs &a) {
    switch (lpr * 100 + cpl) {
        case 101: return launch_bw<1, 1>(g, a);
        case 201: return launch_bw<2, 1>(g, a);
        case 401: return launch_bw<4, 1>(g, a);
        case 801: return launch_bw<8, 1>(g, a);
        case 1601: return launch_bw<16, 1>(g, a);
        case 3201: return launch_bw<32, 1>(g, a);
        case 3202: return launch_bw<32, 2>(g, a);
        default: return fail(AD_ERR_INVALID_ARG, "unsupported R for the reverse mode");
    }
}

static void fill_bw_plan(BwArgs &a, const RowPlan &p) {
    a.big_row = p.big_row; a.big_chunk = p.big_chunk; a.medium_row = p.medium_row; a.small_row = p.small_row;
    a.big_counter = p.big_counter;
    a.n_big = p.n_big; a.n_medium = p.n_medium; a.n_small_rows = p.n_small_rows;
    a.n_tasks = p.tasks();
}

ad_status backward(ad_graph_t g, const float *rhobar_dev, float *wbar_dev) {
    auto *sv = g->saved;
    const int32_t R = sv->R, k = sv->k, c = sv->c, stride = sv->stride;
    const int64_t n = g->n, nnz = g->nnz;
    AD_TRY(ensure_mirror(g));
    RowPlan *plan = nullptr;
    AD_TRY(get_row_plan(g, 32 / sv->lpr, false, &plan));
    // buffers
    std::vector<float *> seg(c + 1, nullptr);
    if (!sv->all)   // (with every iterate kept, seg points into the kept iterates)
        for (int u = 1; u <= c; ++u) AD_TRY(dalloc_t(g, (n + 1) * stride, &seg[u]));
    float *xbar = nullptr, *xbar2 = nullptr, *ybar = nullptr, *part = nullptr;
    float *a_t = nullptr, *a_p = nullptr, *a_k = nullptr;   // scales of sweep t, t - 1 and k
    double *G = nullptr, *C = nullptr, *partA = nullptr, *partB = nullptr, *A = nullptr, *B = nullptr;
    unsigned long long *amin = nullptr, *amax = nullptr;
    uint32_t *scratch_mm = nullptr;
    AD_TRY(dalloc_t(g, (n + 1) * stride, &xbar));
    AD_TRY(dalloc_t(g, (n + 1) * stride, &xbar2));
    AD_TRY(dalloc_t(g, (n + 1) * stride, &ybar));
    // rows [U_j | s_{t-1,j}] side by side, so that the adjoint gather fetches one
    // contiguous 2 * stride row per entry (measured at R-MAT 22: 2% faster backward)
    float *Z = nullptr;
    AD_TRY(dalloc_t(g, (n + 1) * 2 * (size_t)stride, &Z));
    AD_TRY(dalloc_t(g, (size_t)std::max<int64_t>(plan->n_big, 1) * 2 * stride, &part));
    AD_TRY(dalloc_t(g, nnz + 1, &G));
    AD_TRY(dalloc_t(g, n + 1, &C));
    AD_TRY(dalloc_t(g, (size_t)kRedBlocks * stride, &partA));
    AD_TRY(dalloc_t(g, (size_t)kRedBlocks * stride, &partB));
    AD_TRY(dalloc_t(g, stride, &A));
    AD_TRY(dalloc_t(g, stride, &B));
    AD_TRY(dalloc_t(g, stride, &amin));
    AD_TRY(dalloc_t(g, stride, &amax));
    AD_TRY(dalloc_t(g, stride, &a_t));
    AD_TRY(dalloc_t(g, stride, &a_p));
    AD_TRY(dalloc_t(g, stride, &a_k));
    AD_TRY(dalloc_t(g, 2 * stride, &scratch_mm));
    AD_CUDA_TRY(cudaMemsetAsync(G, 0, (nnz + 1) * sizeof(double), g->stream));
    AD_CUDA_TRY(cudaMemsetAsync(C, 0, (n + 1) * sizeof(double), g->stream));
    const uint32_t *mm_min = sv->mm, *mm_max = sv->mm + (size_t)k * stride;
    int sshift = 0;   // stride = 1 << sshift (a power of two, at least 4)
    while ((1 << sshift) < stride) ++sshift;
    auto slot_min = [&](int t) { return mm_min + (size_t)(t - 1) * stride; };   // min/max of s_t, t >= 1
    auto slot_max = [&](int t) { return mm_max + (size_t)(t - 1) * stride; };

    BwArgs a;
    memset(&a, 0, sizeof(a));
    a.rp = g->rp; a.col = g->col; a.w = g->w; a.Dinv = g->Dinv; a.eid = g->eid;
    a.stride = stride; a.nchunks = sv->nchunks; a.R = R; a.omega = (float)sv->omega;
    a.rho = sv->rho; a.rhobar = rhobar_dev;
    a.G = G; a.C = C; a.part = part;
    fill_bw_plan(a, *plan);

    const int nseg = k > 0 ? (k + c - 1) / c : 0;
    if (k == 0) {
        // rho of the raw init: xbar_0 = sum c_ij (x_i - x_j); weights do not enter
        AD_CUDA_TRY(cudaMemsetAsync(wbar_dev, 0, g->m * sizeof(float), g->stream));
        return AD_OK;
    }
    bool have_xbar = false;
    for (int j = nseg - 1; j >= 0; --j) {
        const int t0 = j * c, len = std::min(c, k - t0);
        seg[0] = static_cast<float *>(sv->ckpt[j]);
        for (int u = 1; u <= len; ++u) {
            const int t = t0 + u;   // produce s_t from s_{t-1}
            if (sv->all) {          // kept by the forward: the same values the sweep would give
                seg[u] = static_cast<float *>(sv->ckpt[t]);
                continue;
            }
            AD_CUDA_TRY(cudaMemsetAsync(scratch_mm, 0xff, stride * sizeof(uint32_t), g->stream));
            AD_CUDA_TRY(cudaMemsetAsync(scratch_mm + stride, 0, stride * sizeof(uint32_t), g->stream));
            AD_TRY(sweep_step(g, AD_STORAGE_FP32, R, sv->omega, seg[u - 1], seg[u], t >= 2 ? slot_min(t - 1) : nullptr,
                              t >= 2 ? slot_max(t - 1) : nullptr, scratch_mm, scratch_mm + stride));
        }
        if (!have_xbar) {   // distance backward on s_k
            AD_LAUNCH(k_scale_from_mm, 1, 256, 0, g->stream, slot_min(k), slot_max(k), stride, a_k);
            a.a_k = a_k;
            a.mode = 0;
            a.Sk = seg[len];
            a.xbar_out = xbar;
            AD_TRY(dispatch_bw(g, sv->lpr, sv->cpl, a));
            have_xbar = true;
        }
        for (int u = len; u >= 1; --u) {
            const int t = t0 + u;
            const float *St = seg[u], *Sp = seg[u - 1];
            // rescale adjoint of sweep t
            AD_LAUNCH(k_scale_from_mm, 1, 256, 0, g->stream, slot_min(t), slot_max(t), stride, a_t);
            AD_CUDA_TRY(cudaMemsetAsync(amin, 0xff, stride * sizeof(unsigned long long), g->stream));
            AD_CUDA_TRY(cudaMemsetAsync(amax, 0xff, stride * sizeof(unsigned long long), g->stream));
            AD_LAUNCH(k_bw_partial, kRedBlocks, 256, 0, g->stream, xbar, St, g->rp, n, stride, R, slot_min(t),
                      slot_max(t), a_t, partA, partB, amin, amax);
            AD_LAUNCH(k_bw_reduce, 1, 1024, 0, g->stream, partA, partB, kRedBlocks, R, A, B);
            AD_LAUNCH(k_bw_ybar, g->num_sms * 16, 256, 0, g->stream, xbar, g->rp, g->Dinv, n, sshift, R, a_t, A, B, amin,
                      amax, ybar, Sp, Z);
            // sweep adjoint + weight terms
            if (t >= 2) {
                AD_LAUNCH(k_scale_from_mm, 1, 256, 0, g->stream, slot_min(t - 1), slot_max(t - 1), stride, a_p);
                a.a_prev = a_p;
            } else {
                a.a_prev = nullptr;
            }
            a.mode = 1;
            a.U = Z;
            a.Sprev = Z + stride;
            a.gpitch = 2 * stride;
            a.Ybar = ybar;
            a.xbar_out = xbar2;
            AD_TRY(dispatch_bw(g, sv->lpr, sv->cpl, a));
            std::swap(xbar, xbar2);
        }
    }
    AD_LAUNCH(k_edge_grad, g->num_sms * 16, 256, 0, g->stream, g->rp, g->col, g->upos, g->eoff, g->mirror, g->erow, g->D,
              nnz, G, C, sv->omega, wbar_dev);
    AD_CUDA_TRY(cudaStreamSynchronize(g->stream));
    if (!sv->all)
        for (int u = 1; u <= c; ++u) dfree(g, seg[u]);
    for (void *p : {(void *)xbar, (void *)xbar2, (void *)ybar, (void *)Z, (void *)part, (void *)G, (void *)C,
                    (void *)partA, (void *)partB, (void *)A, (void *)B, (void *)amin, (void *)amax, (void *)a_t, (void *)a_p, (void *)a_k,
                    (void *)scratch_mm})
        dfree(g, p);
    return AD_OK;
}

}  // namespace ad

extern "C" ad_status ad_algebraic_distance_backward(ad_graph_t g, const float *rho_bar, float *w_bar) {
    using namespace ad;
    if (!g) return fail(AD_ERR_INVALID_ARG, "NULL graph");
    if (!g->saved) return fail(AD_ERR_STATE, "no kept state: run ad_algebraic_distance with AD_DIST_KEEP_STATE first");
    if (g->m > 0 && (!rho_bar || !w_bar)) return fail(AD_ERR_INVALID_ARG, "NULL rho_bar or w_bar");
    float *rb = nullptr, *wb = nullptr;
    AD_TRY(dalloc_t(g, g->m + 1, &rb));
    AD_TRY(dalloc_t(g, g->m + 1, &wb));
    AD_TRY(copy_in(g, rb, rho_bar, g->m * sizeof(float)));
    ad_status st = backward(g, rb, wb);
    if (st == AD_OK) st = copy_out(g, w_bar, wb, g->m * sizeof(float));
    if (st == AD_OK) st = cudaStreamSynchronize(g->stream) == cudaSuccess ? AD_OK : fail(AD_ERR_CUDA, "sync");
    dfree(g, rb);
    dfree(g, wb);
    return st;
}
