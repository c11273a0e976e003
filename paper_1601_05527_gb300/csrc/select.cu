// select.cu -- ranking and sampling of edges (Sec. 4, Alg. 2) on sm_103a.
//
// Keys.  A score s >= 0 is ranked through its FP32 bit pattern, which orders
// non-negative floats like their values (-0 is folded onto +0).  "local"
// (keep delta-strong edges) ranks ascending, "global" (keep delta-weak) ranks
// descending, i.e. ascending in the complemented key.  Ties are broken by
// ascending edge id in both modes.
//
// Whole-graph scope: radix select of the K-th key per graph (three digit
// passes of 11/11/10 bits with per-tile shared-memory histograms), then an
// ordered compaction of the keys equal to the threshold so that exactly K
// edges are kept.
//
// Per-node scope (Alg. 2): every CSR entry is ranked inside its row by
// (key, position) -- positions inside a row follow edge ids, because the ids
// enumerate (min, max) pairs row-major.  Node i keeps its entries of rank
// < T(d_i, e).  The exponent e is searched on the 2^-40 grid by passes that
// count the kept set at 15 candidate exponents at once; the integer tables
// T(d, e) come from the host (FP64 pow), so both this library and an FP64
// reference take identical integer decisions.
#include "ad_internal.cuh"

#include <algorithm>
#include <cmath>
#include <cstring>
#include <mutex>

namespace ad {

__device__ __forceinline__ uint32_t score_key(float s, int desc) {
    uint32_t b = __float_as_uint(s);
    if (s == 0.f) b = 0u;   // -0 == +0
    return desc ? ~b : b;
}

constexpr int kTileItems = 16;
constexpr int kTileThreads = 256;
constexpr int64_t kTile = (int64_t)kTileItems * kTileThreads;

struct SelState {
    uint32_t prefix;
    uint32_t pad;
    int64_t k_rem;   // rank (1-based) still to locate inside the current bucket
    int64_t K;
    int64_t m;
};

struct Tiles {
    int64_t n = 0;
    int32_t *graph = nullptr;
    int64_t *start = nullptr, *end = nullptr;
    int32_t *first_tile = nullptr;   // [G] first tile of each graph
    std::vector<int32_t> first_h;
};

static ad_status make_tiles(ad_graph_t g, Tiles &t) {
    std::vector<int32_t> tg;
    std::vector<int64_t> ts, te;
    t.first_h.assign(g->G + 1, 0);
    for (int32_t k = 0; k < g->G; ++k) {
        t.first_h[k] = (int32_t)tg.size();
        for (int64_t s = g->eoff_h[k]; s < g->eoff_h[k + 1]; s += kTile) {
            tg.push_back(k);
            ts.push_back(s);
            te.push_back(std::min<int64_t>(s + kTile, g->eoff_h[k + 1]));
        }
    }
    t.first_h[g->G] = (int32_t)tg.size();
    t.n = (int64_t)tg.size();
    if (t.n == 0) return AD_OK;
    AD_TRY(dalloc_t(g, t.n, &t.graph));
    AD_TRY(dalloc_t(g, t.n, &t.start));
    AD_TRY(dalloc_t(g, t.n, &t.end));
    AD_TRY(dalloc_t(g, g->G + 1, &t.first_tile));
    AD_TRY(copy_in(g, t.graph, tg.data(), t.n * sizeof(int32_t)));
    AD_TRY(copy_in(g, t.start, ts.data(), t.n * sizeof(int64_t)));
    AD_TRY(copy_in(g, t.end, te.data(), t.n * sizeof(int64_t)));
    AD_TRY(copy_in(g, t.first_tile, t.first_h.data(), (g->G + 1) * sizeof(int32_t)));
    return AD_OK;
}
static void free_tiles(ad_graph_t g, Tiles &t) {
    if (t.graph) dfree(g, t.graph);
    if (t.start) dfree(g, t.start);
    if (t.end) dfree(g, t.end);
    if (t.first_tile) dfree(g, t.first_tile);
    t = Tiles();
}

// ----------------------------------------------------------------------------
// Score validation: every score finite and >= 0.
// ----------------------------------------------------------------------------
__global__ void k_check_scores(const float *s, int64_t m, unsigned long long *bad) {
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < m; e += (int64_t)gridDim.x * blockDim.x) {
        const float x = s[e];
        if (!(x >= 0.f) || !isfinite(x)) atomicMin(bad, (unsigned long long)e);
    }
}

// ----------------------------------------------------------------------------
// Whole-graph radix select
// ----------------------------------------------------------------------------
__global__ void k_sel_hist(const float *score, int desc, const int32_t *tg, const int64_t *ts, const int64_t *te,
                           const SelState *st, int shift, int bits, uint32_t hi_mask, uint32_t *hist) {
    __shared__ uint32_t h[2048];
    for (int b = threadIdx.x; b < (1 << bits); b += blockDim.x) h[b] = 0;
    __syncthreads();
    const int gph = tg[blockIdx.x];
    const SelState s = st[gph];
    if (s.k_rem > 0) {
        const uint32_t dmask = (1u << bits) - 1u;
        for (int64_t e = ts[blockIdx.x] + threadIdx.x; e < te[blockIdx.x]; e += blockDim.x) {
            const uint32_t k = score_key(score[e], desc);
            if ((k & hi_mask) == s.prefix) atomicAdd(&h[(k >> shift) & dmask], 1u);
        }
    }
    __syncthreads();
    for (int b = threadIdx.x; b < (1 << bits); b += blockDim.x)
        if (h[b]) atomicAdd(hist + (size_t)gph * 2048 + b, h[b]);
}

// one CTA per graph: locate the bucket holding rank k_rem
__global__ void k_sel_find(uint32_t *hist, SelState *st, int shift, int bits) {
    __shared__ int64_t cnt[2048];
    __shared__ int64_t sh[32];
    const int gph = blockIdx.x;
    SelState s = st[gph];
    const int nb = 1 << bits;
    // each thread owns nb / blockDim consecutive bins (blockDim = 256 -> 8 or 4)
    const int per = nb / blockDim.x;
    int64_t local = 0;
    for (int k = 0; k < per; ++k) {
        const int b = threadIdx.x * per + k;
        cnt[b] = hist[(size_t)gph * 2048 + b];
        local += cnt[b];
    }
    // exclusive scan of the per-thread sums
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    int64_t x = local;
    for (int o = 1; o < 32; o <<= 1) {
        int64_t y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) sh[warp] = x;
    __syncthreads();
    if (warp == 0) {
        int64_t v = lane < nw ? sh[lane] : 0;
        for (int o = 1; o < 32; o <<= 1) {
            int64_t y = __shfl_up_sync(0xffffffffu, v, o);
            if (lane >= o) v += y;
        }
        if (lane < nw) sh[lane] = v;
    }
    __syncthreads();
    int64_t before = (warp > 0 ? sh[warp - 1] : 0) + x - local;
    if (s.k_rem > 0) {
        for (int k = 0; k < per; ++k) {
            const int b = threadIdx.x * per + k;
            if (before < s.k_rem && s.k_rem <= before + cnt[b]) {
                s.prefix |= ((uint32_t)b) << shift;
                s.k_rem -= before;
                st[gph] = s;
            }
            before += cnt[b];
        }
    }
}

__global__ void k_sel_ties(const float *score, int desc, const int32_t *tg, const int64_t *ts, const int64_t *te,
                           const SelState *st, int64_t *tile_ties) {
    __shared__ int64_t sh[32];
    const int gph = tg[blockIdx.x];
    const SelState s = st[gph];
    int64_t c = 0;
    if (s.k_rem > 0)
        for (int64_t e = ts[blockIdx.x] + threadIdx.x; e < te[blockIdx.x]; e += blockDim.x)
            c += (score_key(score[e], desc) == s.prefix) ? 1 : 0;
    for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = c;
    __syncthreads();
    if (threadIdx.x == 0) {
        int64_t t = 0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += sh[w];
        tile_ties[blockIdx.x] = t;
    }
}

// keep = key < t, or key == t among the first k_rem ties (edge-id order)
__global__ void k_sel_write(const float *score, int desc, const int32_t *tg, const int64_t *ts, const int64_t *te,
                            const SelState *st, const int64_t *tie_off, const int32_t *first_tile, uint8_t *keep) {
    __shared__ int64_t sh[32];
    const int gph = tg[blockIdx.x];
    const SelState s = st[gph];
    const int64_t e0 = ts[blockIdx.x] + (int64_t)threadIdx.x * kTileItems, e1 = te[blockIdx.x];
    uint32_t k[kTileItems];
    int64_t my = 0;
#pragma unroll
    for (int i = 0; i < kTileItems; ++i) {
        k[i] = (e0 + i < e1) ? score_key(score[e0 + i], desc) : 0xffffffffu;
        my += (e0 + i < e1 && s.k_rem > 0 && k[i] == s.prefix) ? 1 : 0;
    }
    // block exclusive scan of tie counts (threads own consecutive edges)
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    int64_t x = my;
    for (int o = 1; o < 32; o <<= 1) {
        int64_t y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) sh[warp] = x;
    __syncthreads();
    if (warp == 0) {
        int64_t v = lane < nw ? sh[lane] : 0;
        for (int o = 1; o < 32; o <<= 1) {
            int64_t y = __shfl_up_sync(0xffffffffu, v, o);
            if (lane >= o) v += y;
        }
        if (lane < nw) sh[lane] = v;
    }
    __syncthreads();
    int64_t rank = tie_off[blockIdx.x] - tie_off[first_tile[gph]] + (warp > 0 ? sh[warp - 1] : 0) + x - my;
#pragma unroll
    for (int i = 0; i < kTileItems; ++i) {
        if (e0 + i >= e1) break;
        uint8_t kp = 0;
        if (s.K >= s.m) kp = 1;
        else if (s.K > 0) {
            if (k[i] < s.prefix) kp = 1;
            else if (k[i] == s.prefix) { kp = rank < s.k_rem ? 1 : 0; ++rank; }
        }
        keep[e0 + i] = kp;
    }
}

// ----------------------------------------------------------------------------
// Per-node ranks
// ----------------------------------------------------------------------------
__global__ void k_entry_keys(const int64_t *eid, int64_t nnz, const float *score, int desc, uint32_t *ekey) {
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < nnz; p += (int64_t)gridDim.x * blockDim.x)
        ekey[p] = score_key(score[eid[p]], desc);
}

// The rank r of entry p of row i goes to its edge's info: (rank at the lower
// endpoint, rank at the upper endpoint, degree class of each endpoint).
__device__ __forceinline__ void put_rank(int4 *info, const int64_t *eid, const int32_t *col, const int32_t *dc,
                                         int64_t i, int64_t p, uint32_t r) {
    int *f = reinterpret_cast<int *>(info + eid[p]);
    if (col[p] > i) { f[0] = (int)r; f[2] = dc[i]; }
    else { f[1] = (int)r; f[3] = dc[i]; }
}

// rows of degree <= 32: one warp each, rank by pairwise comparison
__global__ void k_rank_small(const int64_t *rp, const int32_t *col, const int64_t *eid, const int32_t *dc, int64_t n,
                             const uint32_t *ekey, int4 *info) {
    const int lane = threadIdx.x & 31;
    const int64_t W = (int64_t)gridDim.x * (blockDim.x >> 5);
    for (int64_t i = blockIdx.x * (int64_t)(blockDim.x >> 5) + (threadIdx.x >> 5); i < n; i += W) {
        const int64_t p0 = rp[i];
        const int d = (int)(rp[i + 1] - p0);
        if (d == 0 || d > 32) continue;
        const uint32_t k = lane < d ? ekey[p0 + lane] : 0xffffffffu;
        uint32_t r = 0;
        for (int l = 0; l < d; ++l) {
            const uint32_t o = __shfl_sync(0xffffffffu, k, l);
            r += (o < k || (o == k && l < lane)) ? 1u : 0u;
        }
        if (lane < d) put_rank(info, eid, col, dc, i, p0 + lane, r);
    }
}

constexpr int kSortCap = 2048;   // entries sorted by one CTA in shared memory

// Bitonic sort of up to kSortCap 64-bit keys (key << 32 | position) in smem.
__device__ void block_bitonic(unsigned long long *a, int len_pow2) {
    for (int size = 2; size <= len_pow2; size <<= 1) {
        for (int stride = size >> 1; stride > 0; stride >>= 1) {
            for (int t = threadIdx.x; t < len_pow2 / 2; t += blockDim.x) {
                const int lo = 2 * t - (t & (stride - 1));
                const int hi = lo + stride;
                const bool up = ((lo & size) == 0);
                const unsigned long long x = a[lo], y = a[hi];
                if ((x > y) == up) { a[lo] = y; a[hi] = x; }
            }
            __syncthreads();
        }
    }
}

// rows of degree in (32, kSortCap]: a CTA per row; up to 128 entries rank by
// counting, longer rows by a bitonic sort of (key, position) in shared memory
__global__ void k_rank_mid(const int64_t *rp, const int32_t *col, const int64_t *eid, const int32_t *dc,
                           const int32_t *rows, const uint32_t *ekey, int4 *info) {
    __shared__ unsigned long long a[kSortCap];
    const int64_t row = rows[blockIdx.x];
    const int64_t p0 = rp[row];
    const int d = (int)(rp[row + 1] - p0);
    if (d <= 128) {
        for (int t = threadIdx.x; t < d; t += blockDim.x) a[t] = ((unsigned long long)ekey[p0 + t] << 32) | (unsigned)t;
        __syncthreads();
        for (int t = threadIdx.x; t < d; t += blockDim.x) {
            const unsigned long long k = a[t];
            uint32_t r = 0;
            for (int u = 0; u < d; ++u) r += a[u] < k ? 1u : 0u;
            put_rank(info, eid, col, dc, row, p0 + t, r);
        }
        return;
    }
    int len2 = 1;
    while (len2 < d) len2 <<= 1;
    for (int t = threadIdx.x; t < len2; t += blockDim.x)
        a[t] = t < d ? (((unsigned long long)ekey[p0 + t] << 32) | (unsigned)t) : ~0ull;
    __syncthreads();
    block_bitonic(a, len2);
    for (int t = threadIdx.x; t < d; t += blockDim.x)
        put_rank(info, eid, col, dc, row, p0 + (int64_t)(a[t] & 0xffffffffull), (uint32_t)t);
}

// rows of degree > kSortCap: one CTA per (row, chunk of kSortCap entries) sorts
// the chunk; k_rank_merge then adds the ranks from the other chunks
__global__ void k_rank_chunks(const int64_t *rp, const int32_t *rows, const int32_t *chunk, const uint32_t *ekey,
                              uint32_t *rank, unsigned long long *skey) {
    __shared__ unsigned long long a[kSortCap];
    const int64_t row = rows[blockIdx.x];
    const int c = chunk[blockIdx.x];
    const int64_t p0 = rp[row], d = rp[row + 1] - p0;
    const int64_t c0 = (int64_t)c * kSortCap;
    const int len = (int)std::min<int64_t>(kSortCap, d - c0);
    int len2 = 1;
    while (len2 < len) len2 <<= 1;
    for (int t = threadIdx.x; t < len2; t += blockDim.x)
        a[t] = t < len ? (((unsigned long long)ekey[p0 + c0 + t] << 32) | (unsigned long long)(c0 + t)) : ~0ull;
    __syncthreads();
    block_bitonic(a, len2);
    for (int t = threadIdx.x; t < len; t += blockDim.x) {
        const int64_t pos = (int64_t)(a[t] & 0xffffffffull);
        rank[p0 + pos] = (uint32_t)t;
        skey[p0 + c0 + t] = a[t];
    }
}

// rows of several chunks: add the number of smaller keys in every other chunk
__global__ void k_rank_merge(const int64_t *rp, const int32_t *col, const int64_t *eid, const int32_t *dc,
                             const int32_t *rows, const int32_t *chunk, const uint32_t *ekey,
                             const unsigned long long *skey, const uint32_t *rank, int4 *info) {
    const int64_t row = rows[blockIdx.x];
    const int c = chunk[blockIdx.x];
    const int64_t p0 = rp[row], d = rp[row + 1] - p0;
    const int nch = (int)((d + kSortCap - 1) / kSortCap);
    const int64_t c0 = (int64_t)c * kSortCap;
    const int len = (int)std::min<int64_t>(kSortCap, d - c0);
    for (int t = threadIdx.x; t < len; t += blockDim.x) {
        const unsigned long long key = ((unsigned long long)ekey[p0 + c0 + t] << 32) | (unsigned long long)(c0 + t);
        uint32_t add = 0;
        for (int o = 0; o < nch; ++o) {
            if (o == c) continue;
            const int64_t b = p0 + (int64_t)o * kSortCap;
            int lo = 0, hi = (int)std::min<int64_t>(kSortCap, d - (int64_t)o * kSortCap);
            while (lo < hi) {
                const int mid = (lo + hi) >> 1;
                if (skey[b + mid] < key) lo = mid + 1; else hi = mid;
            }
            add += (uint32_t)lo;
        }
        put_rank(info, eid, col, dc, row, p0 + c0 + t, rank[p0 + c0 + t] + add);
    }
}

// tasks per row: mid rows (32, kSortCap] one, big rows one per chunk
__global__ void k_chunk_count(const int64_t *rp, int64_t n, int64_t *nmid, int64_t *nbig) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t d = rp[i + 1] - rp[i];
        nmid[i] = (d > 32 && d <= kSortCap) ? 1 : 0;
        nbig[i] = d > kSortCap ? (d + kSortCap - 1) / kSortCap : 0;
    }
}
__global__ void k_chunk_expand(const int64_t *nch, const int64_t *first, int64_t n, int32_t *rows, int32_t *chunk) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        for (int64_t c = 0; c < nch[i]; ++c) {
            rows[first[i] + c] = (int32_t)i;
            chunk[first[i] + c] = (int32_t)c;
        }
}

// count the kept set at ncand candidate exponents: T[c][dc] tables per graph
__global__ void k_count_cand(const int4 *info, const int32_t *tg, const int64_t *ts, const int64_t *te,
                             const int32_t *T, int32_t ndc, int ncand, unsigned long long *hist) {
    __shared__ unsigned int h[16];
    if (threadIdx.x < 16) h[threadIdx.x] = 0;
    __syncthreads();
    const int gph = tg[blockIdx.x];
    const int32_t *Tg = T + (size_t)gph * ncand * ndc;
    for (int64_t e = ts[blockIdx.x] + threadIdx.x; e < te[blockIdx.x]; e += blockDim.x) {
        const int4 f = info[e];
        int lo = 0, hi = ncand;   // first candidate at which the edge is kept
        while (lo < hi) {
            const int mid = (lo + hi) >> 1;
            const int32_t *Tm = Tg + (size_t)mid * ndc;
            if (f.x < Tm[f.z] || f.y < Tm[f.w]) hi = mid; else lo = mid + 1;
        }
        atomicAdd(&h[lo], 1u);
    }
    __syncthreads();
    if (threadIdx.x < 16 && h[threadIdx.x]) atomicAdd(hist + (size_t)gph * 16 + threadIdx.x, (unsigned long long)h[threadIdx.x]);
}

__global__ void k_keep_at(const int4 *info, const int32_t *tg, const int64_t *ts, const int64_t *te, const int32_t *T,
                          int32_t ndc, uint8_t *keep, unsigned long long *kept) {
    __shared__ unsigned long long sh[32];
    const int gph = tg[blockIdx.x];
    const int32_t *Tg = T + (size_t)gph * ndc;
    unsigned long long c = 0;
    for (int64_t e = ts[blockIdx.x] + threadIdx.x; e < te[blockIdx.x]; e += blockDim.x) {
        const int4 f = info[e];
        const uint8_t k = (f.x < Tg[f.z] || f.y < Tg[f.w]) ? 1 : 0;
        keep[e] = k;
        c += k;
    }
    for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = c;
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned long long t = 0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += sh[w];
        if (t) atomicAdd(kept + gph, t);
    }
}

// ----------------------------------------------------------------------------
// Host side
// ----------------------------------------------------------------------------
int64_t degree_target(int64_t d, double e) {
    if (d <= 0) return 0;
    double t = std::ceil(std::pow((double)d, e) - 1e-9);
    if (t < 1.0) t = 1.0;
    if (t > (double)d) t = (double)d;
    return (int64_t)t;
}

static int64_t target_count(int64_t m, double fraction) { return (int64_t)std::floor(fraction * (double)m + 0.5); }

ad_status select_whole_graph(ad_graph_t g, const float *score, double fraction, ad_mode mode, uint8_t *keep,
                             int64_t *n_kept) {
    const int desc = mode == AD_MODE_GLOBAL ? 1 : 0;
    Tiles t;
    AD_TRY(make_tiles(g, t));
    if (t.n == 0) { if (n_kept) *n_kept = 0; return AD_OK; }
    std::vector<SelState> sh(g->G);
    int64_t total = 0;
    for (int32_t k = 0; k < g->G; ++k) {
        const int64_t m = g->eoff_h[k + 1] - g->eoff_h[k];
        sh[k].prefix = 0;
        sh[k].pad = 0;
        sh[k].K = target_count(m, fraction);
        sh[k].m = m;
        sh[k].k_rem = (sh[k].K > 0 && sh[k].K < m) ? sh[k].K : 0;   // 0: nothing to locate
        total += sh[k].K;
    }
    SelState *st = nullptr;
    uint32_t *hist = nullptr;
    int64_t *ties = nullptr, *tie_off = nullptr;
    AD_TRY(dalloc_t(g, g->G, &st));
    AD_TRY(dalloc_t(g, (size_t)g->G * 2048 * 3, &hist));
    AD_TRY(dalloc_t(g, t.n + 1, &ties));
    AD_TRY(dalloc_t(g, t.n + 1, &tie_off));
    AD_TRY(copy_in(g, st, sh.data(), sizeof(SelState) * g->G));
    AD_CUDA_TRY(cudaMemsetAsync(hist, 0, sizeof(uint32_t) * (size_t)g->G * 2048 * 3, g->stream));
    const int shifts[3] = {21, 10, 0}, bits[3] = {11, 11, 10};
    const uint32_t hi_masks[3] = {0u, 0xFFE00000u, 0xFFFFFC00u};
    for (int pass = 0; pass < 3; ++pass) {
        uint32_t *hp = hist + (size_t)pass * g->G * 2048;
        AD_LAUNCH(k_sel_hist, (int)t.n, 256, 0, g->stream, score, desc, t.graph, t.start, t.end, st, shifts[pass],
                  bits[pass], hi_masks[pass], hp);
        AD_LAUNCH(k_sel_find, g->G, 256, 0, g->stream, hp, st, shifts[pass], bits[pass]);
    }
    AD_LAUNCH(k_sel_ties, (int)t.n, 256, 0, g->stream, score, desc, t.graph, t.start, t.end, st, ties);
    AD_TRY(exclusive_scan_i64(g, ties, tie_off, t.n, nullptr));
    AD_LAUNCH(k_sel_write, (int)t.n, kTileThreads, 0, g->stream, score, desc, t.graph, t.start, t.end, st, tie_off,
              t.first_tile, keep);
    AD_CUDA_TRY(cudaStreamSynchronize(g->stream));
    dfree(g, st);
    dfree(g, hist);
    dfree(g, ties);
    dfree(g, tie_off);
    free_tiles(g, t);
    if (n_kept) *n_kept = total;
    return AD_OK;
}

// Ranks of every CSR entry, gathered per edge: the info of Alg. 2.
static ad_status per_node_info(ad_graph_t g, const float *score, ad_mode mode, int4 **info_out) {
    AD_TRY(ensure_mirror(g));
    AD_TRY(ensure_degree_classes(g));
    const int desc = mode == AD_MODE_GLOBAL ? 1 : 0;
    const int64_t n = g->n, nnz = g->nnz;
    uint32_t *ekey = nullptr, *rank = nullptr;
    unsigned long long *skey = nullptr;
    int64_t *nmid = nullptr, *nbig = nullptr, *fmid = nullptr, *fbig = nullptr;
    int4 *info = nullptr;
    AD_TRY(dalloc_t(g, g->m + 1, &info));
    AD_TRY(dalloc_t(g, nnz + 1, &ekey));
    const int grid = g->num_sms * 16;
    if (nnz > 0) AD_LAUNCH(k_entry_keys, grid, 256, 0, g->stream, g->eid, nnz, score, desc, ekey);
    const int64_t wblocks = std::min<int64_t>((n + 7) / 8 + 1, (int64_t)g->num_sms * 64);
    AD_LAUNCH(k_rank_small, (int)wblocks, 256, 0, g->stream, g->rp, g->col, g->eid, g->deg_class, n, ekey, info);
    AD_TRY(dalloc_t(g, n + 1, &nmid));
    AD_TRY(dalloc_t(g, n + 1, &nbig));
    AD_TRY(dalloc_t(g, n + 1, &fmid));
    AD_TRY(dalloc_t(g, n + 1, &fbig));
    AD_LAUNCH(k_chunk_count, g->num_sms * 8, 256, 0, g->stream, g->rp, n, nmid, nbig);
    int64_t n_mid = 0, n_big = 0;
    AD_TRY(exclusive_scan_i64(g, nmid, fmid, n, &n_mid));
    AD_TRY(exclusive_scan_i64(g, nbig, fbig, n, &n_big));
    if (n_mid > 0) {
        int32_t *rows = nullptr, *chunk = nullptr;
        AD_TRY(dalloc_t(g, n_mid, &rows));
        AD_TRY(dalloc_t(g, n_mid, &chunk));
        AD_LAUNCH(k_chunk_expand, g->num_sms * 8, 256, 0, g->stream, nmid, fmid, n, rows, chunk);
        AD_LAUNCH(k_rank_mid, (int)n_mid, 256, 0, g->stream, g->rp, g->col, g->eid, g->deg_class, rows, ekey, info);
        AD_CUDA_TRY(cudaStreamSynchronize(g->stream));
        dfree(g, rows);
        dfree(g, chunk);
    }
    if (n_big > 0) {
        int32_t *rows = nullptr, *chunk = nullptr;
        AD_TRY(dalloc_t(g, n_big, &rows));
        AD_TRY(dalloc_t(g, n_big, &chunk));
        AD_TRY(dalloc_t(g, nnz + 1, &skey));
        AD_TRY(dalloc_t(g, nnz + 1, &rank));
        AD_LAUNCH(k_chunk_expand, g->num_sms * 8, 256, 0, g->stream, nbig, fbig, n, rows, chunk);
        AD_LAUNCH(k_rank_chunks, (int)n_big, 512, 0, g->stream, g->rp, rows, chunk, ekey, rank, skey);
        AD_LAUNCH(k_rank_merge, (int)n_big, 256, 0, g->stream, g->rp, g->col, g->eid, g->deg_class, rows, chunk, ekey,
                  skey, rank, info);
        AD_CUDA_TRY(cudaStreamSynchronize(g->stream));
        dfree(g, rows);
        dfree(g, chunk);
        dfree(g, skey);
        dfree(g, rank);
    }
    AD_CUDA_TRY(cudaStreamSynchronize(g->stream));
    dfree(g, ekey);
    dfree(g, nmid);
    dfree(g, nbig);
    dfree(g, fmid);
    dfree(g, fbig);
    *info_out = info;
    return AD_OK;
}

static void fill_table(const std::vector<int64_t> &deg, double e, int32_t *out) {
    for (size_t c = 0; c < deg.size(); ++c) out[c] = (int32_t)degree_target(deg[c], e);
}

static ad_status keep_at(ad_graph_t g, const int4 *info, const Tiles &t, const std::vector<double> &e_per_graph,
                         uint8_t *keep, int64_t *n_kept) {
    const int32_t ndc = std::max<int32_t>(g->n_deg_classes, 1);
    std::vector<int32_t> Th((size_t)g->G * ndc, 0);
    for (int32_t k = 0; k < g->G; ++k) fill_table(g->distinct_degrees, e_per_graph[k], Th.data() + (size_t)k * ndc);
    int32_t *T = nullptr;
    unsigned long long *kept = nullptr;
    AD_TRY(dalloc_t(g, Th.size(), &T));
    AD_TRY(dalloc_t(g, g->G, &kept));
    AD_TRY(copy_in(g, T, Th.data(), Th.size() * sizeof(int32_t)));
    AD_CUDA_TRY(cudaMemsetAsync(kept, 0, sizeof(unsigned long long) * g->G, g->stream));
    if (t.n > 0)
        AD_LAUNCH(k_keep_at, (int)t.n, 256, 0, g->stream, info, t.graph, t.start, t.end, T, ndc, keep, kept);
    std::vector<unsigned long long> kh(g->G);
    AD_TRY(copy_out(g, kh.data(), kept, sizeof(unsigned long long) * g->G));
    int64_t tot = 0;
    for (auto v : kh) tot += (int64_t)v;
    if (n_kept) *n_kept = tot;
    dfree(g, T);
    dfree(g, kept);
    return AD_OK;
}

ad_status select_per_node_at(ad_graph_t g, const float *score, double e, ad_mode mode, uint8_t *keep,
                             int64_t *n_kept) {
    int4 *info = nullptr;
    AD_TRY(per_node_info(g, score, mode, &info));
    Tiles t;
    AD_TRY(make_tiles(g, t));
    std::vector<double> ev(g->G, e);
    ad_status st = keep_at(g, info, t, ev, keep, n_kept);
    free_tiles(g, t);
    dfree(g, info);
    return st;
}

// Smallest grid point j * 2^-40 (0 < j <= 2^40) whose kept count reaches K,
// per graph, searched with 15 candidates per pass (the same result as 40
// halvings of [0, 1] because the kept count is monotone in e).
ad_status select_per_node_fit(ad_graph_t g, const float *score, double fraction, ad_mode mode, uint8_t *keep,
                              int64_t *n_kept, double *e_used) {
    int4 *info = nullptr;
    AD_TRY(per_node_info(g, score, mode, &info));
    Tiles t;
    AD_TRY(make_tiles(g, t));
    const int32_t ndc = std::max<int32_t>(g->n_deg_classes, 1);
    const int ncand = 15;
    const int64_t ONE = (int64_t)1 << 40;
    std::vector<int64_t> lo(g->G, 0), hi(g->G, ONE), K(g->G);
    for (int32_t k = 0; k < g->G; ++k) K[k] = target_count(g->eoff_h[k + 1] - g->eoff_h[k], fraction);
    int32_t *T = nullptr;
    unsigned long long *hist = nullptr;
    AD_TRY(dalloc_t(g, (size_t)g->G * ncand * ndc, &T));
    AD_TRY(dalloc_t(g, (size_t)g->G * 16, &hist));
    std::vector<int32_t> Th((size_t)g->G * ncand * ndc);
    std::vector<unsigned long long> hh((size_t)g->G * 16);
    std::vector<std::vector<int64_t>> cand(g->G);
    for (;;) {
        bool any = false;
        for (int32_t k = 0; k < g->G; ++k) {
            cand[k].clear();
            const int64_t span = hi[k] - lo[k];
            if (span > 1) {
                any = true;
                const int64_t step = (span + 15) / 16;
                for (int64_t j = lo[k] + step; j < hi[k] && (int)cand[k].size() < ncand; j += step) cand[k].push_back(j);
            }
            for (int c = 0; c < ncand; ++c) {
                // unused slots repeat hi (kept count there is >= K already)
                const int64_t j = c < (int)cand[k].size() ? cand[k][c] : hi[k];
                fill_table(g->distinct_degrees, std::ldexp((double)j, -40), Th.data() + ((size_t)k * ncand + c) * ndc);
            }
        }
        if (!any) break;
        AD_TRY(copy_in(g, T, Th.data(), Th.size() * sizeof(int32_t)));
        AD_CUDA_TRY(cudaMemsetAsync(hist, 0, sizeof(unsigned long long) * g->G * 16, g->stream));
        if (t.n > 0)
            AD_LAUNCH(k_count_cand, (int)t.n, 256, 0, g->stream, info, t.graph, t.start, t.end, T, ndc, ncand, hist);
        AD_TRY(copy_out(g, hh.data(), hist, sizeof(unsigned long long) * hh.size()));
        for (int32_t k = 0; k < g->G; ++k) {
            int64_t cum = 0;
            int64_t new_lo = lo[k], new_hi = hi[k];
            for (int c = 0; c < (int)cand[k].size(); ++c) {
                cum += (int64_t)hh[(size_t)k * 16 + c];
                if (cum >= K[k]) { new_hi = cand[k][c]; break; }
                new_lo = cand[k][c];
            }
            lo[k] = new_lo;
            hi[k] = new_hi;
        }
    }
    std::vector<double> ev(g->G);
    for (int32_t k = 0; k < g->G; ++k) ev[k] = std::ldexp((double)hi[k], -40);
    ad_status st = keep_at(g, info, t, ev, keep, n_kept);
    if (e_used) *e_used = g->G > 0 ? ev[0] : -1.0;
    dfree(g, T);
    dfree(g, hist);
    free_tiles(g, t);
    dfree(g, info);
    return st;
}

ad_status check_scores(ad_graph_t g, const float *score) {
    if (g->m == 0) return AD_OK;
    unsigned long long *bad = nullptr;
    AD_TRY(dalloc_t(g, 1, &bad));
    AD_CUDA_TRY(cudaMemsetAsync(bad, 0xff, sizeof(unsigned long long), g->stream));
    AD_LAUNCH(k_check_scores, g->num_sms * 8, 256, 0, g->stream, score, g->m, bad);
    unsigned long long b = 0;
    AD_TRY(copy_out(g, &b, bad, sizeof(b)));
    dfree(g, bad);
    if (b != ~0ull) return fail(AD_ERR_INVALID_ARG, "score " + std::to_string(b) + " is negative or not finite");
    return AD_OK;
}

}  // namespace ad

// ----------------------------------------------------------------------------
// Whole-graph selection that allocates nothing (ad_select_whole_graph_noalloc).
//
// Some callers cannot let a library allocate device memory: a process whose
// device memory is entirely pre-reserved by its own allocator or arena (where
// a foreign cudaMalloc would fail or fragment it), or a latency-critical
// service that must not hit the allocator on its request path.  For them the
// radix select above runs with all of its scratch -- selection state, the
// three digit histograms, the tile list and the per-tile tie counts -- in one
// fixed file-scope device array sized for at most kNoAllocMaxEdges edges.
// Every GPU that loads this library holds that array until the process exits.
// All calls on a device share it and it keeps the previous call's contents, so
// each call first rewrites everything it reads; calls whose work overlaps on
// the GPU (two streams, or two host threads) race on it and must be ordered by
// the caller.
// ----------------------------------------------------------------------------
namespace ad {

constexpr int64_t kNoAllocMaxEdges = (int64_t)1 << 26;
constexpr int64_t kNoAllocMaxTiles = kNoAllocMaxEdges / kTile;
constexpr int kNoAllocMaxDevices = 64;

struct NoAllocScratch {
    SelState st;
    unsigned long long bad;
    int32_t first_tile[2];
    uint32_t hist[3 * 2048];
    int32_t tg[kNoAllocMaxTiles];
    int64_t ts[kNoAllocMaxTiles];
    int64_t te[kNoAllocMaxTiles];
    int64_t ties[kNoAllocMaxTiles];
    int64_t tie_off[kNoAllocMaxTiles];
};

static __device__ __align__(256) unsigned char g_noalloc_scratch[sizeof(NoAllocScratch)];

static std::mutex g_noalloc_mu;
static NoAllocScratch *g_noalloc_ptr[kNoAllocMaxDevices] = {};

// Device address of the scratch array on the current device (looked up once per device).
static ad_status noalloc_scratch(NoAllocScratch **out) {
    int dev = 0;
    AD_CUDA_TRY(cudaGetDevice(&dev));
    if (dev < 0 || dev >= kNoAllocMaxDevices) return fail(AD_ERR_INVALID_ARG, "device id out of range");
    std::lock_guard<std::mutex> lk(g_noalloc_mu);
    if (!g_noalloc_ptr[dev]) {
        void *p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || !p)
            return fail(AD_ERR_CUDA, std::string("cudaGetSymbolAddress(scratch): ") + cudaGetErrorString(e));
        g_noalloc_ptr[dev] = static_cast<NoAllocScratch *>(p);
    }
    *out = g_noalloc_ptr[dev];
    return AD_OK;
}

// Rewrites every scratch field a call reads: state, histograms, tile list.
__global__ void k_noalloc_init(NoAllocScratch *s, int64_t m, int64_t K, int64_t ntiles) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < 3 * 2048; t += stride) s->hist[t] = 0;
    for (int64_t b = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; b < ntiles; b += stride) {
        s->tg[b] = 0;
        s->ts[b] = b * kTile;
        s->te[b] = (b + 1) * kTile < m ? (b + 1) * kTile : m;
        s->ties[b] = 0;
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        s->st.prefix = 0;
        s->st.pad = 0;
        s->st.K = K;
        s->st.m = m;
        s->st.k_rem = (K > 0 && K < m) ? K : 0;
        s->bad = ~0ull;
        s->first_tile[0] = 0;
        s->first_tile[1] = (int32_t)ntiles;
    }
}

// Exclusive scan of at most kNoAllocMaxTiles values by one CTA of 1024 threads.
__global__ void k_noalloc_scan(const int64_t *in, int64_t *out, int64_t n) {
    __shared__ int64_t sh[32];
    const int64_t per = (n + blockDim.x - 1) / blockDim.x;
    const int64_t b0 = (int64_t)threadIdx.x * per;
    int64_t local = 0;
    for (int64_t i = b0; i < b0 + per && i < n; ++i) local += in[i];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    int64_t x = local;
    for (int o = 1; o < 32; o <<= 1) {
        const int64_t y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) sh[warp] = x;
    __syncthreads();
    if (warp == 0) {
        int64_t v = lane < nw ? sh[lane] : 0;
        for (int o = 1; o < 32; o <<= 1) {
            const int64_t y = __shfl_up_sync(0xffffffffu, v, o);
            if (lane >= o) v += y;
        }
        if (lane < nw) sh[lane] = v;
    }
    __syncthreads();
    int64_t run = (warp > 0 ? sh[warp - 1] : 0) + x - local;
    for (int64_t i = b0; i < b0 + per && i < n; ++i) {
        out[i] = run;
        run += in[i];
    }
}

}  // namespace ad

extern "C" ad_status ad_select_whole_graph_noalloc(const float *score, int64_t m, double fraction, ad_mode mode,
                                                   uint8_t *keep, int64_t *n_kept, void *stream) {
    using namespace ad;
    if (m < 0 || m > kNoAllocMaxEdges)
        return fail(AD_ERR_INVALID_ARG, "m = " + std::to_string(m) + " exceeds the fixed scratch limit of " +
                                            std::to_string(kNoAllocMaxEdges) + " edges");
    if (!(fraction >= 0.0 && fraction <= 1.0)) return fail(AD_ERR_INVALID_ARG, "fraction must be in [0, 1]");
    if (mode != AD_MODE_LOCAL && mode != AD_MODE_GLOBAL) return fail(AD_ERR_INVALID_ARG, "bad mode");
    if (m > 0 && (!is_device_ptr(score) || !is_device_ptr(keep)))
        return fail(AD_ERR_INVALID_ARG, "score and keep must be device arrays (nothing is staged)");
    NoAllocScratch *s = nullptr;
    AD_TRY(noalloc_scratch(&s));
    const int64_t K = target_count(m, fraction);
    if (n_kept) *n_kept = K;
    if (m == 0) return AD_OK;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const int desc = mode == AD_MODE_GLOBAL ? 1 : 0;
    const int64_t ntiles = (m + kTile - 1) / kTile;
    AD_LAUNCH(k_noalloc_init, 64, 256, 0, st, s, m, K, ntiles);
    AD_LAUNCH(k_check_scores, 152 * 8, 256, 0, st, score, m, &s->bad);
    unsigned long long bad = 0;
    AD_CUDA_TRY(cudaMemcpyAsync(&bad, &s->bad, sizeof(bad), cudaMemcpyDeviceToHost, st));
    AD_CUDA_TRY(cudaStreamSynchronize(st));
    if (bad != ~0ull) return fail(AD_ERR_INVALID_ARG, "score " + std::to_string(bad) + " is negative or not finite");
    const int shifts[3] = {21, 10, 0}, bits[3] = {11, 11, 10};
    const uint32_t hi_masks[3] = {0u, 0xFFE00000u, 0xFFFFFC00u};
    for (int pass = 0; pass < 3; ++pass) {
        AD_LAUNCH(k_sel_hist, (int)ntiles, 256, 0, st, score, desc, s->tg, s->ts, s->te, &s->st, shifts[pass],
                  bits[pass], hi_masks[pass], s->hist + pass * 2048);
        AD_LAUNCH(k_sel_find, 1, 256, 0, st, s->hist + pass * 2048, &s->st, shifts[pass], bits[pass]);
    }
    AD_LAUNCH(k_sel_ties, (int)ntiles, 256, 0, st, score, desc, s->tg, s->ts, s->te, &s->st, s->ties);
    AD_LAUNCH(k_noalloc_scan, 1, 1024, 0, st, s->ties, s->tie_off, ntiles);
    AD_LAUNCH(k_sel_write, (int)ntiles, kTileThreads, 0, st, score, desc, s->tg, s->ts, s->te, &s->st, s->tie_off,
              s->first_tile, keep);
    return AD_OK;
}
