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

// Ranks are written per CSR entry in both orders; k_info then gathers them per
// edge.  Both orders come from one ascending sort of (key, position): with lt
// and leq the numbers of entries of the row with key < k and key <= k, the
// rank of an entry in the descending order (ties still by ascending position)
// is (d - leq) + (r_asc - lt).
struct RankOut {
    uint32_t *asc, *desc;
};
__device__ __forceinline__ void put_ranks(const RankOut &o, int64_t p, int d, uint32_t r_asc, uint32_t lt,
                                          uint32_t leq) {
    o.asc[p] = r_asc;
    o.desc[p] = (uint32_t)d - leq + (r_asc - lt);
}

constexpr int kSortCap = 4096;      // rows up to this degree are sorted by one CTA in shared memory
constexpr int kSortCapLarge = 12288; // ... and up to this one by one CTA holding most of an SM's shared memory

// rows of degree <= GS (8 or 32): a group of GS lanes per row, one entry per
// lane, rank = number of smaller (key, position) pairs in the row
template <int GS>
__global__ void k_rank_count(const int64_t *rp, const int64_t *rows, int64_t nrows, const uint32_t *ekey,
                             RankOut out) {
    const int lane = threadIdx.x & 31, sub = lane / GS, gl = lane % GS;
    const unsigned gmask = GS == 32 ? 0xffffffffu : (((1u << GS) - 1u) << (sub * GS));
    constexpr int RPW = 32 / GS;   // rows per warp
    const int64_t W = (int64_t)gridDim.x * (blockDim.x >> 5) * RPW;
    for (int64_t t = (blockIdx.x * (int64_t)(blockDim.x >> 5) + (threadIdx.x >> 5)) * RPW + sub; ; t += W) {
        const bool live = t < nrows;
        if (!__any_sync(0xffffffffu, live)) break;
        int64_t i = 0, p0 = 0;
        int d = 0;
        if (live) { i = rows[t]; p0 = rp[i]; d = (int)(rp[i + 1] - p0); }
        const uint32_t k = gl < d ? ekey[p0 + gl] : 0xffffffffu;
        uint32_t r = 0, lt = 0, leq = 0;
        // d is the same on every lane of the group, so the group's shuffles stay in step
        for (int l = 0; l < d; ++l) {
            const uint32_t o = __shfl_sync(gmask, k, l, GS);
            r += (o < k || (o == k && l < gl)) ? 1u : 0u;
            lt += o < k ? 1u : 0u;
            leq += o <= k ? 1u : 0u;
        }
        if (gl < d) put_ranks(out, p0 + gl, d, r, lt, leq);
    }
}

// rows of degree <= 32 P: one warp sorts the row's (key, position) pairs in
// registers (bitonic network over index lane * P + j), then writes the ranks
template <int P>
__global__ void __launch_bounds__(256) k_rank_wsort(const int64_t *rp, const int64_t *rows, int64_t nrows,
                                                    const uint32_t *ekey, RankOut out) {
    constexpr int N = 32 * P;
    const int lane = threadIdx.x & 31;
    const int64_t W = (int64_t)gridDim.x * (blockDim.x >> 5);
    for (int64_t t = blockIdx.x * (int64_t)(blockDim.x >> 5) + (threadIdx.x >> 5); t < nrows; t += W) {
        const int64_t i = rows[t];
        const int64_t p0 = rp[i];
        const int d = (int)(rp[i + 1] - p0);
        unsigned long long v[P];
#pragma unroll
        for (int j = 0; j < P; ++j) {
            const int idx = lane * P + j;
            v[j] = idx < d ? (((unsigned long long)ekey[p0 + idx] << 32) | (unsigned)idx) : ~0ull;
        }
#pragma unroll
        for (int size = 2; size <= N; size <<= 1) {
#pragma unroll
            for (int stride = size >> 1; stride > 0; stride >>= 1) {
                if (stride < P) {
#pragma unroll
                    for (int j = 0; j < P; ++j) {
                        if ((j & stride) == 0) {
                            const int jj = j | stride;
                            const bool up = (((lane * P + j) & size) == 0);
                            const unsigned long long a = v[j], b = v[jj];
                            if ((a > b) == up) { v[j] = b; v[jj] = a; }
                        }
                    }
                } else {
                    const int ls = stride / P;
                    const bool lower = (lane & ls) == 0;
#pragma unroll
                    for (int j = 0; j < P; ++j) {
                        const unsigned long long o = __shfl_xor_sync(0xffffffffu, v[j], ls);
                        const bool up = (((lane * P + j) & size) == 0);
                        v[j] = (lower == up) ? (o < v[j] ? o : v[j]) : (o > v[j] ? o : v[j]);
                    }
                }
            }
        }
        // tie runs of equal keys: first = max-scan of run starts, last = min-scan of run ends
        const uint32_t prev_last = (uint32_t)(__shfl_up_sync(0xffffffffu, v[P - 1], 1) >> 32);
        const uint32_t next_first = (uint32_t)(__shfl_down_sync(0xffffffffu, v[0], 1) >> 32);
        int first[P], last[P];
        int run = 0;
#pragma unroll
        for (int j = 0; j < P; ++j) {
            const int idx = lane * P + j;
            const uint32_t kj = (uint32_t)(v[j] >> 32);
            const uint32_t kp = j > 0 ? (uint32_t)(v[j - 1] >> 32) : prev_last;
            if (idx == 0 || kj != kp) run = idx;
            first[j] = run;
        }
        int carry = first[P - 1];
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, carry, o);
            if (lane >= o) carry = max(carry, y);
        }
        int excl = __shfl_up_sync(0xffffffffu, carry, 1);
        if (lane == 0) excl = 0;
#pragma unroll
        for (int j = 0; j < P; ++j) first[j] = max(first[j], excl);
        run = N - 1;
#pragma unroll
        for (int j = P - 1; j >= 0; --j) {
            const int idx = lane * P + j;
            const uint32_t kj = (uint32_t)(v[j] >> 32);
            const uint32_t kn = j < P - 1 ? (uint32_t)(v[j + 1] >> 32) : next_first;
            if (idx == N - 1 || kj != kn) run = idx;
            last[j] = run;
        }
        carry = last[0];
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_down_sync(0xffffffffu, carry, o);
            if (lane + o < 32) carry = min(carry, y);
        }
        int excl_r = __shfl_down_sync(0xffffffffu, carry, 1);
        if (lane == 31) excl_r = N - 1;
#pragma unroll
        for (int j = 0; j < P; ++j) last[j] = min(last[j], excl_r);
#pragma unroll
        for (int j = 0; j < P; ++j)
            if (v[j] != ~0ull)
                put_ranks(out, p0 + (int64_t)(v[j] & 0xffffffffull), d, (uint32_t)(lane * P + j),
                          (uint32_t)first[j], (uint32_t)last[j] + 1);
    }
}

// first index of a sorted shared-memory array holding a value >= v
__device__ __forceinline__ int lower_bound_smem(const unsigned long long *a, int n, unsigned long long v) {
    int lo = 0, hi = n;
    while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if (a[mid] < v) lo = mid + 1; else hi = mid;
    }
    return lo;
}

// Rows of degree in (512, CAP] (CAP = kSortCap, or kSortCapLarge for the rows
// above kSortCap): one CTA per row sorts (key << 32 |
// position) with a stable LSD radix sort in shared memory (8-bit digits; a
// digit pass whose keys all share one digit is skipped).  Each warp owns a
// contiguous segment of whole 32-entry chunks.  Digit counts are shared-memory
// atomics per warp; the offsets run digit-major, warp-minor; inside a chunk,
// entries with equal digits keep lane order (their peer mask comes from one
// ballot per digit bit), so every pass is stable.  Four barriers per pass.
constexpr int kMidThreads = 256, kMidWarps = kMidThreads / 32;
static_assert(kMidThreads == 256, "one thread per 8-bit digit");
constexpr size_t mid_smem(int cap) { return 2 * (size_t)cap * sizeof(unsigned long long) + kMidWarps * 256 * sizeof(uint32_t); }
static_assert(mid_smem(kSortCapLarge) <= 227 * 1024, "the large CTA sort must fit one CTA's shared memory");

template <int CAP>
__global__ void __launch_bounds__(kMidThreads) k_rank_mid(const int64_t *rp, const int64_t *rows, const uint32_t *ekey,
                                                          RankOut out) {
    extern __shared__ unsigned long long mid_sm[];
    unsigned long long *a = mid_sm, *b = mid_sm + CAP;
    uint32_t *cnt = reinterpret_cast<uint32_t *>(mid_sm + 2 * CAP);   // [warp][256] counts, then offsets
    __shared__ uint32_t wsum[kMidWarps];                                    // digit totals of 32-digit blocks
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int64_t row = rows[blockIdx.x];
    const int64_t p0 = rp[row];
    const int d = (int)(rp[row + 1] - p0);
    for (int t = threadIdx.x; t < d; t += kMidThreads) a[t] = ((unsigned long long)ekey[p0 + t] << 32) | (unsigned)t;
    const int seg = (((d + kMidWarps - 1) / kMidWarps) + 31) & ~31;           // entries per warp, whole chunks
    const int s0 = warp * seg, s1 = min(d, s0 + seg);
    const unsigned lt_mask = (1u << lane) - 1u;
    __syncthreads();
    for (int shift = 32; shift < 64; shift += 8) {
        for (int q = lane; q < 256; q += 32) cnt[warp * 256 + q] = 0;
        __syncwarp();
        for (int t = s0 + lane; t < s1; t += 32) atomicAdd(cnt + warp * 256 + (int)((a[t] >> shift) & 0xff), 1u);
        __syncthreads();
        // thread q: digit q's total over warps; offsets digit-major, warp-minor
        const int q = threadIdx.x;
        uint32_t tot = 0;
        for (int w = 0; w < kMidWarps; ++w) tot += cnt[w * 256 + q];
        uint32_t inc = tot;                                                       // inclusive scan over this warp's digits
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(0xffffffffu, inc, o);
            if (lane >= o) inc += y;
        }
        if (lane == 31) wsum[warp] = inc;
        if (__syncthreads_or(tot == (uint32_t)d)) continue;                       // one digit holds all: order unchanged
        uint32_t run = inc - tot;
        for (int w = 0; w < warp; ++w) run += wsum[w];
        for (int w = 0; w < kMidWarps; ++w) {
            const uint32_t c2 = cnt[w * 256 + q];
            cnt[w * 256 + q] = run;
            run += c2;
        }
        __syncthreads();
        for (int c = s0; c < s1; c += 32) {                                       // stable scatter (warp-uniform loop)
            const int t = c + lane;
            const bool live = t < s1;
            const unsigned long long v = live ? a[t] : 0ull;
            const uint32_t dg = live ? (uint32_t)((v >> shift) & 0xff) : 0u;
            unsigned peers = __ballot_sync(0xffffffffu, live);
#pragma unroll
            for (int bit = 0; bit < 8; ++bit) {
                const unsigned bb = __ballot_sync(0xffffffffu, (dg >> bit) & 1u);
                peers &= ((dg >> bit) & 1u) ? bb : ~bb;
            }
            const uint32_t before = (uint32_t)__popc(peers & lt_mask);
            if (live) b[cnt[warp * 256 + dg] + before] = v;
            __syncwarp();
            if (live && before == 0) cnt[warp * 256 + dg] += (uint32_t)__popc(peers);
            __syncwarp();
        }
        __syncthreads();
        unsigned long long *tmp = a;
        a = b;
        b = tmp;
    }
    for (int t = threadIdx.x; t < d; t += kMidThreads) {
        const unsigned long long k32 = a[t] & 0xffffffff00000000ull;
        // tie runs need a search; a key unlike both neighbours is its own run
        const int lt = (t > 0 && (a[t - 1] & 0xffffffff00000000ull) == k32) ? lower_bound_smem(a, d, k32) : t;
        const int leq = (t + 1 < d && (a[t + 1] & 0xffffffff00000000ull) == k32)
                            ? lower_bound_smem(a, d, k32 + 0x100000000ull)   // real keys are < 2^32 - 1
                            : t + 1;
        put_ranks(out, p0 + (int64_t)(a[t] & 0xffffffffull), d, (uint32_t)t, (uint32_t)lt, (uint32_t)leq);
    }
}

// k_rank_mid needs more than the default 48 KB of dynamic shared memory: opt in
// once per device (the attribute belongs to the current device's context)
static ad_status set_mid_smem() {
    static std::mutex mu;
    static bool done[64] = {};
    int dev = 0;
    AD_CUDA_TRY(cudaGetDevice(&dev));
    std::lock_guard<std::mutex> lk(mu);
    if (dev < 0 || dev >= 64) return fail(AD_ERR_CUDA, "device index out of range");
    if (!done[dev]) {
        AD_CUDA_TRY(cudaFuncSetAttribute(k_rank_mid<kSortCap>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)mid_smem(kSortCap)));
        AD_CUDA_TRY(cudaFuncSetAttribute(k_rank_mid<kSortCapLarge>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)mid_smem(kSortCapLarge)));
        done[dev] = true;
    }
    return AD_OK;
}

// Rows of degree > kSortCapLarge.  Their entries are listed once per handle
// (position bpos and row slot bseg, row slots in bstart order); each call sorts
// (row slot, key) with the stable radix sort, whose input order is by position
// inside a row, so each row's entries end up in (key, position) order.
__global__ void k_big_expand(const int64_t *rows, const int64_t *rp, const int64_t *bstart, int64_t *bpos,
                             int32_t *bseg) {
    const int64_t row = rows[blockIdx.x];
    const int64_t p0 = rp[row], d = rp[row + 1] - p0, o = bstart[blockIdx.x];
    for (int64_t t = threadIdx.x; t < d; t += blockDim.x) {
        bpos[o + t] = p0 + t;
        bseg[o + t] = (int32_t)blockIdx.x;
    }
}

__global__ void k_big_keys(const int64_t *bpos, const int32_t *bseg, int64_t nb, const uint32_t *ekey,
                           uint64_t *keys, int64_t *vals) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < nb; i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t p = bpos[i];
        keys[i] = ((uint64_t)(uint32_t)bseg[i] << 32) | ekey[p];
        vals[i] = p;
    }
}

// after the sort: rank = index inside the row's run of the sorted array; the
// first and last index of a run of equal keys give lt and leq (binary search
// only where a neighbour holds the same key)
__global__ void k_big_ranks(const uint64_t *keys, const int64_t *vals, int64_t nb, const int64_t *bstart,
                            RankOut out) {
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < nb; t += (int64_t)gridDim.x * blockDim.x) {
        const uint64_t k = keys[t];
        const int b = (int)(k >> 32);
        const int64_t s = bstart[b], e = bstart[b + 1];
        int64_t lt = t, le = t + 1;
        if (t > s && keys[t - 1] == k) {
            int64_t lo = s, hi = t;
            while (lo < hi) {
                const int64_t mid = (lo + hi) >> 1;
                if (keys[mid] < k) lo = mid + 1; else hi = mid;
            }
            lt = lo;
        }
        if (t + 1 < e && keys[t + 1] == k) {
            int64_t lo = t + 1, hi = e;
            while (lo < hi) {
                const int64_t mid = (lo + hi) >> 1;
                if (keys[mid] <= k) lo = mid + 1; else hi = mid;
            }
            le = lo;
        }
        put_ranks(out, vals[t], (int)(e - s), (uint32_t)(t - s), (uint32_t)(lt - s),
                  (uint32_t)(le - s));
    }
}

__global__ void k_row_degrees(const int64_t *rows, int64_t nrows, const int64_t *rp, int64_t *deg) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < nrows) deg[i] = rp[rows[i] + 1] - rp[rows[i]];
}

// upper CSR entry of every edge (built once per handle)
__global__ void k_edge_pos(const int32_t *erow, const int32_t *col, const int64_t *eid, int64_t nnz, int64_t *epos) {
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < nnz; p += (int64_t)gridDim.x * blockDim.x)
        if (col[p] > erow[p]) epos[eid[p]] = p;
}

// per edge e = (i < j): (rank at i, rank at j, degree class of i, of j) in both orders
__global__ void k_info(const int64_t *epos, const int64_t *mirror, const int32_t *erow, const int32_t *col,
                       const int32_t *dc, int64_t m, const uint32_t *rasc, const uint32_t *rdesc, int4 *info_asc,
                       int4 *info_desc) {
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < m; e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t p = epos[e], q = mirror[p];
        const int di = dc[erow[p]], dj = dc[col[p]];
        info_asc[e] = make_int4((int)rasc[p], (int)rasc[q], di, dj);
        info_desc[e] = make_int4((int)rdesc[p], (int)rdesc[q], di, dj);
    }
}

// rank class of every row: 0 none, 1 d <= 8, 2 d <= 16, 3 d <= 32, 4 d <= 64, 5 d <= 128, 6 d <= 256,
// 7 d <= 512, 8 d <= kSortCap, 9 d <= kSortCapLarge, 10 larger
constexpr int kRankClasses = 11;
__global__ void k_rank_classes(const int64_t *rp, int64_t n, int8_t *cls /* class - 1; -1 for degree 0 */) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t d = rp[i + 1] - rp[i];
        const int c = d == 0 ? 0 : d <= 8 ? 1 : d <= 16 ? 2 : d <= 32 ? 3 : d <= 64 ? 4 : d <= 128 ? 5 : d <= 256 ? 6
                    : d <= 512 ? 7 : d <= kSortCap ? 8 : d <= kSortCapLarge ? 9 : 10;
        cls[i] = (int8_t)(c - 1);
    }
}

__global__ void k_widen_rows(const int32_t *order, int64_t n, int64_t *out) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        out[i] = order[i];
}

// First candidate (1..nc) at which the edge is kept, nc + 1 when it is not kept
// at any; per-graph histograms of that index; the index is stored for compaction.
__device__ __forceinline__ int graph_of_edge(const int64_t *goff_e, int G, int64_t e) {
    int lo = 0, hi = G;
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (__ldg(goff_e + mid) <= e) lo = mid; else hi = mid;
    }
    return lo;
}

// The same for the edges of a whole warp (all 32 lanes call it; e < 0: no
// edge): the graph of the first lane with an edge is looked up once and
// checked by every lane, since a warp's edges mostly lie in one graph; lanes
// outside it search on their own.
__device__ __forceinline__ int graph_of_edge_warp(const int64_t *goff_e, int G, int64_t e) {
    const unsigned have = __ballot_sync(0xffffffffu, e >= 0);
    if (!have) return 0;
    const int src = __ffs(have) - 1;
    const int64_t e0 = __shfl_sync(0xffffffffu, e, src);
    int g0 = 0;
    if ((threadIdx.x & 31) == src) g0 = graph_of_edge(goff_e, G, e0);
    g0 = __shfl_sync(0xffffffffu, g0, src);
    if (e < 0) return 0;
    if (__ldg(goff_e + g0) <= e && e < __ldg(goff_e + g0 + 1)) return g0;
    return graph_of_edge(goff_e, G, e);
}

constexpr int kSharedFitProblems = 8;   // problems whose histograms a block keeps in shared memory
__global__ void k_count_cand(const int4 *info, const int64_t *list, int64_t L, const int64_t *Ld, const int64_t *goff_e,
                             int G, const int32_t *T, int32_t ndc, int nc, unsigned long long *hist, uint8_t *cstar) {
    __shared__ unsigned int h[kSharedFitProblems * 32];
    const bool shared_h = G <= kSharedFitProblems;
    for (int j = threadIdx.x; j < kSharedFitProblems * 32; j += blockDim.x) h[j] = 0;
    __syncthreads();
    if (Ld) L = *Ld;    // length of a list compacted on the device
    const int lane = threadIdx.x & 31;
    // warp-uniform trip count, so that the whole warp meets at the histogram update
    for (int64_t base = blockIdx.x * (int64_t)blockDim.x + (threadIdx.x & ~31); base < L;
         base += (int64_t)gridDim.x * blockDim.x) {
        const int64_t t = base + lane;
        int lo = 32;       // bin of a lane without an edge: never counted
        int gph = 0;
        const int64_t e = t < L ? (list ? list[t] : t) : -1;
        if (G > 1) gph = graph_of_edge_warp(goff_e, G, e);
        if (t < L) {
            const int4 f = info[e];
            const int32_t *Tg = T + (size_t)gph * nc * ndc;
            int l = 0, hi = nc;   // first candidate index (0-based) at which the edge is kept; nc = none
            while (l < hi) {
                const int mid = (l + hi) >> 1;
                const int32_t *Tm = Tg + (size_t)mid * ndc;
                if (f.x < Tm[f.z] || f.y < Tm[f.w]) hi = mid; else l = mid + 1;
            }
            cstar[t] = (uint8_t)l;
            lo = l;
        }
        // lanes with the same (problem, bin) add once (few bins: per-lane atomics would serialise)
        const int key = lo < 32 ? gph * 32 + lo : -1;
        const unsigned peers = __match_any_sync(0xffffffffu, key);
        if (key >= 0 && (peers & ((1u << lane) - 1u)) == 0) {
            if (shared_h) atomicAdd(&h[key], (unsigned)__popc(peers));
            else atomicAdd(hist + key, (unsigned long long)__popc(peers));
        }
    }
    __syncthreads();
    if (shared_h)
        for (int j = threadIdx.x; j < G * 32; j += blockDim.x)
            if (h[j]) atomicAdd(hist + j, (unsigned long long)h[j]);
}

// undecided edges of the next pass: those whose first candidate is the chosen one
__global__ void k_undecided_flags(const int64_t *list, int64_t L, const uint8_t *cstar, const int64_t *goff_e, int G,
                                  const int32_t *jsel, uint8_t *flag) {
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < L; t += (int64_t)gridDim.x * blockDim.x) {
        const int64_t e = list ? list[t] : t;
        const int gph = G > 1 ? graph_of_edge(goff_e, G, e) : 0;
        flag[t] = cstar[t] == jsel[gph] ? 1 : 0;
    }
}

__global__ void k_gather_list(const int64_t *list, const int64_t *idx, int64_t L, int64_t *out) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t < L) out[t] = list ? list[idx[t]] : idx[t];
}

// ----------------------------------------------------------------------------
// Device-resident search of the exponent (same passes as the host loop of
// select_per_node_fit_host, without a host round trip per pass).  T(d, e) is
// evaluated with the device pow; where d^e - 1e-9 lies so close to an integer
// that a pow differing from the host's by a few units in the last place could
// round the other way, the pass raises a flag and the caller repeats the
// search with host tables, so the integer decisions stay those of FP64 pow on
// the host.
// ----------------------------------------------------------------------------
struct FitState {
    int64_t lo, hi, K, base;
    int32_t jsel, pad;
};

constexpr int kFitCand = 16;          // 15 interior grid points + the upper end
constexpr int kFitPasses = 10;        // 16^10 = 2^40: every interval shrinks to one grid step

__device__ __forceinline__ int fit_interior(const FitState &s, int64_t &step) {
    const int64_t span = s.hi - s.lo;
    if (span <= 1) { step = 0; return 0; }
    step = (span + kFitCand - 1) / kFitCand;
    const int64_t n = (span - 1) / step;
    return (int)(n < kFitCand - 1 ? n : kFitCand - 1);
}

__device__ __forceinline__ int64_t fit_point(const FitState &s, int cc) {
    int64_t step;
    const int ni = fit_interior(s, step);
    return cc < ni ? s.lo + step * (cc + 1) : s.hi;
}

// The chosen candidate of a problem from its histogram of first-kept
// candidates: the first candidate whose cumulative count reaches K becomes the
// new upper end, the one before it the new lower end (jsel = -1: converged).
__device__ __forceinline__ FitState fit_choose(FitState s, const unsigned long long *h) {
    int64_t step;
    const int ni = fit_interior(s, step);
    if (s.hi - s.lo <= 1) {
        s.jsel = -1;
        return s;
    }
    int64_t cum = s.base;
    int chosen = ni;                    // the upper end always reaches K
    for (int cc = 0; cc <= ni; ++cc) {
        cum += (int64_t)h[cc];
        if (cum >= s.K) { chosen = cc; break; }
    }
    for (int cc = 0; cc < chosen; ++cc) s.base += (int64_t)h[cc];
    const int64_t nlo = chosen > 0 ? fit_point(s, chosen - 1) : s.lo;
    const int64_t nhi = fit_point(s, chosen);
    s.lo = nlo;
    s.hi = nhi;
    s.jsel = chosen;
    return s;
}

// One step of the search for P problems at once, between the count of pass p
// and the count of pass p + 1: every thread takes one (problem, candidate,
// degree class), re-derives its problem's choice from the histogram of pass
// p, carries T at the new interval ends (Tlo / Thi: T of the chosen point and
// of the one before it, read from pass p's tables) and evaluates T at the
// candidates of pass p + 1.  T is monotone in e, so a class with equal ends
// is constant inside and needs no pow.  With first set, the state is the
// initial one (e in [0, 1]: T = 1 and T = d at the ends) and nothing is chosen.
// State, tables, ends and histograms are double-buffered by pass parity.
__global__ void k_fit_advance(int P, int first, int last, const FitState *st_old, FitState *st_new,
                              const unsigned long long *hist, unsigned long long *hist_next, const int32_t *T_cur,
                              int32_t *T_next, const int32_t *Tlo_old, const int32_t *Thi_old, int32_t *Tlo_new,
                              int32_t *Thi_new, const int64_t *ddeg, int32_t ndc, int64_t *next_len, int *ambiguous) {
    const int64_t gtid = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (gtid == 0) *next_len = 0;
    for (int64_t j = gtid; j < (int64_t)P * 32; j += (int64_t)gridDim.x * blockDim.x) hist_next[j] = 0;
    const int64_t total = (int64_t)P * kFitCand * ndc;
    for (int64_t idx = gtid; idx < total; idx += (int64_t)gridDim.x * blockDim.x) {
        const int q = (int)(idx % ndc);
        const int64_t kc = idx / ndc;
        const int cc = (int)(kc % kFitCand), k = (int)(kc / kFitCand);
        const int64_t d = ddeg[q];
        FitState s = st_old[k];
        int32_t tl, th;
        if (first) {
            tl = d > 0 ? 1 : 0;
            th = (int32_t)d;
        } else {
            s = fit_choose(s, hist + (size_t)k * 32);
            tl = Tlo_old[(size_t)k * ndc + q];
            th = Thi_old[(size_t)k * ndc + q];
            if (s.jsel >= 0) {
                if (s.jsel > 0) tl = T_cur[((size_t)k * kFitCand + s.jsel - 1) * ndc + q];
                th = T_cur[((size_t)k * kFitCand + s.jsel) * ndc + q];
            }
        }
        if (cc == 0) {
            Tlo_new[(size_t)k * ndc + q] = tl;
            Thi_new[(size_t)k * ndc + q] = th;
            if (q == 0) st_new[k] = s;
        }
        if (last) continue;
        int64_t step;
        const int ni = fit_interior(s, step);
        int32_t t;
        if (cc >= ni) {
            t = th;                              // the upper end
        } else if (tl == th) {
            t = tl;
        } else {
            const double e = ldexp((double)(s.lo + step * (cc + 1)), -40);
            const double v = pow((double)d, e);
            const double x = v - 1e-9;
            const double f = x - floor(x);
            const double tol = 4e-15 * fmax(v, 1.0);
            if (f < tol || f > 1.0 - tol) atomicExch(ambiguous, 1);
            double c = ceil(x);
            if (c < 1.0) c = 1.0;
            if (c > (double)d) c = (double)d;
            t = (int32_t)c;
        }
        T_next[idx] = t;
    }
}

// undecided edges of the next pass (order within the list does not matter:
// only counts are taken).  One atomic per block and tile: a single counter
// takes millions of survivors in the first pass.
constexpr int kCompactItems = 4;   // elements per thread per tile
__global__ void __launch_bounds__(256) k_fit_compact(const int64_t *list, int64_t L, const int64_t *Ld,
                                                     const uint8_t *cstar, const int64_t *goff_e, int G,
                                                     const FitState *st, int64_t *out, int64_t *out_len) {
    __shared__ unsigned int wcount[8];
    __shared__ unsigned long long base_sh;
    if (Ld) L = *Ld;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int64_t tile = (int64_t)blockDim.x * kCompactItems;
    for (int64_t t0 = blockIdx.x * tile; t0 < L; t0 += (int64_t)gridDim.x * tile) {
        bool take[kCompactItems];
        int64_t ev[kCompactItems];
        unsigned mine = 0;
#pragma unroll
        for (int u = 0; u < kCompactItems; ++u) {
            const int64_t t = t0 + (int64_t)u * blockDim.x + threadIdx.x;
            const int64_t e = t < L ? (list ? list[t] : t) : -1;
            const int gph = G > 1 ? graph_of_edge_warp(goff_e, G, e) : 0;
            take[u] = t < L && (int)cstar[t] == st[gph].jsel;
            ev[u] = t < L ? e : 0;
            mine += take[u] ? 1u : 0u;
        }
        // exclusive prefix of `mine` over the block: warp scan, then warp totals
        unsigned incl = mine;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const unsigned y = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += y;
        }
        if (lane == 31) wcount[warp] = incl;
        __syncthreads();
        if (threadIdx.x == 0) {
            unsigned tot = 0;
            for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
                const unsigned c = wcount[w];
                wcount[w] = tot;
                tot += c;
            }
            base_sh = tot ? atomicAdd((unsigned long long *)out_len, (unsigned long long)tot) : 0ull;
        }
        __syncthreads();
        unsigned long long pos = base_sh + wcount[warp] + (incl - mine);
#pragma unroll
        for (int u = 0; u < kCompactItems; ++u)
            if (take[u]) out[pos++] = ev[u];
        __syncthreads();
    }
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

}  // namespace ad

// ----------------------------------------------------------------------------
// Cached per-graph selection workspace
// ----------------------------------------------------------------------------
struct ad_graph_s::SelCache {
    ad::Tiles tiles;
    bool have_tiles = false;
    bool have_lists = false;
    int64_t *rows[10] = {};         // rows of rank classes 1..10
    int64_t nrows[10] = {};
    int64_t *bstart = nullptr;      // class 10: first sorted slot of each row (nrows[9] + 1)
    int64_t *bpos = nullptr;        // class 10 entries: CSR position and row slot
    int32_t *bseg = nullptr;
    int64_t nb_entries = 0;
    ad::DevBuf info, ekey, skey, bvals, T, hist, list_a, list_b, cstar, flag, jsel, kept, st, hist3, ties,
        tie_off, ddeg, fit, fit_tb, rank2, info_other;
    int64_t *epos = nullptr;      // upper CSR entry of every edge
    bool have_ddeg = false;       // ddeg: the distinct degrees on the device
    bool info_valid = false;      // info holds the ranks of the handle's own distances
    uint64_t info_version = 0;
};

namespace ad {

void free_sel_cache(ad_graph_t g) {
    if (!g->sel) return;
    delete g->sel;   // device memory is owned by the handle and released with it
    g->sel = nullptr;
}

static ad_status sel_cache(ad_graph_t g, ad_graph_s::SelCache **out) {
    if (!g->sel) g->sel = new ad_graph_s::SelCache();
    auto *c = g->sel;
    if (!c->have_tiles) {
        AD_TRY(make_tiles(g, c->tiles));
        c->have_tiles = true;
    }
    *out = c;
    return AD_OK;
}

static ad_status rank_lists(ad_graph_t g, ad_graph_s::SelCache *c) {
    if (c->have_lists) return AD_OK;
    const int64_t n = g->n;
    constexpr int NC = kRankClasses - 1;
    // one stable partition of the rows by class (rows of class k, by increasing id, at start[k])
    int8_t *cls = nullptr;
    int32_t *order = nullptr;
    int64_t *rows_all = nullptr;
    AD_TRY(dalloc_t(g, n + 1, &cls));
    AD_TRY(dalloc_t(g, n + 1, &order));
    AD_TRY(dalloc_t(g, n + 1, &rows_all));
    if (n > 0) AD_LAUNCH(k_rank_classes, g->num_sms * 8, 256, 0, g->stream, g->rp, n, cls);
    std::vector<int64_t> start;
    AD_TRY(partition_by_class(g, cls, n, NC, order, start));
    if (start[NC] > 0)
        AD_LAUNCH(k_widen_rows, (int)std::min<int64_t>((start[NC] + 255) / 256, (int64_t)g->num_sms * 16), 256, 0,
                  g->stream, order, start[NC], rows_all);
    for (int k = 0; k < NC; ++k) {
        c->rows[k] = rows_all + start[k];
        c->nrows[k] = start[k + 1] - start[k];
    }
    dfree(g, cls);
    dfree(g, order);
    const int64_t nbig = c->nrows[NC - 1];
    if (nbig > 0) {
        int64_t *deg = nullptr;
        AD_TRY(dalloc_t(g, nbig + 1, &deg));
        AD_TRY(dalloc_t(g, nbig + 1, &c->bstart));
        AD_CUDA_TRY(cudaMemsetAsync(deg, 0, (nbig + 1) * sizeof(int64_t), g->stream));
        AD_LAUNCH(k_row_degrees, (int)((nbig + 255) / 256), 256, 0, g->stream, c->rows[NC - 1], nbig, g->rp, deg);
        AD_TRY(exclusive_scan_i64(g, deg, c->bstart, nbig + 1, &c->nb_entries));
        dfree(g, deg);
        AD_TRY(dalloc_t(g, c->nb_entries, &c->bpos));
        AD_TRY(dalloc_t(g, c->nb_entries, &c->bseg));
        AD_LAUNCH(k_big_expand, (int)nbig, 256, 0, g->stream, c->rows[NC - 1], g->rp, c->bstart, c->bpos, c->bseg);
    }
    c->have_lists = true;
    return AD_OK;
}

// T(d, e) of Alg. 2 in FP64 on the host, the reading min(d, max(1, ceil(d^e - 1e-9))).
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
    ad_graph_s::SelCache *c = nullptr;
    AD_TRY(sel_cache(g, &c));
    const Tiles &t = c->tiles;
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
    AD_TRY(ensure(g, c->st, sizeof(SelState) * g->G));
    AD_TRY(ensure(g, c->hist3, sizeof(uint32_t) * (size_t)g->G * 2048 * 3));
    AD_TRY(ensure(g, c->ties, sizeof(int64_t) * (t.n + 1)));
    AD_TRY(ensure(g, c->tie_off, sizeof(int64_t) * (t.n + 1)));
    SelState *st = static_cast<SelState *>(c->st.ptr);
    uint32_t *hist = static_cast<uint32_t *>(c->hist3.ptr);
    int64_t *ties = static_cast<int64_t *>(c->ties.ptr), *tie_off = static_cast<int64_t *>(c->tie_off.ptr);
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
    if (n_kept) *n_kept = total;
    return AD_OK;
}

// Ranks of every CSR entry inside its row by (ekey, position), ascending, in
// both orders (RankOut), by degree class: register counting, warp bitonic
// sorts, a CTA radix sort in shared memory, and the device radix sort for rows
// above the CTA sort's capacity.
static ad_status entry_ranks(ad_graph_t g, ad_graph_s::SelCache *c, const uint32_t *ekey, RankOut out) {
    auto wblocks = [&](int64_t rows_, int per_warp) {
        return (int)std::max<int64_t>(1, std::min<int64_t>((rows_ + 8 * per_warp - 1) / (8 * per_warp),
                                                           (int64_t)g->num_sms * 32));
    };
    const int64_t *const *rows = c->rows;
    const int64_t *nr = c->nrows;
    if (nr[0] > 0)
        AD_LAUNCH(k_rank_count<8>, wblocks(nr[0], 4), 256, 0, g->stream, g->rp, rows[0],
                  nr[0], ekey, out);
    if (nr[1] > 0)
        AD_LAUNCH(k_rank_count<16>, wblocks(nr[1], 2), 256, 0, g->stream, g->rp, rows[1],
                  nr[1], ekey, out);
    if (nr[2] > 0)
        AD_LAUNCH(k_rank_count<32>, wblocks(nr[2], 1), 256, 0, g->stream, g->rp, rows[2],
                  nr[2], ekey, out);
    if (nr[3] > 0)
        AD_LAUNCH(k_rank_wsort<2>, wblocks(nr[3], 1), 256, 0, g->stream, g->rp, rows[3],
                  nr[3], ekey, out);
    if (nr[4] > 0)
        AD_LAUNCH(k_rank_wsort<4>, wblocks(nr[4], 1), 256, 0, g->stream, g->rp, rows[4],
                  nr[4], ekey, out);
    if (nr[5] > 0)
        AD_LAUNCH(k_rank_wsort<8>, wblocks(nr[5], 1), 256, 0, g->stream, g->rp, rows[5],
                  nr[5], ekey, out);
    if (nr[6] > 0)
        AD_LAUNCH(k_rank_wsort<16>, wblocks(nr[6], 1), 256, 0, g->stream, g->rp, rows[6],
                  nr[6], ekey, out);
    if (nr[7] > 0 || nr[8] > 0) AD_TRY(set_mid_smem());
    if (nr[7] > 0)
        AD_LAUNCH(k_rank_mid<kSortCap>, (int)nr[7], kMidThreads, mid_smem(kSortCap), g->stream, g->rp, rows[7], ekey,
                  out);
    if (nr[8] > 0)
        AD_LAUNCH(k_rank_mid<kSortCapLarge>, (int)nr[8], kMidThreads, mid_smem(kSortCapLarge), g->stream, g->rp,
                  rows[8], ekey, out);
    if (c->nb_entries > 0) {
        const int64_t nb = c->nb_entries, nbig = nr[9];
        AD_TRY(ensure(g, c->skey, sizeof(uint64_t) * nb));
        AD_TRY(ensure(g, c->bvals, sizeof(int64_t) * nb));
        uint64_t *keys = static_cast<uint64_t *>(c->skey.ptr);
        int64_t *vals = static_cast<int64_t *>(c->bvals.ptr);
        const int blocks = (int)std::min<int64_t>((nb + 255) / 256, (int64_t)g->num_sms * 16);
        AD_LAUNCH(k_big_keys, blocks, 256, 0, g->stream, c->bpos, c->bseg, nb, ekey, keys, vals);
        std::vector<int> shifts = {0, 8, 16, 24};          // the 32-bit key
        for (int sh = 32; sh < 64 && ((nbig - 1) >> (sh - 32)) > 0; sh += 8) shifts.push_back(sh);   // row slot
        AD_TRY(radix_sort_pairs(g, keys, vals, nb, shifts));
        AD_LAUNCH(k_big_ranks, blocks, 256, 0, g->stream, keys, vals, nb, c->bstart, out);
    }
    return AD_OK;
}

// Rank of every CSR entry inside its row by (key, position), ascending, for
// caller keys (rank_out[nnz], device; desc_scratch[nnz] receives the
// descending ranks, which the ranking yields as well).
ad_status row_ranks(ad_graph_t g, const uint32_t *ekey, uint32_t *rank_out, uint32_t *desc_scratch) {
    AD_TRY(ensure_degree_classes(g));
    ad_graph_s::SelCache *c = nullptr;
    AD_TRY(sel_cache(g, &c));
    AD_TRY(rank_lists(g, c));
    RankOut out;
    out.asc = rank_out;
    out.desc = desc_scratch;
    return entry_ranks(g, c, ekey, out);
}

// The rows of degree above 512, by increasing id (device array, owned by the
// handle's selection cache; valid until the handle is destroyed).
ad_status long_rows(ad_graph_t g, const int64_t **rows, int64_t *count) {
    AD_TRY(ensure_degree_classes(g));
    ad_graph_s::SelCache *c = nullptr;
    AD_TRY(sel_cache(g, &c));
    AD_TRY(rank_lists(g, c));
    constexpr int NC = kRankClasses - 1;   // classes NC-3 .. NC-1 (degree > 512) are adjacent in one array
    *rows = c->rows[NC - 3];
    *count = c->nrows[NC - 3] + c->nrows[NC - 2] + c->nrows[NC - 1];
    return AD_OK;
}

// Ranks of every CSR entry in both orders, gathered per edge: the info of
// Alg. 2.  For the handle's own distances the result is kept until they change.
static ad_status per_node_info(ad_graph_t g, const float *score, ad_mode mode, int4 **info_out) {
    AD_TRY(ensure_mirror(g));
    AD_TRY(ensure_degree_classes(g));
    ad_graph_s::SelCache *c = nullptr;
    AD_TRY(sel_cache(g, &c));
    AD_TRY(rank_lists(g, c));
    const int64_t nnz = g->nnz;
    AD_TRY(ensure(g, c->info, sizeof(int4) * (2 * g->m + 1)));   // local records, then the global ones
    int4 *info_asc = static_cast<int4 *>(c->info.ptr), *info_desc = info_asc + g->m;
    *info_out = mode == AD_MODE_GLOBAL ? info_desc : info_asc;
    const bool own = score == g->rho && g->have_rho;
    if (own && c->info_valid && c->info_version == g->rho_version) return AD_OK;
    c->info_valid = false;
    if (!c->epos) {
        AD_TRY(dalloc_t(g, g->m + 1, &c->epos));
        if (nnz > 0)
            AD_LAUNCH(k_edge_pos, g->num_sms * 16, 256, 0, g->stream, g->erow, g->col, g->eid, nnz, c->epos);
    }
    AD_TRY(ensure(g, c->rank2, 2 * sizeof(uint32_t) * (nnz + 1)));
    RankOut out;
    out.asc = static_cast<uint32_t *>(c->rank2.ptr);
    out.desc = out.asc + (nnz + 1);
    AD_TRY(ensure(g, c->ekey, sizeof(uint32_t) * (nnz + 1)));
    uint32_t *ekey = static_cast<uint32_t *>(c->ekey.ptr);
    if (nnz > 0) AD_LAUNCH(k_entry_keys, g->num_sms * 16, 256, 0, g->stream, g->eid, nnz, score, 0, ekey);
    AD_TRY(entry_ranks(g, c, ekey, out));
    if (g->m > 0)
        AD_LAUNCH(k_info, g->num_sms * 16, 256, 0, g->stream, c->epos, g->mirror, g->erow, g->col, g->deg_class, g->m,
                  out.asc, out.desc, info_asc, info_desc);
    if (own) {
        c->info_valid = true;
        c->info_version = g->rho_version;
    }
    return AD_OK;
}

static void fill_table(const std::vector<int64_t> &deg, double e, int32_t *out) {
    for (size_t c = 0; c < deg.size(); ++c) out[c] = (int32_t)degree_target(deg[c], e);
}

static ad_status keep_at(ad_graph_t g, const int4 *info, const std::vector<double> &e_per_graph, uint8_t *keep,
                         int64_t *n_kept) {
    ad_graph_s::SelCache *c = g->sel;
    const Tiles &t = c->tiles;
    const int32_t ndc = std::max<int32_t>(g->n_deg_classes, 1);
    std::vector<int32_t> Th((size_t)g->G * ndc, 0);
    for (int32_t k = 0; k < g->G; ++k) fill_table(g->distinct_degrees, e_per_graph[k], Th.data() + (size_t)k * ndc);
    AD_TRY(ensure(g, c->T, Th.size() * sizeof(int32_t)));
    AD_TRY(ensure(g, c->kept, sizeof(unsigned long long) * g->G));
    int32_t *T = static_cast<int32_t *>(c->T.ptr);
    unsigned long long *kept = static_cast<unsigned long long *>(c->kept.ptr);
    AD_TRY(copy_in(g, T, Th.data(), Th.size() * sizeof(int32_t)));
    AD_CUDA_TRY(cudaMemsetAsync(kept, 0, sizeof(unsigned long long) * g->G, g->stream));
    if (t.n > 0)
        AD_LAUNCH(k_keep_at, (int)t.n, 256, 0, g->stream, info, t.graph, t.start, t.end, T, ndc, keep, kept);
    std::vector<unsigned long long> kh(g->G);
    AD_TRY(copy_out(g, kh.data(), kept, sizeof(unsigned long long) * g->G));
    int64_t tot = 0;
    for (auto v : kh) tot += (int64_t)v;
    if (n_kept) *n_kept = tot;
    return AD_OK;
}

ad_status select_per_node_at(ad_graph_t g, const float *score, double e, ad_mode mode, uint8_t *keep,
                             int64_t *n_kept) {
    int4 *info = nullptr;
    AD_TRY(per_node_info(g, score, mode, &info));
    std::vector<double> ev(g->G, e);
    return keep_at(g, info, ev, keep, n_kept);
}

// Smallest grid point j * 2^-40 (0 < j <= 2^40) whose kept count reaches K,
// per graph (the result of 40 halvings of [0, 1], because the kept count is
// monotone in e).  Each pass counts the kept set at 15 interior points of the
// current interval and its upper end; edges whose fate the chosen
// sub-interval already decides drop out of the next pass.
static ad_status select_per_node_fit_host(ad_graph_t g, const int4 *info, double fraction, uint8_t *keep,
                                          int64_t *n_kept, double *e_used) {
    ad_graph_s::SelCache *c = g->sel;
    const int32_t ndc = std::max<int32_t>(g->n_deg_classes, 1);
    const int ncand = 16;   // 15 interior points + the upper end
    const int64_t ONE = (int64_t)1 << 40;
    const int G = g->G;
    std::vector<int64_t> lo(G, 0), hi(G, ONE), K(G), base(G, 0);
    for (int32_t k = 0; k < G; ++k) K[k] = target_count(g->eoff_h[k + 1] - g->eoff_h[k], fraction);
    AD_TRY(ensure(g, c->T, (size_t)G * ncand * ndc * sizeof(int32_t)));
    AD_TRY(ensure(g, c->hist, (size_t)G * 32 * sizeof(unsigned long long)));
    AD_TRY(ensure(g, c->jsel, (size_t)(G + 1) * sizeof(int32_t)));
    AD_TRY(ensure(g, c->cstar, (size_t)(g->m + 1)));
    AD_TRY(ensure(g, c->flag, (size_t)(g->m + 1)));
    int32_t *T = static_cast<int32_t *>(c->T.ptr);
    unsigned long long *hist = static_cast<unsigned long long *>(c->hist.ptr);
    int32_t *jsel_d = static_cast<int32_t *>(c->jsel.ptr);
    uint8_t *cstar = static_cast<uint8_t *>(c->cstar.ptr), *flag = static_cast<uint8_t *>(c->flag.ptr);
    std::vector<int32_t> Th((size_t)G * ncand * ndc);
    std::vector<unsigned long long> hh((size_t)G * 32);
    std::vector<std::vector<int64_t>> cand(G);
    std::vector<int32_t> jsel(G + 1, -1);
    // T at the current interval ends (e = 0: every node keeps 1; e = 1: all of its edges).
    // T is monotone in e, so a class with equal values at both ends is constant inside.
    std::vector<int32_t> Tlo((size_t)G * ndc, 1), Thi((size_t)G * ndc, 0);
    for (int32_t k = 0; k < G; ++k)
        for (int32_t q = 0; q < g->n_deg_classes; ++q) Thi[(size_t)k * ndc + q] = (int32_t)g->distinct_degrees[q];
    const int64_t *list = nullptr;   // nullptr: all edges
    int64_t L = g->m;
    int64_t *owned_list = nullptr;
    for (;;) {
        bool any = false;
        for (int32_t k = 0; k < G; ++k) {
            cand[k].clear();
            const int64_t span = hi[k] - lo[k];
            if (span > 1) {
                any = true;
                const int64_t step = (span + 15) / 16;
                for (int64_t j = lo[k] + step; j < hi[k] && (int)cand[k].size() < ncand - 1; j += step) cand[k].push_back(j);
            }
            cand[k].push_back(hi[k]);
            const int32_t *tl = Tlo.data() + (size_t)k * ndc, *th = Thi.data() + (size_t)k * ndc;
            for (int cc = 0; cc < ncand; ++cc) {
                const int64_t j = cc < (int)cand[k].size() ? cand[k][cc] : hi[k];
                int32_t *out = Th.data() + ((size_t)k * ncand + cc) * ndc;
                if (j == hi[k]) {
                    for (int32_t q = 0; q < ndc; ++q) out[q] = th[q];
                    continue;
                }
                const double e = std::ldexp((double)j, -40);
                for (int32_t q = 0; q < g->n_deg_classes; ++q)
                    out[q] = tl[q] == th[q] ? tl[q] : (int32_t)degree_target(g->distinct_degrees[q], e);
            }
        }
        if (!any || L == 0) break;
        AD_TRY(copy_in(g, T, Th.data(), Th.size() * sizeof(int32_t)));
        AD_CUDA_TRY(cudaMemsetAsync(hist, 0, sizeof(unsigned long long) * G * 32, g->stream));
        const int blocks = (int)std::max<int64_t>(1, std::min<int64_t>((L + 255) / 256, (int64_t)g->num_sms * 16));
        AD_LAUNCH(k_count_cand, blocks, 256, 0, g->stream, info, list, L, (const int64_t *)nullptr, g->goff_e, G, T, ndc,
                  ncand, hist, cstar);
        AD_TRY(copy_out(g, hh.data(), hist, sizeof(unsigned long long) * hh.size()));
        for (int32_t k = 0; k < G; ++k) {
            if (hi[k] - lo[k] <= 1) { jsel[k] = -1; continue; }
            int64_t cum = base[k];
            int chosen = (int)cand[k].size() - 1;   // the upper end always reaches K
            for (int cc = 0; cc < (int)cand[k].size(); ++cc) {
                cum += (int64_t)hh[(size_t)k * 32 + cc];
                if (cum >= K[k]) { chosen = cc; break; }
            }
            // edges first kept before the chosen point stay kept in the new interval
            for (int cc = 0; cc < chosen; ++cc) base[k] += (int64_t)hh[(size_t)k * 32 + cc];
            if (chosen > 0) {
                const int32_t *src = Th.data() + ((size_t)k * ncand + chosen - 1) * ndc;
                std::copy(src, src + ndc, Tlo.begin() + (size_t)k * ndc);
            }
            {
                const int32_t *src = Th.data() + ((size_t)k * ncand + chosen) * ndc;
                std::copy(src, src + ndc, Thi.begin() + (size_t)k * ndc);
            }
            lo[k] = chosen > 0 ? cand[k][chosen - 1] : lo[k];
            hi[k] = cand[k][chosen];
            jsel[k] = chosen;
        }
        // next pass: the edges whose first kept point is the chosen one
        AD_TRY(copy_in(g, jsel_d, jsel.data(), (G + 1) * sizeof(int32_t)));
        const int fblocks = (int)std::max<int64_t>(1, std::min<int64_t>((L + 255) / 256, (int64_t)g->num_sms * 16));
        AD_LAUNCH(k_undecided_flags, fblocks, 256, 0, g->stream, list, L, cstar, g->goff_e, G, jsel_d, flag);
        int64_t *idx = nullptr, nL = 0;
        AD_TRY(compact_flags(g, flag, L, &idx, &nL));
        int64_t *next = nullptr;
        if (nL > 0) {
            AD_TRY(dalloc_t(g, nL, &next));
            AD_LAUNCH(k_gather_list, (int)((nL + 255) / 256), 256, 0, g->stream, list, idx, nL, next);
        }
        if (idx) dfree(g, idx);
        if (owned_list) dfree(g, owned_list);
        owned_list = next;
        list = next;
        L = nL;
    }
    if (owned_list) dfree(g, owned_list);
    // no undecided edge left: the count is constant on (lo, hi], so the first grid point reaches K
    for (int32_t k = 0; k < G; ++k)
        if (hi[k] - lo[k] > 1) hi[k] = lo[k] + 1;
    std::vector<double> ev(G);
    for (int32_t k = 0; k < G; ++k) ev[k] = std::ldexp((double)hi[k], -40);
    AD_TRY(keep_at(g, info, ev, keep, n_kept));
    if (e_used) *e_used = G > 0 ? ev[0] : -1.0;
    return AD_OK;
}

// The same search with every pass on the device; falls back to host tables
// when a device T(d, e) is too close to a rounding boundary to be trusted.
static ad_status fit_search(ad_graph_t g, const int4 *info, double fraction, uint8_t *keep, int64_t *n_kept,
                            double *e_used);

ad_status select_per_node_fit(ad_graph_t g, const float *score, double fraction, ad_mode mode, uint8_t *keep,
                              int64_t *n_kept, double *e_used) {
    int4 *info = nullptr;
    AD_TRY(per_node_info(g, score, mode, &info));
    return fit_search(g, info, fraction, keep, n_kept, e_used);
}

// Per-edge records (rank at each end, degree class of each end) from ranks
// given per CSR entry in `rank`, then the fit of e and the kept set: Alg. 2's
// union and search for any per-node selection order (SparsifyB's included).
ad_status select_per_node_fit_ranked(ad_graph_t g, const uint32_t *rank, double fraction, uint8_t *keep,
                                     int64_t *n_kept, double *e_used) {
    AD_TRY(ensure_mirror(g));
    AD_TRY(ensure_degree_classes(g));
    ad_graph_s::SelCache *c = nullptr;
    AD_TRY(sel_cache(g, &c));
    if (!c->epos) {
        AD_TRY(dalloc_t(g, g->m + 1, &c->epos));
        if (g->nnz > 0)
            AD_LAUNCH(k_edge_pos, g->num_sms * 16, 256, 0, g->stream, g->erow, g->col, g->eid, g->nnz, c->epos);
    }
    AD_TRY(ensure(g, c->info_other, 2 * sizeof(int4) * (g->m + 1)));
    int4 *info = static_cast<int4 *>(c->info_other.ptr);
    if (g->m > 0)   // the second output (the other order) is not needed: it goes to the spare half
        AD_LAUNCH(k_info, g->num_sms * 16, 256, 0, g->stream, c->epos, g->mirror, g->erow, g->col, g->deg_class, g->m,
                  rank, rank, info, info + (g->m + 1));
    return fit_search(g, info, fraction, keep, n_kept, e_used);
}

// key of entry (i, j) for Local Degree: larger degree of j first
__global__ void k_ld_keys(const int64_t *rp, const int32_t *col, int64_t nnz, uint32_t *ekey) {
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < nnz; p += (int64_t)gridDim.x * blockDim.x) {
        const int32_t j = col[p];
        ekey[p] = ~(uint32_t)(rp[j + 1] - rp[j]);
    }
}

// Local Degree (the comparison method of Sec. 1.1 and Sec. 6): node i takes the
// edges to its T(d_i, e) neighbours of largest degree (ties: smaller CSR
// position); union and fit of e as Alg. 2.
ad_status select_local_degree(ad_graph_t g, double fraction, uint8_t *keep, int64_t *n_kept, double *e_used) {
    AD_TRY(ensure_mirror(g));
    AD_TRY(ensure_degree_classes(g));
    ad_graph_s::SelCache *c = nullptr;
    AD_TRY(sel_cache(g, &c));
    AD_TRY(rank_lists(g, c));
    const int64_t nnz = g->nnz;
    AD_TRY(ensure(g, c->ekey, sizeof(uint32_t) * (nnz + 1)));
    AD_TRY(ensure(g, c->rank2, 2 * sizeof(uint32_t) * (nnz + 1)));
    uint32_t *ekey = static_cast<uint32_t *>(c->ekey.ptr);
    RankOut out;
    out.asc = static_cast<uint32_t *>(c->rank2.ptr);
    out.desc = out.asc + (nnz + 1);
    if (nnz > 0) AD_LAUNCH(k_ld_keys, g->num_sms * 16, 256, 0, g->stream, g->rp, g->col, nnz, ekey);
    AD_TRY(entry_ranks(g, c, ekey, out));
    return select_per_node_fit_ranked(g, out.asc, fraction, keep, n_kept, e_used);
}

// The exponent search of nsets * G problems at once: problem s * G + k is
// graph k ranked by the records at info + s * m (set s), its edges
// [s * m + goff_e[k], s * m + goff_e[k+1]).  ev receives the fitted e of every
// problem; *ambiguous is set when a table entry lay too close to an integer
// for the device pow to decide it (the caller then takes the host tables).
static ad_status fit_multi(ad_graph_t g, const int4 *info, int nsets, double fraction, std::vector<double> &ev,
                           bool *ambiguous) {
    ad_graph_s::SelCache *c = g->sel;
    const int G = g->G, P = nsets * G;
    const int64_t m = g->m, L0 = (int64_t)nsets * m;
    const int32_t ndc = std::max<int32_t>(g->n_deg_classes, 1);
    std::vector<FitState> sh(P);
    std::vector<int64_t> pgoff(P + 1);
    for (int sidx = 0; sidx < nsets; ++sidx)
        for (int32_t k = 0; k < G; ++k) {
            FitState &f = sh[sidx * G + k];
            f.lo = 0;
            f.hi = (int64_t)1 << 40;
            f.K = target_count(g->eoff_h[k + 1] - g->eoff_h[k], fraction);
            f.base = 0;
            f.jsel = -1;
            f.pad = 0;
            pgoff[sidx * G + k] = sidx * m + g->eoff_h[k];
        }
    pgoff[P] = L0;
    if (!c->have_ddeg) {
        AD_TRY(ensure(g, c->ddeg, sizeof(int64_t) * ndc));
        AD_TRY(copy_in(g, c->ddeg.ptr, g->distinct_degrees.data(), sizeof(int64_t) * g->n_deg_classes));
        c->have_ddeg = true;
    }
    const size_t tsz = (size_t)P * kFitCand * ndc, bsz = (size_t)P * ndc;
    AD_TRY(ensure(g, c->T, 2 * tsz * sizeof(int32_t)));
    AD_TRY(ensure(g, c->hist, (size_t)2 * P * 32 * sizeof(unsigned long long)));
    AD_TRY(ensure(g, c->cstar, (size_t)(L0 + 1)));
    AD_TRY(ensure(g, c->list_a, sizeof(int64_t) * (L0 + 1)));
    AD_TRY(ensure(g, c->list_b, sizeof(int64_t) * (L0 + 1)));
    AD_TRY(ensure(g, c->fit, 3 * sizeof(FitState) * P + 4 * sizeof(int64_t) + sizeof(int64_t) * (P + 1)));
    AD_TRY(ensure(g, c->fit_tb, 4 * bsz * sizeof(int32_t)));
    FitState *stb = static_cast<FitState *>(c->fit.ptr);          // [0], [1]: by pass parity; [2]: initial
    FitState *st[2] = {stb, stb + P};
    int64_t *len = reinterpret_cast<int64_t *>(stb + 3 * P);      // [0], [1]: list lengths; [2]: ambiguity flag
    int *amb = reinterpret_cast<int *>(len + 2);
    int64_t *goff = len + 4;
    int32_t *tb = static_cast<int32_t *>(c->fit_tb.ptr);
    int32_t *Tlo[2] = {tb, tb + bsz}, *Thi[2] = {tb + 2 * bsz, tb + 3 * bsz};
    int32_t *T[2] = {static_cast<int32_t *>(c->T.ptr), static_cast<int32_t *>(c->T.ptr) + tsz};
    unsigned long long *hist[2] = {static_cast<unsigned long long *>(c->hist.ptr),
                                   static_cast<unsigned long long *>(c->hist.ptr) + (size_t)P * 32};
    uint8_t *cstar = static_cast<uint8_t *>(c->cstar.ptr);
    int64_t *lists[2] = {static_cast<int64_t *>(c->list_a.ptr), static_cast<int64_t *>(c->list_b.ptr)};
    const int64_t *ddeg = static_cast<const int64_t *>(c->ddeg.ptr);
    AD_TRY(copy_in(g, stb + 2 * P, sh.data(), sizeof(FitState) * P));
    AD_TRY(copy_in(g, goff, pgoff.data(), sizeof(int64_t) * (P + 1)));
    AD_CUDA_TRY(cudaMemsetAsync(len, 0, 4 * sizeof(int64_t), g->stream));
    const int big = g->num_sms * 16;
    const int ablocks = (int)std::max<int64_t>(1, std::min<int64_t>(((int64_t)tsz + 255) / 256, big));
    const int cblocks = (int)std::max<int64_t>(1, std::min<int64_t>((L0 + 255) / 256, big));
    // initial state, ends and the tables of pass 0
    AD_LAUNCH(k_fit_advance, ablocks, 256, 0, g->stream, P, 1, 0, stb + 2 * P, st[0], hist[1], hist[0], T[1], T[0],
              Tlo[1], Thi[1], Tlo[0], Thi[0], ddeg, ndc, len + 1, amb);
    for (int pass = 0; pass < kFitPasses; ++pass) {
        const int a = pass & 1, b = a ^ 1;
        const bool last = pass + 1 == kFitPasses;
        AD_LAUNCH(k_count_cand, cblocks, 256, 0, g->stream, info, pass == 0 ? nullptr : lists[a], L0,
                  pass == 0 ? nullptr : len + a, goff, P, T[a], ndc, kFitCand, hist[a], cstar);
        AD_LAUNCH(k_fit_advance, ablocks, 256, 0, g->stream, P, 0, last ? 1 : 0, st[a], st[b], hist[a], hist[b], T[a],
                  T[b], Tlo[a], Thi[a], Tlo[b], Thi[b], ddeg, ndc, len + b, amb);
        if (!last)
            AD_LAUNCH(k_fit_compact, cblocks, 256, 0, g->stream, pass == 0 ? nullptr : lists[a], L0,
                      pass == 0 ? nullptr : len + a, cstar, goff, P, st[b], lists[b], len + b);
    }
    AD_TRY(copy_out(g, sh.data(), st[kFitPasses & 1], sizeof(FitState) * P));
    int amb_h = 0;
    AD_TRY(copy_out(g, &amb_h, amb, sizeof(int)));
    *ambiguous = amb_h != 0;
    ev.assign(P, -1.0);
    if (*ambiguous) return AD_OK;
    for (int k = 0; k < P; ++k) {
        if (sh[k].hi - sh[k].lo > 1) return fail(AD_ERR_CUDA, "exponent search did not converge");
        ev[k] = std::ldexp((double)sh[k].hi, -40);
    }
    return AD_OK;
}

static ad_status fit_search(ad_graph_t g, const int4 *info, double fraction, uint8_t *keep, int64_t *n_kept,
                            double *e_used) {
    if (g->m == 0 || g->n_deg_classes == 0) return select_per_node_fit_host(g, info, fraction, keep, n_kept, e_used);
    std::vector<double> ev;
    bool amb = false;
    AD_TRY(fit_multi(g, info, 1, fraction, ev, &amb));
    if (amb) return select_per_node_fit_host(g, info, fraction, keep, n_kept, e_used);
    AD_TRY(keep_at(g, info, ev, keep, n_kept));
    if (e_used) *e_used = g->G > 0 ? ev[0] : -1.0;
    return AD_OK;
}

// Alg. 2 in both orders (local: smallest rho first; global: largest first) on
// the same scores: one ranking pass, one two-set exponent search.
ad_status select_per_node_fit_both(ad_graph_t g, const float *score, double fraction, uint8_t *keep_local,
                                   uint8_t *keep_global, int64_t *n_kept, double *e_used) {
    int4 *info = nullptr;
    AD_TRY(per_node_info(g, score, AD_MODE_LOCAL, &info));   // the global records follow at info + m
    uint8_t *keep[2] = {keep_local, keep_global};
    if (g->m == 0 || g->n_deg_classes == 0) {
        for (int sidx = 0; sidx < 2; ++sidx)
            AD_TRY(select_per_node_fit_host(g, info + sidx * g->m, fraction, keep[sidx], n_kept + sidx, e_used + sidx));
        return AD_OK;
    }
    std::vector<double> ev;
    bool amb = false;
    AD_TRY(fit_multi(g, info, 2, fraction, ev, &amb));
    for (int sidx = 0; sidx < 2; ++sidx) {
        const int4 *inf = info + sidx * g->m;
        if (amb) {
            AD_TRY(select_per_node_fit_host(g, inf, fraction, keep[sidx], n_kept + sidx, e_used + sidx));
            continue;
        }
        std::vector<double> es(ev.begin() + sidx * g->G, ev.begin() + (sidx + 1) * g->G);
        AD_TRY(keep_at(g, inf, es, keep[sidx], n_kept + sidx));
        e_used[sidx] = g->G > 0 ? es[0] : -1.0;
    }
    return AD_OK;
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
static int g_noalloc_sms[kNoAllocMaxDevices] = {};

// Device address of the scratch array on the current device and its SM count
// (looked up once per device).
static ad_status noalloc_scratch(NoAllocScratch **out, int *num_sms) {
    int dev = 0;
    AD_CUDA_TRY(cudaGetDevice(&dev));
    if (dev < 0 || dev >= kNoAllocMaxDevices) return fail(AD_ERR_INVALID_ARG, "device id out of range");
    std::lock_guard<std::mutex> lk(g_noalloc_mu);
    if (!g_noalloc_ptr[dev]) {
        void *p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || !p)
            return fail(AD_ERR_CUDA, std::string("cudaGetSymbolAddress(scratch): ") + cudaGetErrorString(e));
        int sms = 0;
        AD_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
        g_noalloc_sms[dev] = sms > 0 ? sms : kNumSMs;
        g_noalloc_ptr[dev] = static_cast<NoAllocScratch *>(p);
    }
    *out = g_noalloc_ptr[dev];
    *num_sms = g_noalloc_sms[dev];
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
    int num_sms = kNumSMs;
    AD_TRY(noalloc_scratch(&s, &num_sms));
    const int64_t K = target_count(m, fraction);
    if (m == 0) {
        if (n_kept) *n_kept = K;
        return AD_OK;
    }
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const int desc = mode == AD_MODE_GLOBAL ? 1 : 0;
    const int64_t ntiles = (m + kTile - 1) / kTile;
    AD_LAUNCH(k_noalloc_init, 64, 256, 0, st, s, m, K, ntiles);
    AD_LAUNCH(k_check_scores, num_sms * 8, 256, 0, st, score, m, &s->bad);
    unsigned long long bad = 0;
    AD_CUDA_TRY(cudaMemcpyAsync(&bad, &s->bad, sizeof(bad), cudaMemcpyDeviceToHost, st));
    AD_CUDA_TRY(cudaStreamSynchronize(st));
    if (bad != ~0ull) return fail(AD_ERR_INVALID_ARG, "score " + std::to_string(bad) + " is negative or not finite");
    if (n_kept) *n_kept = K;
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
