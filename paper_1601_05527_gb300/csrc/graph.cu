// graph.cu -- graph set-up on the device: validation of the CSR (Sec. 2:
// undirected, positive weights, no self loops or multi-edges), weighted
// degrees in FP64, the upper-triangle edge numbering, and the task plans of
// the row-parallel kernels.
#include "ad_internal.cuh"

#include <algorithm>
#include <climits>
#include <cstring>

namespace ad {

// ----------------------------------------------------------------------------
// Exclusive scan of int64 (three phases: block sums, scan of sums, add back).
// ----------------------------------------------------------------------------
constexpr int kScanThreads = 512;
constexpr int kScanItems = 8;
constexpr int kScanTile = kScanThreads * kScanItems;

__device__ __forceinline__ int64_t block_exclusive_scan(int64_t v, int64_t *sh, int64_t *total) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    int64_t x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        int64_t y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) sh[warp] = x;
    __syncthreads();
    if (warp == 0) {
        int64_t s = lane < nw ? sh[lane] : 0;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            int64_t y = __shfl_up_sync(0xffffffffu, s, o);
            if (lane >= o) s += y;
        }
        if (lane < nw) sh[lane] = s;
    }
    __syncthreads();
    const int64_t warp_prefix = warp > 0 ? sh[warp - 1] : 0;
    if (total) *total = sh[nw - 1];
    __syncthreads();
    return warp_prefix + x - v;
}

__global__ void k_scan_tiles(const int64_t *in, int64_t *out, int64_t n, int64_t *tile_sums) {
    __shared__ int64_t sh[32];
    const int64_t base = (int64_t)blockIdx.x * kScanTile + (int64_t)threadIdx.x * kScanItems;
    int64_t v[kScanItems], s = 0;
#pragma unroll
    for (int k = 0; k < kScanItems; ++k) {
        v[k] = (base + k < n) ? in[base + k] : 0;
        s += v[k];
    }
    int64_t tot;
    int64_t pre = block_exclusive_scan(s, sh, &tot);
#pragma unroll
    for (int k = 0; k < kScanItems; ++k) {
        if (base + k < n) out[base + k] = pre;
        pre += v[k];
    }
    if (threadIdx.x == 0 && tile_sums) tile_sums[blockIdx.x] = tot;
}

__global__ void k_scan_add(int64_t *out, int64_t n, const int64_t *tile_prefix) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] += tile_prefix[i / kScanTile];
}

// Scan of n values with the tile sums of every level carved from ws.
static ad_status scan_rec(ad_graph_t g, const int64_t *in, int64_t *out, int64_t n, int64_t *ws) {
    const int64_t tiles = (n + kScanTile - 1) / kScanTile;
    int64_t *sums = ws, *pref = ws + tiles + 1;
    AD_LAUNCH(k_scan_tiles, (int)tiles, kScanThreads, 0, g->stream, in, out, n, sums);
    if (tiles > 1) {
        AD_TRY(scan_rec(g, sums, pref, tiles, ws + 2 * (tiles + 1)));
        AD_LAUNCH(k_scan_add, (int)((n + 255) / 256), 256, 0, g->stream, out, n, pref);
    }
    return AD_OK;
}

// out[0..n) = exclusive scan of in; *total_host (optional) = sum (synchronises).
// Scratch comes from a workspace cached in the handle.
ad_status exclusive_scan_i64(ad_graph_t g, const int64_t *in, int64_t *out, int64_t n, int64_t *total_host) {
    if (n <= 0) {
        if (total_host) *total_host = 0;
        return AD_OK;
    }
    size_t words = 0;
    for (int64_t len = n; len > 1; len = (len + kScanTile - 1) / kScanTile) words += 2 * ((len + kScanTile - 1) / kScanTile + 1);
    words += 4;
    AD_TRY(ensure(g, g->scan_ws, words * sizeof(int64_t)));
    AD_TRY(scan_rec(g, in, out, n, static_cast<int64_t *>(g->scan_ws.ptr)));
    if (total_host) {
        int64_t last_in = 0, last_out = 0;
        AD_TRY(copy_out(g, &last_in, in + n - 1, sizeof(int64_t)));
        AD_TRY(copy_out(g, &last_out, out + n - 1, sizeof(int64_t)));
        *total_host = last_in + last_out;
    }
    return AD_OK;
}

// ----------------------------------------------------------------------------
// Validation.  err = min over violations of (priority << 56 | position), so
// that a structural fault is reported before the asymmetries it causes.
// ----------------------------------------------------------------------------
enum : int { P_CSR = 0, P_SELF = 1, P_DUP = 2, P_WEIGHT = 3, P_BATCH = 4, P_SYM = 5 };
static const ad_status kPrioCode[] = {AD_ERR_BAD_CSR, AD_ERR_SELF_LOOP, AD_ERR_DUPLICATE_EDGE, AD_ERR_BAD_WEIGHT,
                                      AD_ERR_INVALID_ARG, AD_ERR_NOT_SYMMETRIC};
static const char *kPrioText[] = {"row_ptr / col out of range", "self loop", "unsorted or repeated column",
                                  "weight not positive and finite", "edge joins two graphs of the batch",
                                  "entry without its mirror, or unequal mirrored weights"};

__device__ __forceinline__ void report(unsigned long long *err, int prio, int64_t pos) {
    atomicMin(err, ((unsigned long long)prio << 56) | (unsigned long long)(pos & 0x00ffffffffffffffLL));
}

__global__ void k_check_rows(const int64_t *rp, int64_t n, int64_t nnz, unsigned long long *err) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i <= n; i += (int64_t)gridDim.x * blockDim.x) {
        if (i == 0 && rp[0] != 0) report(err, P_CSR, 0);
        if (i == n && rp[n] != nnz) report(err, P_CSR, n);
        if (i < n && rp[i + 1] < rp[i]) report(err, P_CSR, i);
    }
}

__device__ __forceinline__ int64_t find_in_row(const int64_t *rp, const int32_t *col, int64_t r, int32_t c) {
    int64_t lo = rp[r], hi = rp[r + 1];
    while (lo < hi) {
        const int64_t mid = (lo + hi) >> 1;
        if (col[mid] < c) lo = mid + 1; else hi = mid;
    }
    return (lo < rp[r + 1] && col[lo] == c) ? lo : -1;
}

__global__ void k_entry_rows(const int64_t *rp, int64_t n, int32_t *erow);

// one thread per entry (row ids from k_entry_rows); records the mirror position
// of every entry on the way, which the selection and the multilevel code reuse
__global__ void k_check_entries(const int64_t *rp, const int32_t *col, const float *w, const int32_t *erow, int64_t n,
                                int64_t nnz, const int64_t *voff, int32_t G, unsigned long long *err,
                                int64_t *mirror) {
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < nnz; p += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = erow[p];
        const int32_t j = col[p];
        mirror[p] = -1;
        if (j < 0 || j >= n) { report(err, P_CSR, p); continue; }
        if (j == i) { report(err, P_SELF, p); continue; }
        if (p > rp[i] && col[p - 1] >= j) { report(err, P_DUP, p); continue; }
        if (w) {
            const float x = w[p];
            if (!(x > 0.f) || !isfinite(x)) { report(err, P_WEIGHT, p); continue; }
        }
        if (G > 1) {   // both ends in one graph of the batch
            int lo = 0, hi = G;
            while (hi - lo > 1) { int mid = (lo + hi) >> 1; if (voff[mid] <= i) lo = mid; else hi = mid; }
            if (j < voff[lo] || j >= voff[lo + 1]) { report(err, P_BATCH, p); continue; }
        }
        const int64_t q = find_in_row(rp, col, j, (int32_t)i);
        if (q < 0) { report(err, P_SYM, p); continue; }
        if (w && __float_as_uint(w[q]) != __float_as_uint(w[p])) report(err, P_SYM, p);
        mirror[p] = q;
    }
}

// Fast validation pass over valid-looking input: the same per-entry checks, but
// each undirected pair is looked up once -- by the entry of the longer row
// (equal lengths: of the larger row id), in the shorter row -- and that thread
// records both mirror positions.  Found partners are distinct entries of the
// other kind, so with no violation reported, 2 * pairs == nnz means every entry
// has its mirror; otherwise the caller reruns k_check_entries for the report.
__global__ void k_check_pairs(const int64_t *rp, const int32_t *col, const float *w, const int32_t *erow, int64_t n,
                              int64_t nnz, const int64_t *voff, int32_t G, unsigned long long *err,
                              unsigned long long *pairs, int64_t *mirror) {
    unsigned long long found = 0;
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < nnz; p += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = erow[p];
        const int32_t j = col[p];
        if (j < 0 || j >= n) { report(err, P_CSR, p); continue; }
        if (j == i) { report(err, P_SELF, p); continue; }
        if (p > rp[i] && col[p - 1] >= j) { report(err, P_DUP, p); continue; }
        if (w) {
            const float x = w[p];
            if (!(x > 0.f) || !isfinite(x)) { report(err, P_WEIGHT, p); continue; }
        }
        if (G > 1) {
            int lo = 0, hi = G;
            while (hi - lo > 1) { int mid = (lo + hi) >> 1; if (voff[mid] <= i) lo = mid; else hi = mid; }
            if (j < voff[lo] || j >= voff[lo + 1]) { report(err, P_BATCH, p); continue; }
        }
        const int64_t di = rp[i + 1] - rp[i], dj = rp[j + 1] - rp[j];
        if (!(dj < di || (dj == di && j < i))) continue;     // the pair's other entry looks it up
        const int64_t q = find_in_row(rp, col, j, (int32_t)i);
        if (q < 0) { report(err, P_SYM, p); continue; }
        if (w && __float_as_uint(w[q]) != __float_as_uint(w[p])) report(err, P_SYM, p < q ? p : q);
        mirror[p] = q;
        mirror[q] = p;
        ++found;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) found += __shfl_xor_sync(0xffffffffu, found, o);
    if ((threadIdx.x & 31) == 0 && found) atomicAdd(pairs, found);
}

// ----------------------------------------------------------------------------
// Degrees and edge numbering
// ----------------------------------------------------------------------------
// First upper entry of every row (rows are sorted), and D, D^-1 for unit
// weights: one thread per row, so that the binary searches of many rows are in
// flight at once.
__global__ void k_degrees(const int64_t *rp, const int32_t *col, const float *w, int64_t n, double *D, float *Dinv,
                          int64_t *upos, int64_t *ucount) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t b = rp[i], e = rp[i + 1];
        int64_t lo = b, hi = e;   // first position with col > i
        while (lo < hi) {
            const int64_t mid = (lo + hi) >> 1;
            if (col[mid] <= i) lo = mid + 1; else hi = mid;
        }
        upos[i] = lo;
        ucount[i] = e - lo;
        if (!w) {
            const double s = (double)(e - b);
            D[i] = s;
            Dinv[i] = s > 0.0 ? (float)(1.0 / s) : 0.f;
        }
    }
}

// weighted degrees D_i = sum_j w_ij in FP64: a warp per row, lanes strided over
// the row.  When the row's weights span few enough binary orders of magnitude,
// every partial sum of them is an exact FP64 number -- the weights are
// multiples of the smallest weight's unit in the last place, and d of them stay
// below 2^(largest exponent + 1 + ceil log2 d) -- so any summation order gives
// the same bits as summing one after the other in CSR order.  Rows where that
// bound does not hold are summed one entry after the other in CSR order by one
// lane.  exact_out[i] records which case row i is (the seed rule relies on it).
__device__ __forceinline__ int fp32_biased_exponent(float v) { return (int)((__float_as_uint(v) >> 23) & 0xffu); }

__global__ void k_wdegrees(const int64_t *rp, const float *w, int64_t n, double *D, float *Dinv, uint8_t *exact_out) {
    const int lane = threadIdx.x & 31;
    const int64_t W = (int64_t)gridDim.x * (blockDim.x >> 5);
    for (int64_t i = blockIdx.x * (int64_t)(blockDim.x >> 5) + (threadIdx.x >> 5); i < n; i += W) {
        const int64_t b = rp[i], e = rp[i + 1];
        double s0 = 0.0, s1 = 0.0, s2 = 0.0, s3 = 0.0;   // four independent loads in flight per lane
        int emax = 0, emin = 255;
        int64_t p = b + lane;
        for (; p + 96 < e; p += 128) {
            const float w0 = w[p], w1 = w[p + 32], w2 = w[p + 64], w3 = w[p + 96];
            s0 += (double)w0;
            s1 += (double)w1;
            s2 += (double)w2;
            s3 += (double)w3;
            emax = max(emax, max(max(fp32_biased_exponent(w0), fp32_biased_exponent(w1)),
                                 max(fp32_biased_exponent(w2), fp32_biased_exponent(w3))));
            emin = min(emin, min(min(fp32_biased_exponent(w0), fp32_biased_exponent(w1)),
                                 min(fp32_biased_exponent(w2), fp32_biased_exponent(w3))));
        }
        for (; p < e; p += 32) {
            const float w0 = w[p];
            s0 += (double)w0;
            emax = max(emax, fp32_biased_exponent(w0));
            emin = min(emin, fp32_biased_exponent(w0));
        }
        double s = (s0 + s1) + (s2 + s3);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            s += __shfl_xor_sync(0xffffffffu, s, o);
            emax = max(emax, __shfl_xor_sync(0xffffffffu, emax, o));
            emin = min(emin, __shfl_xor_sync(0xffffffffu, emin, o));
        }
        int lg = 0;
        while (((int64_t)1 << lg) < e - b) ++lg;   // ceil(log2 d)
        // bits spanned by every partial sum: (emax - 127 + 1 + lg) - (max(emin, 1) - 150)
        const bool exact = e == b || emax - max(emin, 1) + lg + 24 <= 53;
        if (lane == 0) {
            if (!exact) {   // the plain definition's order, one entry after the other
                s = 0.0;
                for (int64_t q = b; q < e; ++q) s += (double)w[q];
            }
            D[i] = s;
            Dinv[i] = s > 0.0 ? (float)(1.0 / s) : 0.f;
            exact_out[i] = exact ? 1 : 0;
        }
    }
}

// row of every entry (stores only, so a warp per row is cheap even for hubs)
__global__ void k_entry_rows(const int64_t *rp, int64_t n, int32_t *erow) {
    const int lane = threadIdx.x & 31;
    const int64_t W = (int64_t)gridDim.x * (blockDim.x >> 5);
    // 32 rows per warp and round: their bounds are loaded at once, then written row by row
    for (int64_t base = (blockIdx.x * (int64_t)(blockDim.x >> 5) + (threadIdx.x >> 5)) * 32; base < n; base += W * 32) {
        const int64_t i = base + lane;
        const long long b = i < n ? rp[i] : 0, e = i < n ? rp[i + 1] : 0;
        for (int r = 0; r < 32; ++r) {
            const long long br = __shfl_sync(0xffffffffu, b, r), er = __shfl_sync(0xffffffffu, e, r);
            for (long long p = br + lane; p < er; p += 32) erow[p] = (int32_t)(base + r);
        }
    }
}

// Position of the reverse entry of every entry (mirror preset to -1): each
// undirected pair is looked up once, by binary search in the shorter of its
// two rows (equal lengths: from the larger row id), and both positions are
// recorded.  An entry whose pair is missing (unvalidated asymmetric input)
// keeps -1.
__global__ void k_mirror(const int64_t *rp, const int32_t *col, const int32_t *erow, int64_t nnz, int64_t *mirror) {
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < nnz; p += (int64_t)gridDim.x * blockDim.x) {
        const int32_t i = erow[p], j = col[p];
        const int64_t di = rp[i + 1] - rp[i], dj = rp[j + 1] - rp[j];
        if (!(dj < di || (dj == di && j < i))) continue;     // the pair's other entry looks it up
        const int64_t q = find_in_row(rp, col, j, i);
        if (q < 0) continue;
        mirror[p] = q;
        mirror[q] = p;
    }
}

// one thread per entry: the id of its edge (upper entries numbered row-major)
__global__ void k_entry_eids(const int32_t *col, const int32_t *erow, const int64_t *upos, const int64_t *eoff,
                             const int64_t *mirror, int64_t nnz, int64_t *eid) {
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < nnz; p += (int64_t)gridDim.x * blockDim.x) {
        const int32_t i = erow[p], j = col[p];
        if (j > i) { eid[p] = eoff[i] + (p - upos[i]); continue; }
        const int64_t q = mirror[p];   // -1 only for unvalidated asymmetric input
        eid[p] = q >= 0 ? eoff[j] + (q - upos[j]) : eoff[i];
    }
}

// anchor of each graph: the vertex of largest weighted degree, ties to the smaller id
__global__ void k_anchor_max(const double *D, const int64_t *voff, int G, int64_t n, unsigned long long *best) {
    unsigned long long mine = 0;   // D >= 0: bit patterns order like the values
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const unsigned long long b = (unsigned long long)__double_as_longlong(D[i]);
        if (G > 1) {
            int lo = 0, hi = G;
            while (hi - lo > 1) { int mid = (lo + hi) >> 1; if (voff[mid] <= i) lo = mid; else hi = mid; }
            atomicMax(best + lo, b);
        } else if (b > mine) {
            mine = b;
        }
    }
    if (G == 1) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) mine = max(mine, __shfl_xor_sync(0xffffffffu, mine, o));
        if ((threadIdx.x & 31) == 0 && mine) atomicMax(best, mine);
    }
}
__global__ void k_anchor_pick(const double *D, const int64_t *voff, int G, int64_t n, const unsigned long long *best,
                              int32_t *anchor) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        int g = 0;
        if (G > 1) { int lo = 0, hi = G; while (hi - lo > 1) { int mid = (lo + hi) >> 1; if (voff[mid] <= i) lo = mid; else hi = mid; } g = lo; }
        if ((unsigned long long)__double_as_longlong(D[i]) == best[g]) atomicMin(anchor + g, (int32_t)i);
    }
}

static ad_status compute_anchors(ad_graph_t g) {
    if (!g->anchor) AD_TRY(dalloc_t(g, g->G + 1, &g->anchor));
    // non-empty graphs start at INT32_MAX and take the smallest id of maximum D;
    // an empty graph keeps its first id (no kernel reads it)
    std::vector<int32_t> init(g->G + 1, 0);
    for (int32_t k = 0; k < g->G; ++k)
        init[k] = g->voff_h[k + 1] > g->voff_h[k] ? INT32_MAX : (int32_t)std::min<int64_t>(g->voff_h[k], INT32_MAX);
    AD_TRY(copy_in(g, g->anchor, init.data(), (g->G + 1) * sizeof(int32_t)));
    if (g->n > 0) {
        unsigned long long *best = nullptr;
        AD_TRY(dalloc_t(g, g->G + 1, &best));
        AD_CUDA_TRY(cudaMemsetAsync(best, 0, (g->G + 1) * sizeof(unsigned long long), g->stream));
        AD_LAUNCH(k_anchor_max, g->num_sms * 8, 256, 0, g->stream, g->D, g->voff, g->G, g->n, best);
        AD_LAUNCH(k_anchor_pick, g->num_sms * 8, 256, 0, g->stream, g->D, g->voff, g->G, g->n, best, g->anchor);
        AD_CUDA_TRY(cudaStreamSynchronize(g->stream));
        dfree(g, best);
    }
    return AD_OK;
}

ad_status recompute_degrees(ad_graph_t g) {
    int64_t *ucount = nullptr;
    AD_TRY(dalloc_t(g, g->n + 1, &ucount));
    const int64_t tblocks = std::min<int64_t>((g->n + 255) / 256 + 1, (int64_t)g->num_sms * 16);
    AD_LAUNCH(k_degrees, (int)tblocks, 256, 0, g->stream, g->rp, g->col, g->w, g->n, g->D, g->Dinv, g->upos,
              ucount);
    if (g->w) {
        const int64_t wblocks = std::min<int64_t>((g->n + 7) / 8 + 1, (int64_t)g->num_sms * 64);
        if (!g->dexact) AD_TRY(dalloc_t(g, g->n + 1, &g->dexact));
        AD_LAUNCH(k_wdegrees, (int)wblocks, 256, 0, g->stream, g->rp, g->w, g->n, g->D, g->Dinv, g->dexact);
    }
    int64_t m = 0;
    ad_status st = exclusive_scan_i64(g, ucount, g->eoff, g->n, &m);
    dfree(g, ucount);
    AD_TRY(st);
    AD_CUDA_TRY(cudaMemcpyAsync(g->eoff + g->n, &m, sizeof(int64_t), cudaMemcpyHostToDevice, g->stream));
    AD_CUDA_TRY(cudaStreamSynchronize(g->stream));
    g->m = m;
    return compute_anchors(g);
}

__global__ void k_count_active(const int64_t *rp, int64_t n, unsigned long long *cnt) {
    unsigned long long c = 0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        c += (rp[i + 1] > rp[i]) ? 1 : 0;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
    if ((threadIdx.x & 31) == 0 && c) atomicAdd(cnt, c);
}

// out[k] = src[idx[k]] (idx[k] >= limit: fill); a handful of values read back with one copy
__global__ void k_pick_i64(const int64_t *src, const int64_t *idx, int64_t count, int64_t limit, int64_t fill,
                           int64_t *out) {
    const int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (k < count) out[k] = idx[k] < limit ? src[idx[k]] : fill;
}

ad_status graph_setup(ad_graph_t g, int32_t flags) {
    const int64_t n = g->n;
    unsigned long long *err = nullptr;   // [0] first violation, [1] active rows, [2] pairs found
    AD_TRY(dalloc_t(g, 3, &err));
    AD_CUDA_TRY(cudaMemsetAsync(err, 0xff, sizeof(unsigned long long), g->stream));
    AD_CUDA_TRY(cudaMemsetAsync(err + 1, 0, 2 * sizeof(unsigned long long), g->stream));
    const int grid = g->num_sms * 8;
    if (!(flags & AD_CREATE_SKIP_VALIDATION)) {
        AD_LAUNCH(k_check_rows, grid, 256, 0, g->stream, g->rp, n, g->nnz, err);
        unsigned long long e0 = 0;
        AD_TRY(copy_out(g, &e0, err, sizeof(e0)));
        if (e0 == ~0ull && g->nnz > 0) {   // row pointers are sound: row ids, then the entries
            AD_TRY(dalloc_t(g, g->nnz, &g->erow));
            AD_TRY(dalloc_t(g, g->nnz, &g->mirror));
            const int64_t wblocks = std::min<int64_t>((n + 255) / 256 + 1, (int64_t)g->num_sms * 16);
            AD_LAUNCH(k_entry_rows, (int)wblocks, 256, 0, g->stream, g->rp, n, g->erow);
            AD_LAUNCH(k_check_pairs, g->num_sms * 16, 256, 0, g->stream, g->rp, g->col, g->w, g->erow, n, g->nnz,
                      g->voff, g->G, err, err + 2, g->mirror);
            unsigned long long fast[3] = {0, 0, 0};
            AD_TRY(copy_out(g, fast, err, sizeof(fast)));
            if (fast[0] != ~0ull || 2 * fast[2] != (unsigned long long)g->nnz) {
                // a violation: the per-entry pass reports the first one by priority and position
                AD_CUDA_TRY(cudaMemsetAsync(err, 0xff, sizeof(unsigned long long), g->stream));
                AD_LAUNCH(k_check_entries, g->num_sms * 16, 256, 0, g->stream, g->rp, g->col, g->w, g->erow, n,
                          g->nnz, g->voff, g->G, err, g->mirror);
            }
        }
        AD_TRY(copy_out(g, &e0, err, sizeof(e0)));
        if (e0 != ~0ull) {
            const int prio = (int)(e0 >> 56);
            const long long pos = (long long)(e0 & 0x00ffffffffffffffULL);
            dfree(g, err);
            return fail(kPrioCode[prio], std::string("invalid graph: ") + kPrioText[prio] + " at " +
                                             (prio == P_CSR ? "index " : "CSR entry ") + std::to_string(pos));
        }
    }
    AD_LAUNCH(k_count_active, grid, 256, 0, g->stream, g->rp, n, err + 1);
    unsigned long long na = 0;
    AD_TRY(copy_out(g, &na, err + 1, sizeof(na)));
    g->n_active = (int64_t)na;
    dfree(g, err);
    AD_TRY(dalloc_t(g, n + 1, &g->D));
    AD_TRY(dalloc_t(g, n + 1, &g->Dinv));
    AD_TRY(dalloc_t(g, n + 1, &g->upos));
    AD_TRY(dalloc_t(g, n + 1, &g->eoff));
    AD_TRY(recompute_degrees(g));
    // per-graph edge offsets: the edge numbering at each graph's first vertex
    g->eoff_h.assign(g->G + 1, 0);
    AD_TRY(dalloc_t(g, g->G + 1, &g->goff_e));
    AD_LAUNCH(k_pick_i64, (g->G + 1 + 255) / 256, 256, 0, g->stream, g->eoff, g->voff, (int64_t)(g->G + 1), n, g->m,
              g->goff_e);
    AD_TRY(copy_out(g, g->eoff_h.data(), g->goff_e, sizeof(int64_t) * (g->G + 1)));
    return AD_OK;
}

ad_status ensure_mirror(ad_graph_t g) {
    if (g->eid || g->nnz == 0) return AD_OK;
    const int grid = g->num_sms * 16;
    if (!g->mirror) {   // not recorded by validation (handles created without it)
        AD_TRY(dalloc_t(g, g->nnz, &g->erow));
        AD_TRY(dalloc_t(g, g->nnz, &g->mirror));
        const int64_t wblocks = std::min<int64_t>((g->n + 255) / 256 + 1, (int64_t)g->num_sms * 16);
        AD_LAUNCH(k_entry_rows, (int)wblocks, 256, 0, g->stream, g->rp, g->n, g->erow);
        AD_CUDA_TRY(cudaMemsetAsync(g->mirror, 0xff, g->nnz * sizeof(int64_t), g->stream));
        AD_LAUNCH(k_mirror, grid, 256, 0, g->stream, g->rp, g->col, g->erow, g->nnz, g->mirror);
    }
    AD_TRY(dalloc_t(g, g->nnz, &g->eid));
    AD_LAUNCH(k_entry_eids, grid, 256, 0, g->stream, g->col, g->erow, g->upos, g->eoff, g->mirror, g->nnz, g->eid);
    return AD_OK;
}

// ----------------------------------------------------------------------------
// Stable multiway partition of rows by class (< 32 classes): per-tile class
// counts, a class-major exclusive scan, then an order-preserving scatter.
// ----------------------------------------------------------------------------
constexpr int kPartThreads = 256;
constexpr int kClasses = 32;

__global__ void k_class_counts(const int8_t *cls, int64_t n, int64_t *counts /* [kClasses][tiles] */, int64_t tiles) {
    __shared__ int c[kClasses];
    if (threadIdx.x < kClasses) c[threadIdx.x] = 0;
    __syncthreads();
    const int64_t i = (int64_t)blockIdx.x * kPartThreads + threadIdx.x;
    if (i < n && cls[i] >= 0) atomicAdd(&c[cls[i]], 1);
    __syncthreads();
    if (threadIdx.x < kClasses) counts[threadIdx.x * tiles + blockIdx.x] = c[threadIdx.x];
}

__global__ void k_class_scatter(const int8_t *cls, int64_t n, const int64_t *offsets /* [kClasses][tiles] */,
                                int64_t tiles, int32_t *out) {
    __shared__ int warp_cnt[kClasses][kPartThreads / 32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int64_t i = (int64_t)blockIdx.x * kPartThreads + threadIdx.x;
    const int c = (i < n) ? cls[i] : -1;
    int rank_in_warp = 0;
    for (int k = 0; k < kClasses; ++k) {
        const unsigned b = __ballot_sync(0xffffffffu, c == k);
        if (c == k) rank_in_warp = __popc(b & ((1u << lane) - 1u));
        if (lane == 0) warp_cnt[k][warp] = __popc(b);
    }
    __syncthreads();
    if (c >= 0) {
        int before = 0;
        for (int w2 = 0; w2 < warp; ++w2) before += warp_cnt[c][w2];
        out[offsets[c * tiles + blockIdx.x] + before + rank_in_warp] = (int32_t)i;
    }
}

// Stable partition of rows 0..n-1 by cls[i] in [0, nclasses) (negative: left
// out): order lists the rows class by class, by increasing id inside a class;
// start[c] is the first slot of class c, start[nclasses] the number of rows kept.
ad_status partition_by_class(ad_graph_t g, const int8_t *cls, int64_t n, int nclasses, int32_t *order,
                             std::vector<int64_t> &start) {
    start.assign(nclasses + 1, 0);
    if (n == 0) return AD_OK;
    if (nclasses > kClasses) return fail(AD_ERR_INVALID_ARG, "too many classes");
    const int64_t tiles = (n + kPartThreads - 1) / kPartThreads;
    int64_t *counts = nullptr, *offs = nullptr, *at_d = nullptr, *picked = nullptr;
    AD_TRY(dalloc_t(g, (size_t)kClasses * tiles, &counts));
    AD_TRY(dalloc_t(g, (size_t)kClasses * tiles, &offs));
    AD_LAUNCH(k_class_counts, (int)tiles, kPartThreads, 0, g->stream, cls, n, counts, tiles);
    int64_t total = 0;
    AD_TRY(exclusive_scan_i64(g, counts, offs, (int64_t)kClasses * tiles, &total));
    AD_LAUNCH(k_class_scatter, (int)tiles, kPartThreads, 0, g->stream, cls, n, offs, tiles, order);
    std::vector<int64_t> at(nclasses);
    for (int c = 0; c < nclasses; ++c) at[c] = (int64_t)c * tiles;
    AD_TRY(dalloc_t(g, nclasses, &at_d));
    AD_TRY(dalloc_t(g, nclasses, &picked));
    AD_TRY(copy_in(g, at_d, at.data(), nclasses * sizeof(int64_t)));
    AD_LAUNCH(k_pick_i64, 1, kClasses, 0, g->stream, offs, at_d, (int64_t)nclasses, (int64_t)kClasses * tiles, total,
              picked);
    AD_TRY(copy_out(g, start.data(), picked, nclasses * sizeof(int64_t)));
    start[nclasses] = total;
    for (void *p : {(void *)counts, (void *)offs, (void *)at_d, (void *)picked}) dfree(g, p);
    return AD_OK;
}

// Class of a row for a plan: -1 inactive, 0 big, 1..10 medium by decreasing
// log2 degree, 11 small.
__global__ void k_row_class(const int64_t *rp, const int64_t *upos, int64_t n, int small_max, int upper,
                            int8_t *cls, int64_t *nchunks) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t d = rp[i + 1] - (upper ? upos[i] : rp[i]);
        int8_t c;
        int64_t ch = 0;
        if (d <= 0) c = -1;
        else if (d > kBig) { c = 0; ch = (d + kChunk - 1) / kChunk; }
        else if (d <= small_max) c = 11;
        else {
            const int lg = 63 - __clzll((unsigned long long)d);   // floor(log2 d) in [0, 9]
            c = (int8_t)(10 - lg);
        }
        cls[i] = c;
        nchunks[i] = ch;
    }
}

__global__ void k_expand_chunks(const int32_t *big_rows, int64_t nb, const int64_t *rp, const int64_t *upos, int upper,
                                const int64_t *first, int32_t *big_row, int32_t *big_chunk) {
    const int lane = threadIdx.x & 31;
    const int64_t W = (int64_t)gridDim.x * (blockDim.x >> 5);
    for (int64_t b = blockIdx.x * (int64_t)(blockDim.x >> 5) + (threadIdx.x >> 5); b < nb; b += W) {
        const int32_t r = big_rows[b];
        const int64_t d = rp[r + 1] - (upper ? upos[r] : rp[r]);
        const int64_t nc = (d + kChunk - 1) / kChunk;
        for (int64_t c = lane; c < nc; c += 32) {
            big_row[first[b] + c] = r;
            big_chunk[first[b] + c] = (int32_t)c;
        }
    }
}

__global__ void k_gather_i64(const int64_t *src, const int32_t *idx, int64_t n, int64_t *dst) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) dst[i] = src[idx[i]];
}

ad_status build_row_plan(ad_graph_t g, int groups, int small_max, bool upper_only, RowPlan &plan) {
    plan = RowPlan();
    plan.groups = groups;
    plan.small_max = small_max;
    plan.upper_only = upper_only;
    const int64_t n = g->n;
    if (n == 0) return AD_OK;
    int8_t *cls = nullptr;
    int64_t *nchunks = nullptr, *counts = nullptr, *offs = nullptr;
    int32_t *order = nullptr;
    const int64_t tiles = (n + kPartThreads - 1) / kPartThreads;
    AD_TRY(dalloc_t(g, n, &cls));
    AD_TRY(dalloc_t(g, n, &nchunks));
    AD_TRY(dalloc_t(g, (size_t)kClasses * tiles, &counts));
    AD_TRY(dalloc_t(g, (size_t)kClasses * tiles, &offs));
    AD_TRY(dalloc_t(g, n, &order));
    AD_LAUNCH(k_row_class, g->num_sms * 8, 256, 0, g->stream, g->rp, g->upos, n, small_max, upper_only ? 1 : 0, cls,
              nchunks);
    AD_LAUNCH(k_class_counts, (int)tiles, kPartThreads, 0, g->stream, cls, n, counts, tiles);
    int64_t total = 0;
    AD_TRY(exclusive_scan_i64(g, counts, offs, (int64_t)kClasses * tiles, &total));
    AD_LAUNCH(k_class_scatter, (int)tiles, kPartThreads, 0, g->stream, cls, n, offs, tiles, order);
    // class boundaries: offsets at tile 0 of each class
    std::vector<int64_t> start(kClasses + 1);
    {
        std::vector<int64_t> at(kClasses);
        for (int c = 0; c < kClasses; ++c) at[c] = (int64_t)c * tiles;
        int64_t *at_d = nullptr, *picked = nullptr;
        AD_TRY(dalloc_t(g, kClasses, &at_d));
        AD_TRY(dalloc_t(g, kClasses, &picked));
        AD_TRY(copy_in(g, at_d, at.data(), kClasses * sizeof(int64_t)));
        AD_LAUNCH(k_pick_i64, 1, kClasses, 0, g->stream, offs, at_d, (int64_t)kClasses, (int64_t)kClasses * tiles,
                  total, picked);
        AD_TRY(copy_out(g, start.data(), picked, kClasses * sizeof(int64_t)));
        dfree(g, at_d);
        dfree(g, picked);
    }
    start[kClasses] = total;
    const int64_t n_big_rows = start[1] - start[0];
    const int64_t n_med = start[11] - start[1];
    const int64_t n_small = start[12] - start[11];
    // big rows -> chunk tasks
    if (n_big_rows > 0) {
        int64_t *ch = nullptr, *first = nullptr;
        AD_TRY(dalloc_t(g, n_big_rows, &ch));
        AD_TRY(dalloc_t(g, n_big_rows, &first));
        AD_LAUNCH(k_gather_i64, (int)((n_big_rows + 255) / 256), 256, 0, g->stream, nchunks, order, n_big_rows, ch);
        int64_t n_chunks = 0;
        AD_TRY(exclusive_scan_i64(g, ch, first, n_big_rows, &n_chunks));
        AD_TRY(dalloc_t(g, n_chunks, &plan.big_row));
        AD_TRY(dalloc_t(g, n_chunks, &plan.big_chunk));
        AD_TRY(dalloc_t(g, n_chunks, &plan.big_counter));
        AD_CUDA_TRY(cudaMemsetAsync(plan.big_counter, 0, n_chunks * sizeof(uint32_t), g->stream));
        AD_LAUNCH(k_expand_chunks, (int)std::min<int64_t>((n_big_rows + 7) / 8, 4096), 256, 0, g->stream, order,
                  n_big_rows, g->rp, g->upos, upper_only ? 1 : 0, first, plan.big_row, plan.big_chunk);
        plan.n_big = n_chunks;
        dfree(g, ch);
        dfree(g, first);
    }
    if (n_med > 0) {
        AD_TRY(dalloc_t(g, n_med, &plan.medium_row));
        AD_CUDA_TRY(cudaMemcpyAsync(plan.medium_row, order + start[1], n_med * sizeof(int32_t),
                                    cudaMemcpyDeviceToDevice, g->stream));
    }
    if (n_small > 0) {
        AD_TRY(dalloc_t(g, n_small, &plan.small_row));
        AD_CUDA_TRY(cudaMemcpyAsync(plan.small_row, order + start[11], n_small * sizeof(int32_t),
                                    cudaMemcpyDeviceToDevice, g->stream));
    }
    plan.n_medium = n_med;
    plan.n_small_rows = n_small;
    AD_CUDA_TRY(cudaStreamSynchronize(g->stream));
    dfree(g, cls);
    dfree(g, nchunks);
    dfree(g, counts);
    dfree(g, offs);
    dfree(g, order);
    return AD_OK;
}

// ----------------------------------------------------------------------------
// Degree classes for Alg. 2: index of each row's degree among the distinct
// degrees (host table of distinct degrees kept in the handle).
// ----------------------------------------------------------------------------
__global__ void k_degree_hist_flags(const int64_t *rp, int64_t n, int64_t maxd, int32_t *present) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t d = rp[i + 1] - rp[i];
        if (d > 0) present[d] = 1;
    }
}
__global__ void k_degree_class(const int64_t *rp, int64_t n, const int32_t *index_of_degree, int32_t *dc) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t d = rp[i + 1] - rp[i];
        dc[i] = d > 0 ? index_of_degree[d] : -1;
    }
}
__global__ void k_row_degree_max(const int64_t *rp, int64_t n, unsigned long long *mx) {
    unsigned long long v = 0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        v = max(v, (unsigned long long)(rp[i + 1] - rp[i]));
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = max(v, __shfl_xor_sync(0xffffffffu, v, o));
    if ((threadIdx.x & 31) == 0 && v) atomicMax(mx, v);
}

ad_status ensure_degree_classes(ad_graph_t g) {
    if (g->deg_class || g->n == 0) return AD_OK;
    unsigned long long *mx = nullptr;
    AD_TRY(dalloc_t(g, 1, &mx));
    AD_CUDA_TRY(cudaMemsetAsync(mx, 0, sizeof(unsigned long long), g->stream));
    AD_LAUNCH(k_row_degree_max, g->num_sms * 8, 256, 0, g->stream, g->rp, g->n, mx);
    unsigned long long maxd = 0;
    AD_TRY(copy_out(g, &maxd, mx, sizeof(maxd)));
    dfree(g, mx);
    int32_t *present = nullptr;
    AD_TRY(dalloc_t(g, maxd + 1, &present));
    AD_CUDA_TRY(cudaMemsetAsync(present, 0, (maxd + 1) * sizeof(int32_t), g->stream));
    AD_LAUNCH(k_degree_hist_flags, g->num_sms * 8, 256, 0, g->stream, g->rp, g->n, (int64_t)maxd, present);
    std::vector<int32_t> ph(maxd + 1);
    AD_TRY(copy_out(g, ph.data(), present, (maxd + 1) * sizeof(int32_t)));
    g->distinct_degrees.clear();
    std::vector<int32_t> idx(maxd + 1, -1);
    for (uint64_t d = 1; d <= maxd; ++d)
        if (ph[d]) {
            idx[d] = (int32_t)g->distinct_degrees.size();
            g->distinct_degrees.push_back((int64_t)d);
        }
    AD_TRY(copy_in(g, present, idx.data(), (maxd + 1) * sizeof(int32_t)));
    AD_TRY(dalloc_t(g, g->n, &g->deg_class));
    AD_LAUNCH(k_degree_class, g->num_sms * 8, 256, 0, g->stream, g->rp, g->n, present, g->deg_class);
    AD_CUDA_TRY(cudaStreamSynchronize(g->stream));
    dfree(g, present);
    g->n_deg_classes = (int32_t)g->distinct_degrees.size();
    return AD_OK;
}

}  // namespace ad
