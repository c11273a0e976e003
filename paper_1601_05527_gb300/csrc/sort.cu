// sort.cu -- stable LSD radix sort of (uint64 key, int64 value) pairs and
// flag compaction, used by the Galerkin coarsening (sorting coarse edge pairs)
// and by the construction of coarse and sparsified CSR graphs.
//
// One pass per 8-bit digit: per-tile digit histograms, an exclusive scan in
// digit-major order, then a stable scatter.  Inside a tile each warp owns a
// contiguous segment; warps are ordered by a per-digit prefix over warps and
// lanes of one 32-element chunk by __match_any_sync peer ranks, so equal
// digits keep their input order.
#include "ad_internal.cuh"

namespace ad {

constexpr int kRsThreads = 256;
constexpr int kRsWarps = kRsThreads / 32;
constexpr int kRsPerWarp = 256;                     // elements per warp segment
constexpr int kRsTile = kRsWarps * kRsPerWarp;      // 2048 elements per CTA

__global__ void k_rs_hist(const uint64_t *keys, int64_t n, int shift, uint32_t *counts, int64_t tiles) {
    __shared__ uint32_t h[256];
    h[threadIdx.x] = 0;
    __syncthreads();
    const int64_t base = (int64_t)blockIdx.x * kRsTile;
    for (int t = threadIdx.x; t < kRsTile; t += kRsThreads) {
        const int64_t i = base + t;
        if (i < n) atomicAdd(&h[(keys[i] >> shift) & 0xff], 1u);
    }
    __syncthreads();
    counts[(int64_t)threadIdx.x * tiles + blockIdx.x] = h[threadIdx.x];
}

__global__ void k_rs_scatter(const uint64_t *kin, const int64_t *vin, uint64_t *kout, int64_t *vout, int64_t n,
                             int shift, const int64_t *offsets, int64_t tiles) {
    __shared__ uint32_t wh[kRsWarps][256];
    __shared__ int64_t wbase[kRsWarps][256];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int d = lane; d < 256; d += 32) wh[warp][d] = 0;
    __syncwarp();
    const int64_t seg = (int64_t)blockIdx.x * kRsTile + (int64_t)warp * kRsPerWarp;
    for (int c = 0; c < kRsPerWarp; c += 32) {
        const int64_t i = seg + c + lane;
        if (i < n) atomicAdd(&wh[warp][(kin[i] >> shift) & 0xff], 1u);
    }
    __syncthreads();
    {   // thread d: base of digit d for every warp of the tile
        const int d = threadIdx.x;
        int64_t b = offsets[(int64_t)d * tiles + blockIdx.x];
        for (int w = 0; w < kRsWarps; ++w) {
            wbase[w][d] = b;
            b += wh[w][d];
        }
    }
    __syncthreads();
    const unsigned lt = (1u << lane) - 1u;
    for (int c = 0; c < kRsPerWarp; c += 32) {
        const int64_t i = seg + c + lane;
        const bool valid = i < n;
        const uint64_t k = valid ? kin[i] : 0;
        const int d = valid ? (int)((k >> shift) & 0xff) : 256;
        const unsigned peers = __match_any_sync(0xffffffffu, d);
        if (valid) {
            const int64_t pos = wbase[warp][d] + __popc(peers & lt);
            kout[pos] = k;
            vout[pos] = vin[i];
        }
        __syncwarp();
        if (valid && (peers & lt) == 0) wbase[warp][d] += __popc(peers);   // lowest peer advances
        __syncwarp();
    }
}

__global__ void k_widen_u32(const uint32_t *in, int64_t n, int64_t *out) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] = in[i];
}

// Sort n pairs by the bit ranges [shift, shift + 8) listed in shifts (LSD order).
// keys/vals are sorted in place (through a scratch pair of buffers).
ad_status radix_sort_pairs(ad_graph_t g, uint64_t *keys, int64_t *vals, int64_t n, const std::vector<int> &shifts) {
    if (n <= 1 || shifts.empty()) return AD_OK;
    const int64_t tiles = (n + kRsTile - 1) / kRsTile;
    uint64_t *k2 = nullptr;
    int64_t *v2 = nullptr;
    uint32_t *counts = nullptr;
    int64_t *cnt64 = nullptr, *offs = nullptr;
    AD_TRY(dalloc_t(g, n, &k2));
    AD_TRY(dalloc_t(g, n, &v2));
    AD_TRY(dalloc_t(g, 256 * tiles, &counts));
    AD_TRY(dalloc_t(g, 256 * tiles, &cnt64));
    AD_TRY(dalloc_t(g, 256 * tiles, &offs));
    uint64_t *ka = keys, *kb = k2;
    int64_t *va = vals, *vb = v2;
    for (int sh : shifts) {
        AD_LAUNCH(k_rs_hist, (int)tiles, kRsThreads, 0, g->stream, ka, n, sh, counts, tiles);
        AD_LAUNCH(k_widen_u32, (int)((256 * tiles + 255) / 256), 256, 0, g->stream, counts, 256 * tiles, cnt64);
        AD_TRY(exclusive_scan_i64(g, cnt64, offs, 256 * tiles, nullptr));
        AD_LAUNCH(k_rs_scatter, (int)tiles, kRsThreads, 0, g->stream, ka, va, kb, vb, n, sh, offs, tiles);
        std::swap(ka, kb);
        std::swap(va, vb);
    }
    if (ka != keys) {
        AD_CUDA_TRY(cudaMemcpyAsync(keys, ka, n * sizeof(uint64_t), cudaMemcpyDeviceToDevice, g->stream));
        AD_CUDA_TRY(cudaMemcpyAsync(vals, va, n * sizeof(int64_t), cudaMemcpyDeviceToDevice, g->stream));
    }
    AD_CUDA_TRY(cudaStreamSynchronize(g->stream));
    dfree(g, k2);
    dfree(g, v2);
    dfree(g, counts);
    dfree(g, cnt64);
    dfree(g, offs);
    return AD_OK;
}

__global__ void k_flags_u8(const uint8_t *f, int64_t n, int64_t *out) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] = f[i] ? 1 : 0;
}

__global__ void k_compact_idx(const uint8_t *f, const int64_t *pos, int64_t n, int64_t *out) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n && f[i]) out[pos[i]] = i;
}

// Indices i with flag[i] != 0, in increasing order; *count receives their number.
ad_status compact_flags(ad_graph_t g, const uint8_t *flag, int64_t n, int64_t **idx_out, int64_t *count) {
    *idx_out = nullptr;
    *count = 0;
    if (n <= 0) return AD_OK;
    int64_t *f64 = nullptr, *pos = nullptr, *idx = nullptr;
    AD_TRY(dalloc_t(g, n, &f64));
    AD_TRY(dalloc_t(g, n, &pos));
    AD_LAUNCH(k_flags_u8, (int)((n + 255) / 256), 256, 0, g->stream, flag, n, f64);
    int64_t total = 0;
    AD_TRY(exclusive_scan_i64(g, f64, pos, n, &total));
    AD_TRY(dalloc_t(g, total + 1, &idx));
    AD_LAUNCH(k_compact_idx, (int)((n + 255) / 256), 256, 0, g->stream, flag, pos, n, idx);
    AD_CUDA_TRY(cudaStreamSynchronize(g->stream));
    dfree(g, f64);
    dfree(g, pos);
    *idx_out = idx;
    *count = total;
    return AD_OK;
}

}  // namespace ad
