// binned.cu -- selection order of SparsifyB (Alg. 3) on sm_103a.
//
// Per node i of degree d, with the distances rho of its incident edges:
//   mean and sigma (population) in FP64, bin width h = 3.5 sigma / cbrt(d)
//   (the rule quoted in Sec. 4), bin of an entry = floor((rho - min) / h) in
//   FP64, a single bin when sigma = 0;
//   entries of a bin in order of a Philox word of the edge id, bins in order
//   of a Philox word of (i, 1 + bin); the selection order is a round robin
//   over the bins -- round r takes the r-th entry of every bin that has one,
//   bins in their order -- so every bin contributes before any contributes
//   twice.  Node i keeps its entries of rank < T(d, e); the union over the two
//   ends of an edge and the fit of e are those of Alg. 2 (select.cu).
//
// Rows of up to 32 entries are summed by one lane, sequentially in CSR order,
// exactly as the definition states; longer rows by FP64 reductions over the
// lanes of a warp (the two orders differ only in the rounding of the FP64
// sums, far below the FP32 resolution of the distances).  Every other step
// that decides a bin is the same IEEE FP64 operation as in the definition:
// the bin index is taken from an FP32 estimate only where a bound on its error
// proves it equal to the FP64 quotient's floor, and cbrt(d) comes from the
// host's FP64 cbrt.
//
// Pipeline: per-row statistics (one warp per 32 rows, one block per row above
// 512 entries), per-entry bin and Philox word, one per-row rank by (bin, top
// bits of the word) with the rare ties of the truncated word put in full-word
// order afterwards, runs of equal (row, bin) = the non-empty bins, their order
// inside the row (counted directly for rows of few bins), and per entry the
// round-robin rank (counted directly where that is cheaper than a per-row rank
// pass).
#include "ad_internal.cuh"

#include <algorithm>
#include <cmath>
#include <vector>

namespace ad {

constexpr uint32_t kBinStream = 0xB1000000u;   // Philox counter word 3 of the binning draws
constexpr int kBinBits = 24;                   // bins per row < 2^24 (at most ~0.4 d^(5/6) for any data)

__device__ __forceinline__ uint32_t bin_word(uint64_t seed, uint64_t a, uint32_t z) {
    const uint4 c = make_uint4((uint32_t)a, (uint32_t)(a >> 32), z, kBinStream);
    return philox4x32_10(c, make_uint2((uint32_t)seed, (uint32_t)(seed >> 32))).x;
}

// the distance of every CSR entry, in CSR order, so that the per-row sums
// below read one contiguous run instead of chasing edge ids
__global__ void k_bin_gather(const int64_t *eid, const float *score, int64_t nnz, float *xs) {
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < nnz; p += (int64_t)gridDim.x * blockDim.x)
        xs[p] = score[eid[p]];
}

// A butterfly sum of one FP64 value per lane; every add is an explicitly
// rounded FP64 one.
__device__ __forceinline__ double warp_sum_f64(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = __dadd_rn(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}

// Sums in FP32 pairs.  The GB300's FP64 pipe is narrow, so the per-entry
// terms of the row sums are added in FP32 with error-free transformations
// (Knuth's TwoSum, and an FMA for the exact rounding error of a square): the
// pair (h, l) keeps the running sum h and the accumulated rounding errors l,
// so a lane's sum of c terms is within about c * 2^-48 (relative) of the exact
// one -- at the FP64 level for every row length that occurs.  Only the
// combination of the lanes' pairs and the per-row divisions and square root
// run in FP64.
struct PairSum {
    float h = 0.0f, l = 0.0f;
};

__device__ __forceinline__ void two_sum(float a, float b, float &s, float &e) {
    s = __fadd_rn(a, b);
    const float bp = __fsub_rn(s, a);
    e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bp)), __fsub_rn(b, bp));
}

__device__ __forceinline__ void pair_add(PairSum &a, float x) {
    float s, e;
    two_sum(a.h, x, s, e);
    a.h = s;
    a.l = __fadd_rn(a.l, e);
}

// adds (x - m)^2 for m = mh + ml: x - m is carried exactly as th + dl + dll
// (three error-free sums), renormalised to a + b with |b| at most about one
// ulp of a, and squared as a^2 (exactly, p + pe) + 2ab; b^2 is below 2^-48 a^2
__device__ __forceinline__ void pair_add_sq(PairSum &q, float x, float mh, float ml) {
    float th, tl, dl, dll, a, b;
    two_sum(x, -mh, th, tl);
    two_sum(tl, -ml, dl, dll);
    two_sum(th, dl, a, b);
    b = __fadd_rn(b, dll);
    const float p = __fmul_rn(a, a);
    float pe = __fmaf_rn(a, a, -p);
    pe = __fmaf_rn(__fmul_rn(2.0f, a), b, pe);
    float s, e;
    two_sum(q.h, p, s, e);
    q.h = s;
    q.l = __fadd_rn(q.l, __fadd_rn(e, pe));
}

__device__ __forceinline__ double pair_value(const PairSum &a) { return __dadd_rn((double)a.h, (double)a.l); }

// 2^k for |k| <= 126 as an FP32 value, and 2^k as an FP64 value
__device__ __forceinline__ float pow2f(int k) { return __int_as_float((127 + k) << 23); }
__device__ __forceinline__ double pow2d(int k) { return __longlong_as_double((long long)(1023 + k) << 52); }

// The row is scaled by 2^k (two exact FP32 multiplications) so that its
// largest distance lies in [1, 2): the pairs then stay far from overflow and
// from the subnormal range whatever the scale of the distances.
__device__ __forceinline__ int row_scale_exp(float hi) {
    if (!(hi > 0.0f)) return 0;
    int e;
    frexpf(hi, &e);            // hi = f 2^e, f in [0.5, 1)
    return 1 - e;
}

__device__ __forceinline__ float scaled(float x, float a, float b) { return __fmul_rn(__fmul_rn(x, a), b); }

constexpr int kShortRow = 32;       // rows up to this length are summed by one lane
constexpr int kWarpRowMax = (int)kLongRowDegree;   // longer rows take a whole block

// sigma of the unscaled distances, sqrt(q / d) / 2^k, and from it the row's
// bin width h and its FP32 reciprocal
__device__ __forceinline__ void finish_row(int64_t i, int64_t d, float lo, float hi, double q, int k, const int32_t *dc,
                                           const double *cbrt_dc, float *lo_out, double *h_out, float *rinv_out) {
    const double sigma = __dmul_rn(__dsqrt_rn(__ddiv_rn(q, (double)d)), pow2d(-k));
    const double h = (sigma > 0.0 && hi > lo) ? __ddiv_rn(__dmul_rn(3.5, sigma), cbrt_dc[dc[i]]) : 0.0;
    const double inv = h > 0.0 ? __ddiv_rn(1.0, h) : 0.0;
    lo_out[i] = lo;
    h_out[i] = h;
    rinv_out[i] = (inv > 0x1p-100 && inv < 0x1p100) ? __double2float_rn(inv) : 0.0f;
}

// Per row: lo = min rho, h = bin width in FP64 (0: a single bin) and
// rinv = 1/h rounded to FP32 (0 when 1/h is outside the FP32 normal range).
// One warp takes 32 consecutive rows.  A row of up to kShortRow entries is
// summed by its own lane, sequentially in CSR order; a row of up to
// kWarpRowMax by the whole warp (longer rows: k_bin_stats_big), every lane summing every 32nd entry and the lane sums added by an FP64
// butterfly.  Three passes over the row: min and max, the sum (for the mean),
// the sum of squared deviations from the mean.  The divisions and the square
// root of the 32 rows run once, one row per lane.
__global__ void k_bin_stats(const int64_t *rp, const float *xs, const int32_t *dc, const double *cbrt_dc, int64_t n,
                            float *lo_out, double *h_out, float *rinv_out) {
    const int lane = threadIdx.x & 31;
    const int64_t W = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t base = ((blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5) << 5; base < n; base += W << 5) {
        const int64_t i = base + lane;
        int64_t p0 = 0, d = 0;
        if (i < n) {
            p0 = rp[i];
            d = rp[i + 1] - p0;
        }
        const bool own = d <= kShortRow;
        const unsigned longs = __ballot_sync(0xffffffffu, !own && d <= kWarpRowMax);
        // pass 1: min and max
        float lo = INFINITY, hi = -INFINITY;
        if (own)
            for (int64_t t = 0; t < d; ++t) {
                const float v = xs[p0 + t];
                lo = fminf(lo, v);
                hi = fmaxf(hi, v);
            }
        for (unsigned m = longs; m; m &= m - 1) {
            const int r = __ffs(m) - 1;
            const int64_t q0 = __shfl_sync(0xffffffffu, p0, r), dq = __shfl_sync(0xffffffffu, d, r);
            float l = INFINITY, u = -INFINITY;
            for (int64_t t = lane; t < dq; t += 32) {
                const float v = xs[q0 + t];
                l = fminf(l, v);
                u = fmaxf(u, v);
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                l = fminf(l, __shfl_xor_sync(0xffffffffu, l, o));
                u = fmaxf(u, __shfl_xor_sync(0xffffffffu, u, o));
            }
            if (lane == r) {
                lo = l;
                hi = u;
            }
        }
        const int k = row_scale_exp(hi);
        const float sa = pow2f(k / 2), sb = pow2f(k - k / 2);
        // pass 2: the sum of the scaled distances
        double sum = 0.0;
        if (own) {
            PairSum acc;
            for (int64_t t = 0; t < d; ++t) pair_add(acc, scaled(xs[p0 + t], sa, sb));
            sum = pair_value(acc);
        }
        for (unsigned m = longs; m; m &= m - 1) {
            const int r = __ffs(m) - 1;
            const int64_t q0 = __shfl_sync(0xffffffffu, p0, r), dq = __shfl_sync(0xffffffffu, d, r);
            const float ra = __shfl_sync(0xffffffffu, sa, r), rb = __shfl_sync(0xffffffffu, sb, r);
            PairSum acc;
            for (int64_t t = lane; t < dq; t += 32) pair_add(acc, scaled(xs[q0 + t], ra, rb));
            const double s = warp_sum_f64(pair_value(acc));
            if (lane == r) sum = s;
        }
        const double mean = __ddiv_rn(sum, d > 0 ? (double)d : 1.0);
        const float mh = __double2float_rn(mean), ml = __double2float_rn(__dsub_rn(mean, (double)mh));
        // pass 3: the sum of squared deviations from the mean
        double q = 0.0;
        if (own) {
            PairSum acc;
            for (int64_t t = 0; t < d; ++t) pair_add_sq(acc, scaled(xs[p0 + t], sa, sb), mh, ml);
            q = pair_value(acc);
        }
        for (unsigned m = longs; m; m &= m - 1) {
            const int r = __ffs(m) - 1;
            const int64_t q0 = __shfl_sync(0xffffffffu, p0, r), dq = __shfl_sync(0xffffffffu, d, r);
            const float ra = __shfl_sync(0xffffffffu, sa, r), rb = __shfl_sync(0xffffffffu, sb, r);
            const float rh = __shfl_sync(0xffffffffu, mh, r), rl = __shfl_sync(0xffffffffu, ml, r);
            PairSum acc;
            for (int64_t t = lane; t < dq; t += 32) pair_add_sq(acc, scaled(xs[q0 + t], ra, rb), rh, rl);
            const double s = warp_sum_f64(pair_value(acc));
            if (lane == r) q = s;
        }
        if (i < n && d > 0 && d <= kWarpRowMax) finish_row(i, d, lo, hi, q, k, dc, cbrt_dc, lo_out, h_out, rinv_out);
    }
}

// A block per row longer than kWarpRowMax, from the list of such rows (the
// hubs: at R-MAT scale 20 the rows above 1024 entries hold 43% of the entries,
// and a warp that met several of them would hold up the whole launch).  The same three passes; the threads' pairs
// are combined in FP64 through shared memory.
constexpr int kBigRowThreads = 256;

__device__ __forceinline__ double block_sum_f64(double v, double *sh) {
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    v = warp_sum_f64(v);
    if (lane == 0) sh[w] = v;
    __syncthreads();
    if (w == 0) {
        v = lane < kBigRowThreads / 32 ? sh[lane] : 0.0;
        v = warp_sum_f64(v);
        if (lane == 0) sh[kBigRowThreads / 32] = v;
    }
    __syncthreads();
    const double r = sh[kBigRowThreads / 32];
    __syncthreads();
    return r;
}

__global__ void __launch_bounds__(kBigRowThreads) k_bin_stats_big(const int64_t *rp, const float *xs, const int32_t *dc,
                                                                  const double *cbrt_dc, const int64_t *rows,
                                                                  int64_t nrows, float *lo_out, double *h_out,
                                                                  float *rinv_out) {
    __shared__ double shd[kBigRowThreads / 32 + 1];
    __shared__ float shl[kBigRowThreads / 32], shu[kBigRowThreads / 32];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    for (int64_t b = blockIdx.x; b < nrows; b += gridDim.x) {
        const int64_t i = rows[b], p0 = rp[i], d = rp[i + 1] - p0;
        const float *x = xs + p0;
        float lo = INFINITY, hi = -INFINITY;
        for (int64_t t = threadIdx.x; t < d; t += kBigRowThreads) {
            const float v = x[t];
            lo = fminf(lo, v);
            hi = fmaxf(hi, v);
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            lo = fminf(lo, __shfl_xor_sync(0xffffffffu, lo, o));
            hi = fmaxf(hi, __shfl_xor_sync(0xffffffffu, hi, o));
        }
        if (lane == 0) {
            shl[w] = lo;
            shu[w] = hi;
        }
        __syncthreads();
        lo = shl[0];
        hi = shu[0];
        for (int j = 1; j < kBigRowThreads / 32; ++j) {
            lo = fminf(lo, shl[j]);
            hi = fmaxf(hi, shu[j]);
        }
        const int k = row_scale_exp(hi);
        const float sa = pow2f(k / 2), sb = pow2f(k - k / 2);
        PairSum acc;
        for (int64_t t = threadIdx.x; t < d; t += kBigRowThreads) pair_add(acc, scaled(x[t], sa, sb));
        const double sum = block_sum_f64(pair_value(acc), shd);
        const double mean = __ddiv_rn(sum, (double)d);
        const float mh = __double2float_rn(mean), ml = __double2float_rn(__dsub_rn(mean, (double)mh));
        PairSum acc2;
        for (int64_t t = threadIdx.x; t < d; t += kBigRowThreads) pair_add_sq(acc2, scaled(x[t], sa, sb), mh, ml);
        const double q = block_sum_f64(pair_value(acc2), shd);
        if (threadIdx.x == 0) finish_row(i, d, lo, hi, q, k, dc, cbrt_dc, lo_out, h_out, rinv_out);
    }
}

// Bin of one entry: floor((x - lo) / h), the FP64 quotient of the definition.
// The FP32 estimate t = (x - lo) * rinv is within 2^-21 t of that quotient
// (four FP32 roundings of at most 2^-24 each, plus the FP64 ones); when t is
// further than 2^-20 t from every integer, floor(t) is the FP64 result, and
// otherwise (rarely) the FP64 division itself decides.
__device__ __forceinline__ int64_t bin_of(float x, float lo, double h, float rinv) {
    if (!(h > 0.0)) return 0;
    if (rinv > 0.0f) {
        const float t = __fmul_rn(__fsub_rn(x, lo), rinv);
        if (t < 0x1p22f) {
            const float f = floorf(t), m = t * 0x1p-20f;
            if (__fadd_rn(t, m) < f + 1.0f && (f == 0.0f || __fsub_rn(t, m) > f)) return (int64_t)f;
        }
    }
    return (int64_t)floor(__ddiv_rn(__dsub_rn((double)x, (double)lo), h));
}

// per entry: its bin and Philox word; keys for the first sort (by word), values = positions
__global__ void k_bin_entries(const int32_t *erow, const int64_t *eid, const float *xs, const float *lo,
                              const double *h, const float *rinv, int64_t nnz, uint64_t seed, uint32_t *bin, uint64_t *keys,
                              int64_t *vals, unsigned long long *max_bin) {
    unsigned long long mb = 0;
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < nnz; p += (int64_t)gridDim.x * blockDim.x) {
        const int32_t i = erow[p];
        const int64_t b = bin_of(xs[p], lo[i], h[i], rinv[i]);
        bin[p] = (uint32_t)b;
        mb = (unsigned long long)b > mb ? (unsigned long long)b : mb;
        keys[p] = bin_word(seed, (uint64_t)eid[p], 0u);
        vals[p] = p;
    }
    for (int o = 16; o > 0; o >>= 1) {
        const unsigned long long y = __shfl_xor_sync(0xffffffffu, mb, o);
        mb = y > mb ? y : mb;
    }
    if ((threadIdx.x & 31) == 0 && mb) atomicMax(max_bin, mb);
}

// keys of the second sort: (row, bin) of the entry now at each slot
__global__ void k_bin_rowkeys(const int64_t *vals, const int32_t *erow, const uint32_t *bin, int64_t nnz,
                              uint64_t *keys) {
    for (int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; s < nnz; s += (int64_t)gridDim.x * blockDim.x) {
        const int64_t p = vals[s];
        keys[s] = ((uint64_t)(uint32_t)erow[p] << kBinBits) | bin[p];
    }
}

// run starts: slot s begins a non-empty bin when its (row, bin) differs from slot s - 1
__global__ void k_bin_run_flags(const uint64_t *keys, int64_t nnz, int64_t *flag) {
    for (int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; s < nnz; s += (int64_t)gridDim.x * blockDim.x)
        flag[s] = (s == 0 || keys[s] != keys[s - 1]) ? 1 : 0;
}

// the exclusive scan of the run starts counts the starts before a slot; the
// run of the slot is that count, less one unless the slot starts a run itself
__global__ void k_bin_inclusive(const int64_t *flag, int64_t nnz, int64_t *run_of) {
    for (int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; s < nnz; s += (int64_t)gridDim.x * blockDim.x)
        run_of[s] += flag[s] - 1;
}

// run records: first slot of each run, its bin's Philox word; runs of a row are contiguous
__global__ void k_bin_runs(const uint64_t *keys, const int64_t *flag, const int64_t *run_of, int64_t nnz, uint64_t seed,
                           int64_t *run_start, uint32_t *run_word, int64_t *row_runs) {
    for (int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; s < nnz; s += (int64_t)gridDim.x * blockDim.x) {
        if (s == nnz - 1) run_start[run_of[s] + 1] = nnz;   // end of the last run
        if (!flag[s]) continue;
        const int64_t r = run_of[s];
        const uint64_t k = keys[s];
        const uint64_t row = k >> kBinBits;
        const uint32_t b = (uint32_t)(k & ((1u << kBinBits) - 1u));
        run_start[r] = s;
        run_word[r] = bin_word(seed, row, 1u + b);
        if (s == 0 || (keys[s - 1] >> kBinBits) != row) row_runs[row] = r;   // first run of the row
    }
}

// per entry: round-robin rank = sum over the row's bins c of min(size_c, r)
// plus the bins that have an r-th entry and come before the entry's bin,
// with r the entry's place inside its bin
__global__ void k_bin_ranks(const uint64_t *keys, const int64_t *vals, const int64_t *run_of, const int64_t *run_start,
                            const uint32_t *run_word, const int64_t *row_runs, const int64_t *rp, int64_t nnz,
                            int64_t nruns, uint32_t *rank) {
    for (int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; s < nnz; s += (int64_t)gridDim.x * blockDim.x) {
        const int64_t row = (int64_t)(keys[s] >> kBinBits);
        const int64_t r0 = row_runs[row];
        const int64_t slot_end = rp[row + 1];   // rows keep their CSR ranges in the sorted order
        const int64_t me = run_of[s];
        const int64_t r = s - run_start[me];
        const uint32_t wm = run_word[me];
        const uint64_t bm = keys[s] & ((1ull << kBinBits) - 1ull);
        int64_t rk = 0;
        for (int64_t c = r0; c < nruns && run_start[c] < slot_end; ++c) {
            const int64_t next = (c + 1 < nruns) ? run_start[c + 1] : nnz;
            const int64_t size = (next < slot_end ? next : slot_end) - run_start[c];
            rk += size < r ? size : r;
            const uint64_t bc = keys[run_start[c]] & ((1ull << kBinBits) - 1ull);
            const bool before = run_word[c] < wm || (run_word[c] == wm && bc < bm);
            if (size > r && before) ++rk;
        }
        rank[vals[s]] = (uint32_t)rk;
    }
}

// ----------------------------------------------------------------------------
// The same order from per-row ranks of 32-bit keys (rows of at most 2^18
// entries, whose bins are then fewer than 2^14).  The round-robin rank of an
// entry is its position when the row's entries are ordered by (its index
// inside its bin, its bin's place in the random bin order): round r lists the
// r-th entries of the bins, bins in their order.  So:
//   1. rank by Philox word inside the row (ties by position);
//   2. rank by (bin, that rank): the row in bin order, random order inside bins;
//   3. the index r of each entry inside its bin, from the runs of equal bins;
//   4. the bins of each row ordered by their Philox word (a sort of the runs);
//   5. rank by (r, the bin's place) = the selection rank.
// ----------------------------------------------------------------------------
constexpr int kRowRankBits = 18;   // rank inside a row < 2^18
constexpr int kBinOrderBits = 14;  // bins of a row < 2^14

__global__ void k_bin_words(const int32_t *erow, const int64_t *eid, const float *xs, const float *lo, const double *h,
                            const float *rinv, int64_t nnz, uint64_t seed, uint32_t *bin, uint32_t *word, unsigned long long *max_bin) {
    unsigned long long mb = 0;
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < nnz; p += (int64_t)gridDim.x * blockDim.x) {
        const int32_t i = erow[p];
        const int64_t b = bin_of(xs[p], lo[i], h[i], rinv[i]);
        bin[p] = (uint32_t)b;
        mb = (unsigned long long)b > mb ? (unsigned long long)b : mb;
        word[p] = bin_word(seed, (uint64_t)eid[p], 0u);
    }
    for (int o = 16; o > 0; o >>= 1) {
        const unsigned long long y = __shfl_xor_sync(0xffffffffu, mb, o);
        mb = y > mb ? y : mb;
    }
    if ((threadIdx.x & 31) == 0 && mb) atomicMax(max_bin, mb);
}

// Key of the one per-row ranking pass: the bin in the top bbits bits, the top
// 32 - bbits bits of the entry's Philox word below it.  Ranking by (key,
// position) orders a row by (bin, word) except among entries of one bin whose
// truncated words tie; k_bin_fix_ties puts those in (word, position) order.
__global__ void k_bin_key1(const uint32_t *bin, const uint32_t *word, int64_t nnz, int bbits, uint32_t *key) {
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < nnz; p += (int64_t)gridDim.x * blockDim.x)
        key[p] = bbits == 0 ? word[p] : (bin[p] << (32 - bbits)) | (word[p] >> bbits);
}

// Runs of equal key inside a row in the sorted slots: the first slot of each
// run of two or more reorders it by (full word, position) -- an insertion sort,
// the runs being short (two entries collide with probability 2^(bbits - 32)).
__global__ void k_bin_fix_ties(int32_t *sorted, const int32_t *erow, const uint32_t *key, const uint32_t *word,
                               int64_t nnz) {
    for (int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; s < nnz; s += (int64_t)gridDim.x * blockDim.x) {
        const int32_t p = sorted[s];
        const int32_t row = erow[p];
        const uint32_t k = key[p];
        if (s > 0) {
            const int32_t pp = sorted[s - 1];
            if (erow[pp] == row && key[pp] == k) continue;     // not the first slot of its run
        }
        int64_t e = s + 1;
        while (e < nnz && erow[sorted[e]] == row && key[sorted[e]] == k) ++e;
        for (int64_t a = s + 1; a < e; ++a) {
            const int32_t v = sorted[a];
            const uint32_t wv = word[v];
            int64_t b = a - 1;
            while (b >= s) {
                const int32_t u = sorted[b];
                const uint32_t wu = word[u];
                if (wu < wv || (wu == wv && u < v)) break;
                sorted[b + 1] = u;
                --b;
            }
            sorted[b + 1] = v;
        }
    }
}

// entries in (bin, word) order inside their rows: slot rp[row] + rank
__global__ void k_bin_place(const int32_t *erow, const int64_t *rp, const uint32_t *s2, const uint32_t *bin, int64_t nnz,
                            int32_t *sorted, uint32_t *sbin) {
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < nnz; p += (int64_t)gridDim.x * blockDim.x) {
        const int64_t slot = rp[erow[p]] + s2[p];
        sorted[slot] = (int32_t)p;
        sbin[slot] = bin[p];
    }
}

// slot s starts a run (a non-empty bin of a row) when its row or bin differs from slot s - 1
__global__ void k_bin_run_starts(const int32_t *sorted, const int32_t *erow, const uint32_t *sbin, int64_t nnz,
                                 int64_t *flag) {
    for (int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; s < nnz; s += (int64_t)gridDim.x * blockDim.x)
        flag[s] = (s == 0 || erow[sorted[s]] != erow[sorted[s - 1]] || sbin[s] != sbin[s - 1]) ? 1 : 0;
}

// per run: first slot, sort key (row, Philox word of the bin), run id; first
// run of each row; *work += the sum over rows of d * (bins of the row), the
// cost of counting the round-robin ranks directly
__global__ void k_bin_run_keys(const int32_t *sorted, const int32_t *erow, const uint32_t *sbin, const int64_t *flag,
                               const int64_t *run_of, const int64_t *rp, int64_t nnz, uint64_t seed, int64_t *run_start,
                               uint64_t *rkey, int64_t *rval, int64_t *row_runs, unsigned long long *work) {
    unsigned long long w = 0;
    for (int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; s < nnz; s += (int64_t)gridDim.x * blockDim.x) {
        if (s == nnz - 1) run_start[run_of[s] + 1] = nnz;   // end of the last run
        if (!flag[s]) continue;
        const int64_t r = run_of[s];
        const int32_t row = erow[sorted[s]];
        run_start[r] = s;
        rkey[r] = ((uint64_t)(uint32_t)row << 32) | bin_word(seed, (uint64_t)row, 1u + sbin[s]);
        rval[r] = r;
        if (s == 0 || erow[sorted[s - 1]] != row) row_runs[row] = r;
        w += (unsigned long long)(rp[row + 1] - rp[row]);
    }
    for (int o = 16; o > 0; o >>= 1) w += __shfl_xor_sync(0xffffffffu, w, o);
    if ((threadIdx.x & 31) == 0 && w) atomicAdd(work, w);
}

// place of each bin in its row's random bin order (rows keep their run ranges in the sorted order)
__global__ void k_bin_order(const uint64_t *rkey, const int64_t *rval, const int64_t *row_runs, int64_t nruns,
                            uint32_t *order) {
    for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < nruns; j += (int64_t)gridDim.x * blockDim.x)
        order[rval[j]] = (uint32_t)(j - row_runs[rkey[j] >> 32]);
}

// The same place counted directly, for rows of few bins: the number of the
// row's bins whose (Philox word, bin) pair is smaller -- the order the stable
// sort of the keys gives.  Threads of one row read the same words.
constexpr unsigned long long kCountOrderMaxBins = 4096;
__global__ void k_bin_run_order(const uint64_t *rkey, const int64_t *row_runs, const int64_t *run_of, const int64_t *rp,
                                int64_t nruns, uint32_t *order) {
    for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < nruns; r += (int64_t)gridDim.x * blockDim.x) {
        const uint64_t kr = rkey[r];
        const int64_t row = (int64_t)(kr >> 32);
        const uint32_t w = (uint32_t)kr;
        const int64_t first = row_runs[row], last = run_of[rp[row + 1] - 1];
        uint32_t c = 0;
        for (int64_t j = first; j <= last; ++j) {
            const uint32_t wj = (uint32_t)__ldg(rkey + j);
            c += (wj < w || (wj == w && j < r)) ? 1u : 0u;
        }
        order[r] = c;
    }
}

// key of the round robin: (index inside the bin, place of the bin)
__global__ void k_bin_key3(const int32_t *sorted, const int64_t *run_of, const int64_t *run_start, const uint32_t *order,
                           int64_t nnz, uint32_t *key) {
    for (int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; s < nnz; s += (int64_t)gridDim.x * blockDim.x) {
        const int64_t r = run_of[s];
        key[sorted[s]] = ((uint32_t)(s - run_start[r]) << kBinOrderBits) | order[r];
    }
}

// The round-robin rank counted directly, for rows of few bins: the entry at
// index k of its bin follows the first min(size, k) entries of every bin of
// its row (rounds 0 .. k-1) and, in round k, the k-th entry of every bin that
// has one and comes earlier in the bin order.
constexpr unsigned long long kCountRankMaxBins = 4096;   // longest loop of one thread
constexpr int64_t kCountRankMaxWork = 64;                 // sum of d * bins per entry
__global__ void k_bin_rr_ranks(const int32_t *sorted, const int32_t *erow, const int64_t *run_of,
                               const int64_t *run_start, const uint32_t *order, const int64_t *row_runs, const int64_t *rp,
                               int64_t nnz, uint32_t *rank) {
    for (int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; s < nnz; s += (int64_t)gridDim.x * blockDim.x) {
        const int32_t e = sorted[s];
        const int64_t r = run_of[s], k = s - run_start[r];
        const int64_t row = erow[e];
        const int64_t first = row_runs[row], last = run_of[rp[row + 1] - 1];
        const uint32_t ob = order[r];
        int64_t acc = 0;
        int64_t a = __ldg(run_start + first);
        for (int64_t j = first; j <= last; ++j) {
            const int64_t b = __ldg(run_start + j + 1), size = b - a;
            acc += size < k ? size : k;
            acc += (size > k && __ldg(order + j) < ob) ? 1 : 0;
            a = b;
        }
        rank[e] = (uint32_t)acc;
    }
}

static ad_status binned_ranks_sorted(ad_graph_t g, const float *score_dev, uint64_t seed, uint32_t *rank_dev,
                                     uint32_t *bin_dev);

// Selection rank of every CSR entry under SparsifyB, written to rank_dev[nnz]
// (device); bin_dev[nnz] (device, may be NULL) receives the bin of every entry.
// score_dev: FP32 distances per edge (device).
ad_status binned_ranks(ad_graph_t g, const float *score_dev, uint64_t seed, uint32_t *rank_dev, uint32_t *bin_dev) {
    const int64_t n = g->n, nnz = g->nnz;
    if (nnz == 0) return AD_OK;
    AD_TRY(ensure_mirror(g));
    AD_TRY(ensure_degree_classes(g));
    const int64_t maxd = g->distinct_degrees.empty() ? 0 : g->distinct_degrees.back();
    if (maxd >= ((int64_t)1 << kRowRankBits) || n >= ((int64_t)1 << 31))
        return binned_ranks_sorted(g, score_dev, seed, rank_dev, bin_dev);
    std::vector<double> cb(std::max<int32_t>(g->n_deg_classes, 1));
    for (int32_t q = 0; q < g->n_deg_classes; ++q) cb[q] = std::cbrt((double)g->distinct_degrees[q]);
    double *cbrt_dc = nullptr, *h = nullptr;
    float *lo = nullptr, *xs = nullptr, *rinv = nullptr;
    uint32_t *bin = nullptr, *key = nullptr, *rk = nullptr, *desc = nullptr, *sbin = nullptr, *order = nullptr,
             *tkey = nullptr;
    int32_t *sorted = nullptr;
    int64_t *flag = nullptr, *run_of = nullptr, *run_start = nullptr, *rval = nullptr, *row_runs = nullptr;
    uint64_t *rkey = nullptr;
    unsigned long long *max_bin = nullptr;
    AD_TRY(dalloc_t(g, cb.size(), &cbrt_dc));
    AD_TRY(dalloc_t(g, n + 1, &lo));
    AD_TRY(dalloc_t(g, n + 1, &h));
    AD_TRY(dalloc_t(g, n + 1, &rinv));
    AD_TRY(dalloc_t(g, nnz, &xs));
    AD_TRY(dalloc_t(g, nnz, &bin));
    AD_TRY(dalloc_t(g, nnz, &key));
    AD_TRY(dalloc_t(g, nnz, &rk));
    AD_TRY(dalloc_t(g, nnz, &desc));
    AD_TRY(dalloc_t(g, 1, &max_bin));
    AD_TRY(copy_in(g, cbrt_dc, cb.data(), cb.size() * sizeof(double)));
    AD_CUDA_TRY(cudaMemsetAsync(max_bin, 0, sizeof(unsigned long long), g->stream));
    const int big = g->num_sms * 16;
    AD_LAUNCH(k_bin_gather, big, 256, 0, g->stream, g->eid, score_dev, nnz, xs);
    AD_LAUNCH(k_bin_stats, (int)std::min<int64_t>((n + 255) / 256, big), 256, 0, g->stream, g->rp, xs, g->deg_class,
              cbrt_dc, n, lo, h, rinv);
    if (maxd > kWarpRowMax) {
        const int64_t *lrows = nullptr;
        int64_t nlong = 0;
        AD_TRY(long_rows(g, &lrows, &nlong));
        AD_LAUNCH(k_bin_stats_big, (int)std::min<int64_t>(nlong, big), kBigRowThreads, 0, g->stream, g->rp, xs,
                  g->deg_class, cbrt_dc, lrows, nlong, lo, h, rinv);
    }
    AD_LAUNCH(k_bin_words, big, 256, 0, g->stream, g->erow, g->eid, xs, lo, h, rinv, nnz, seed, bin, key, max_bin);
    unsigned long long mb = 0;
    AD_TRY(copy_out(g, &mb, max_bin, sizeof(mb)));
    auto release = [&]() {
        for (void *p : {(void *)cbrt_dc, (void *)lo, (void *)h, (void *)rinv, (void *)xs, (void *)bin, (void *)key,
                        (void *)tkey, (void *)rk,
                        (void *)desc, (void *)max_bin, (void *)sbin, (void *)sorted, (void *)flag, (void *)run_of,
                        (void *)run_start, (void *)rval, (void *)row_runs, (void *)rkey, (void *)order})
            if (p) dfree(g, p);
    };
    if (mb >= ((unsigned long long)1 << kBinOrderBits)) {   // (cannot happen below 2^18 entries per row)
        release();
        return binned_ranks_sorted(g, score_dev, seed, rank_dev, bin_dev);
    }
    if (bin_dev) AD_CUDA_TRY(cudaMemcpyAsync(bin_dev, bin, nnz * sizeof(uint32_t), cudaMemcpyDeviceToDevice, g->stream));
    int bbits = 0;                                                          // bits of the largest bin index
    while (((unsigned long long)1 << bbits) <= mb) ++bbits;
    AD_TRY(dalloc_t(g, nnz, &tkey));
    AD_LAUNCH(k_bin_key1, big, 256, 0, g->stream, bin, key, nnz, bbits, tkey);
    AD_TRY(row_ranks(g, tkey, rk, desc));                                  // 1. by (bin, word)
    AD_TRY(dalloc_t(g, nnz, &sorted));
    AD_TRY(dalloc_t(g, nnz, &sbin));
    AD_TRY(dalloc_t(g, nnz, &flag));
    AD_TRY(dalloc_t(g, nnz, &run_of));
    AD_LAUNCH(k_bin_place, big, 256, 0, g->stream, g->erow, g->rp, rk, bin, nnz, sorted, sbin);
    if (bbits > 0) AD_LAUNCH(k_bin_fix_ties, big, 256, 0, g->stream, sorted, g->erow, tkey, key, nnz);
    AD_LAUNCH(k_bin_run_starts, big, 256, 0, g->stream, sorted, g->erow, sbin, nnz, flag);
    int64_t nruns = 0;
    AD_TRY(exclusive_scan_i64(g, flag, run_of, nnz, &nruns));
    AD_LAUNCH(k_bin_inclusive, big, 256, 0, g->stream, flag, nnz, run_of);  // 3. run of every slot
    AD_TRY(dalloc_t(g, nruns + 1, &run_start));
    AD_TRY(dalloc_t(g, nruns + 1, &rkey));
    AD_TRY(dalloc_t(g, nruns + 1, &rval));
    AD_TRY(dalloc_t(g, nruns + 1, &order));
    AD_TRY(dalloc_t(g, n + 1, &row_runs));
    AD_CUDA_TRY(cudaMemsetAsync(max_bin, 0, sizeof(unsigned long long), g->stream));   // reused: direct-rank work
    AD_LAUNCH(k_bin_run_keys, big, 256, 0, g->stream, sorted, g->erow, sbin, flag, run_of, g->rp, nnz, seed, run_start,
              rkey, rval, row_runs, max_bin);
    if (mb < kCountOrderMaxBins) {                                         // 4. bins by word inside each row
        AD_LAUNCH(k_bin_run_order, big, 256, 0, g->stream, rkey, row_runs, run_of, g->rp, nruns, order);
    } else {
        std::vector<int> shifts = {0, 8, 16, 24};
        for (int sh = 32; sh < 64 && ((uint64_t)(n - 1) >> (sh - 32)) != 0; sh += 8) shifts.push_back(sh);
        AD_TRY(radix_sort_pairs(g, rkey, rval, nruns, shifts));
        AD_LAUNCH(k_bin_order, big, 256, 0, g->stream, rkey, rval, row_runs, nruns, order);
    }
    unsigned long long work = 0;
    AD_TRY(copy_out(g, &work, max_bin, sizeof(work)));
    if (mb < kCountRankMaxBins && work <= (unsigned long long)(kCountRankMaxWork * nnz)) {   // 5. round robin
        AD_LAUNCH(k_bin_rr_ranks, big, 256, 0, g->stream, sorted, g->erow, run_of, run_start, order, row_runs, g->rp,
                  nnz, rank_dev);
    } else {
        AD_LAUNCH(k_bin_key3, big, 256, 0, g->stream, sorted, run_of, run_start, order, nnz, key);
        AD_TRY(row_ranks(g, key, rank_dev, desc));
    }
    AD_CUDA_TRY(cudaStreamSynchronize(g->stream));
    release();
    return AD_OK;
}

// The order through two global radix sorts (any row length).
static ad_status binned_ranks_sorted(ad_graph_t g, const float *score_dev, uint64_t seed, uint32_t *rank_dev,
                                     uint32_t *bin_dev) {
    const int64_t n = g->n, nnz = g->nnz;
    if (nnz == 0) return AD_OK;
    if (n >= ((int64_t)1 << (64 - kBinBits))) return fail(AD_ERR_INVALID_ARG, "graph too large for binned ranks");
    AD_TRY(ensure_mirror(g));
    AD_TRY(ensure_degree_classes(g));
    const int64_t maxd = g->distinct_degrees.empty() ? 0 : g->distinct_degrees.back();
    // cbrt of every distinct degree, from the host's FP64 cbrt
    std::vector<double> cb(std::max<int32_t>(g->n_deg_classes, 1));
    for (int32_t q = 0; q < g->n_deg_classes; ++q) cb[q] = std::cbrt((double)g->distinct_degrees[q]);
    double *cbrt_dc = nullptr, *h = nullptr;
    float *lo = nullptr, *xs = nullptr, *rinv = nullptr;
    uint32_t *bin = nullptr, *run_word = nullptr;
    uint64_t *keys = nullptr;
    int64_t *vals = nullptr, *flag = nullptr, *run_of = nullptr, *run_start = nullptr, *row_runs = nullptr;
    unsigned long long *max_bin = nullptr;
    AD_TRY(dalloc_t(g, cb.size(), &cbrt_dc));
    AD_TRY(dalloc_t(g, n + 1, &lo));
    AD_TRY(dalloc_t(g, n + 1, &h));
    AD_TRY(dalloc_t(g, n + 1, &rinv));
    AD_TRY(dalloc_t(g, nnz, &xs));
    AD_TRY(dalloc_t(g, nnz, &bin));
    AD_TRY(dalloc_t(g, nnz, &keys));
    AD_TRY(dalloc_t(g, nnz, &vals));
    AD_TRY(dalloc_t(g, 1, &max_bin));
    AD_TRY(copy_in(g, cbrt_dc, cb.data(), cb.size() * sizeof(double)));
    AD_CUDA_TRY(cudaMemsetAsync(max_bin, 0, sizeof(unsigned long long), g->stream));
    const int big = g->num_sms * 16;
    AD_LAUNCH(k_bin_gather, big, 256, 0, g->stream, g->eid, score_dev, nnz, xs);
    AD_LAUNCH(k_bin_stats, (int)std::min<int64_t>((n + 255) / 256, big), 256, 0, g->stream, g->rp, xs, g->deg_class,
              cbrt_dc, n, lo, h, rinv);
    if (maxd > kWarpRowMax) {
        const int64_t *lrows = nullptr;
        int64_t nlong = 0;
        AD_TRY(long_rows(g, &lrows, &nlong));
        AD_LAUNCH(k_bin_stats_big, (int)std::min<int64_t>(nlong, big), kBigRowThreads, 0, g->stream, g->rp, xs,
                  g->deg_class, cbrt_dc, lrows, nlong, lo, h, rinv);
    }
    AD_LAUNCH(k_bin_entries, big, 256, 0, g->stream, g->erow, g->eid, xs, lo, h, rinv, nnz, seed, bin, keys, vals,
              max_bin);
    unsigned long long mb = 0;
    AD_TRY(copy_out(g, &mb, max_bin, sizeof(mb)));
    if (mb >= (1ull << kBinBits)) return fail(AD_ERR_INVALID_ARG, "too many bins in one row");
    if (bin_dev) AD_CUDA_TRY(cudaMemcpyAsync(bin_dev, bin, nnz * sizeof(uint32_t), cudaMemcpyDeviceToDevice, g->stream));
    AD_TRY(radix_sort_pairs(g, keys, vals, nnz, {0, 8, 16, 24}));            // by Philox word, then position
    AD_LAUNCH(k_bin_rowkeys, big, 256, 0, g->stream, vals, g->erow, bin, nnz, keys);
    std::vector<int> shifts;                                                  // bin bits in use, then row bits
    int bbits = 0;
    while (bbits < kBinBits && (mb >> bbits) != 0) ++bbits;
    int rbits = 0;
    while (rbits < 64 - kBinBits && ((uint64_t)(n - 1) >> rbits) != 0) ++rbits;
    for (int sh = 0; sh < bbits; sh += 8) shifts.push_back(sh);
    for (int sh = kBinBits; sh < kBinBits + rbits; sh += 8) shifts.push_back(sh);
    AD_TRY(radix_sort_pairs(g, keys, vals, nnz, shifts));                     // by (row, bin), stable
    AD_TRY(dalloc_t(g, nnz, &flag));
    AD_TRY(dalloc_t(g, nnz, &run_of));
    AD_LAUNCH(k_bin_run_flags, big, 256, 0, g->stream, keys, nnz, flag);
    int64_t nruns = 0;
    AD_TRY(exclusive_scan_i64(g, flag, run_of, nnz, &nruns));
    AD_TRY(dalloc_t(g, nruns + 1, &run_start));
    AD_TRY(dalloc_t(g, nruns + 1, &run_word));
    AD_TRY(dalloc_t(g, n + 1, &row_runs));
    AD_LAUNCH(k_bin_inclusive, big, 256, 0, g->stream, flag, nnz, run_of);
    AD_LAUNCH(k_bin_runs, big, 256, 0, g->stream, keys, flag, run_of, nnz, seed, run_start, run_word, row_runs);
    AD_LAUNCH(k_bin_ranks, big, 256, 0, g->stream, keys, vals, run_of, run_start, run_word, row_runs, g->rp, nnz, nruns,
              rank_dev);
    AD_CUDA_TRY(cudaStreamSynchronize(g->stream));
    for (void *p : {(void *)cbrt_dc, (void *)lo, (void *)h, (void *)rinv, (void *)xs, (void *)bin, (void *)keys, (void *)vals, (void *)max_bin,
                    (void *)flag, (void *)run_of, (void *)run_start, (void *)run_word, (void *)row_runs})
        dfree(g, p);
    return AD_OK;
}

}  // namespace ad
