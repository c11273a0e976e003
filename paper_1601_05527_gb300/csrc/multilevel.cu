// multilevel.cu -- the multilevel framework of Sec. 5 / Alg. 6 (MLSparsify) on
// the device: seeds (createSeeds), the restriction P of Eq. (P), the Galerkin
// coarse graph L_c = P^T L_f P, uncoarsening of removed edges and the
// recomputation of distances on the sparsified finer graphs.
//
// Seeds.  The sequential rule visits active vertices by decreasing weighted
// degree (ties: smaller id first) and makes i a seed when its weight to the
// seeds chosen before it is <= Q D_i.  Its result is computed exactly in
// parallel rounds: vertex i decides as soon as the states of the neighbours
// that precede it are known well enough -- F when the weight to decided
// seeds already exceeds Q D_i, seed when even all undecided predecessors
// becoming seeds would keep it <= Q D_i.  Decisions are final and match the
// sequential ones; the first undecided vertex in visiting order always
// decides, so the rounds terminate.
#include "ad_internal.cuh"

#include <algorithm>
#include <climits>
#include <cmath>

struct ad_ml_s {
    ad_graph_t g0 = nullptr;
    ad_ml_params p{};
    struct Level {
        ad_graph_t g = nullptr;     // graph of the level (level 0 borrowed from the caller)
        bool owned = false;
        float *rho = nullptr;       // [m] distances computed on the way down
        int32_t *agg = nullptr;     // [n] aggregate in the next coarser level
        int64_t *f2c = nullptr;     // [m] coarse edge of each edge (-1 inside an aggregate)
        // upward trace of the last ad_ml_sparsify call (when tracing is on)
        uint8_t *t_inh = nullptr;   // [m] edges left after the coarser level's removals
        uint8_t *t_keep = nullptr;  // [m] edges kept at this level
        float *t_rho = nullptr;     // [m] distances recomputed on the kept subgraph (NaN: not in it / not recomputed)
    };
    std::vector<Level> lv;
    bool trace = false;
    bool have_trace = false;
};

namespace ad {

// ----------------------------------------------------------------------------
// Seeds
// ----------------------------------------------------------------------------
enum : int8_t { S_UNDECIDED = 0, S_SEED = 1, S_F = 2, S_INACTIVE = 3 };

__global__ void k_seed_init(const double *D, int64_t n, int8_t *state) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        state[i] = D[i] > 0.0 ? S_UNDECIDED : S_INACTIVE;
}

// The sums below are exact in any order on rows whose weights pass the
// exactness bound of the weighted degrees (dexact; unit weights always do), so
// they equal the sequential sums of the definition bit for bit.  On the other
// rows a vertex waits until every predecessor is decided and then sums its
// seed neighbours one after the other in CSR order, as the definition does.
// One round over the vertices still undecided: list[0 .. *len) (list NULL: all
// n vertices).  Vertices that stay undecided are appended to next[]
// (*next_len counts them); their order there does not matter, since a
// decision depends only on the final states of the vertex's predecessors.
__global__ void k_seed_round(const int64_t *rp, const int32_t *col, const float *w, const double *D,
                             const uint8_t *dexact, const int64_t *list, const unsigned long long *len, int64_t n,
                             double Q, int8_t *state, int64_t *next, unsigned long long *next_len) {
    const int lane = threadIdx.x & 31;
    const int64_t W = (int64_t)gridDim.x * (blockDim.x >> 5);
    const int64_t L = list ? (int64_t)*len : n;
    volatile int8_t *vs = state;
    for (int64_t t = blockIdx.x * (int64_t)(blockDim.x >> 5) + (threadIdx.x >> 5); t < L; t += W) {
        const int64_t i = list ? list[t] : t;
        if (vs[i] != S_UNDECIDED) continue;
        const double Di = D[i];
        const bool exact = !w || dexact[i];
        double seed_w = 0.0, und_w = 0.0;
        bool und_any = false;
        for (int64_t p = rp[i] + lane; p < rp[i + 1]; p += 32) {
            const int32_t j = col[p];
            const double Dj = D[j];
            if (Dj > Di || (Dj == Di && j < i)) {          // j is visited before i
                const int8_t sj = vs[j];
                const double wj = w ? (double)w[p] : 1.0;
                if (sj == S_SEED) seed_w += wj;
                else if (sj == S_UNDECIDED) { und_w += wj; und_any = true; }
            }
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            seed_w += __shfl_xor_sync(0xffffffffu, seed_w, o);
            und_w += __shfl_xor_sync(0xffffffffu, und_w, o);
        }
        und_any = __any_sync(0xffffffffu, und_any);
        if (lane == 0) {
            const double lim = Q * Di;
            bool waiting = false;
            if (exact) {
                if (seed_w > lim) vs[i] = S_F;
                else if (seed_w + und_w <= lim) vs[i] = S_SEED;
                else waiting = true;
            } else if (und_any) {
                waiting = true;
            } else {
                double s = 0.0;   // successors may already be decided: only predecessors count
                for (int64_t p = rp[i]; p < rp[i + 1]; ++p) {
                    const int32_t j = col[p];
                    const double Dj = D[j];
                    if ((Dj > Di || (Dj == Di && j < i)) && vs[j] == S_SEED) s += (double)w[p];
                }
                vs[i] = s <= lim ? S_SEED : S_F;
            }
            if (waiting) next[atomicAdd(next_len, 1ull)] = i;
        }
    }
}

// Rounds over the undecided vertices until none is left; the count is read
// back every kSeedRoundsPerCheck rounds (a round on an empty list returns at once).
constexpr int kSeedRoundsPerCheck = 4;
static ad_status create_seeds(ad_graph_t g, double Q, int8_t *state) {
    const int64_t n = g->n;
    if (n == 0) return AD_OK;
    const int grid = g->num_sms * 8;
    AD_LAUNCH(k_seed_init, grid, 256, 0, g->stream, g->D, n, state);
    int64_t *lists = nullptr;
    unsigned long long *lens = nullptr;
    AD_TRY(dalloc_t(g, 2 * (size_t)n, &lists));
    AD_TRY(dalloc_t(g, 2, &lens));
    auto release = [&]() {
        dfree(g, lists);
        dfree(g, lens);
    };
    const int64_t wblocks = std::min<int64_t>((n + 7) / 8 + 1, (int64_t)g->num_sms * 32);
    for (int64_t round = 0;; ++round) {
        if (round > n + kSeedRoundsPerCheck) {
            release();
            return fail(AD_ERR_STATE, "seed selection did not converge");
        }
        const int a = (int)(round & 1), b = a ^ 1;
        AD_CUDA_TRY(cudaMemsetAsync(lens + b, 0, sizeof(unsigned long long), g->stream));
        AD_LAUNCH(k_seed_round, (int)wblocks, 256, 0, g->stream, g->rp, g->col, g->w, g->D, g->dexact,
                  round == 0 ? nullptr : lists + (size_t)a * n, lens + a, n, Q, state, lists + (size_t)b * n, lens + b);
        unsigned long long u = 1;
        if ((round + 1) % kSeedRoundsPerCheck == 0) AD_TRY(copy_out(g, &u, lens + b, sizeof(u)));
        if (u == 0) break;
    }
    release();
    return AD_OK;
}

// ----------------------------------------------------------------------------
// Eq. (P): an F vertex joins the seed neighbour with the largest delta, i.e.
// the smallest rho; ties go to the smaller seed id.
// ----------------------------------------------------------------------------

__global__ void k_seed_flags(const int8_t *state, int64_t n, int64_t *flag) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) flag[i] = state[i] == S_SEED ? 1 : 0;
}

__global__ void k_aggregate(const int64_t *rp, const int32_t *col, const int64_t *eid, const float *score, const int8_t *state, const int64_t *cid,
                            int64_t n, int32_t *agg, unsigned long long *orphans) {
    const int lane = threadIdx.x & 31;
    const int64_t W = (int64_t)gridDim.x * (blockDim.x >> 5);
    for (int64_t i = blockIdx.x * (int64_t)(blockDim.x >> 5) + (threadIdx.x >> 5); i < n; i += W) {
        const int8_t s = state[i];
        if (s != S_F) {
            if (lane == 0) agg[i] = s == S_SEED ? (int32_t)cid[i] : -1;
            continue;
        }
        float best_s = INFINITY;
        int32_t best_j = INT_MAX;
        for (int64_t p = rp[i] + lane; p < rp[i + 1]; p += 32) {
            const int32_t j = col[p];
            if (state[j] != S_SEED) continue;
            const float sc = score[eid[p]];
            if (sc < best_s || (sc == best_s && j < best_j)) { best_s = sc; best_j = j; }
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            const float os = __shfl_xor_sync(0xffffffffu, best_s, o);
            const int32_t oj = __shfl_xor_sync(0xffffffffu, best_j, o);
            if (os < best_s || (os == best_s && oj < best_j)) { best_s = os; best_j = oj; }
        }
        if (lane == 0) {
            if (best_j == INT_MAX) { agg[i] = -1; atomicAdd(orphans, 1ull); }
            else agg[i] = (int32_t)cid[best_j];
        }
    }
}

// ----------------------------------------------------------------------------
// Galerkin coarse graph
// ----------------------------------------------------------------------------
__global__ void k_coarse_pairs(const int64_t *rp, const int32_t *col, const float *w, const int64_t *upos,
                               const int64_t *eoff, const int32_t *agg, int64_t n, uint8_t *inter, uint64_t *key,
                               double *we) {
    const int lane = threadIdx.x & 31;
    const int64_t W = (int64_t)gridDim.x * (blockDim.x >> 5);
    for (int64_t i = blockIdx.x * (int64_t)(blockDim.x >> 5) + (threadIdx.x >> 5); i < n; i += W)
        for (int64_t p = upos[i] + lane; p < rp[i + 1]; p += 32) {
            const int64_t e = eoff[i] + (p - upos[i]);
            const int32_t I = agg[i], J = agg[col[p]];
            inter[e] = (I != J && I >= 0 && J >= 0) ? 1 : 0;
            const uint64_t a = (uint64_t)min(I, J), b = (uint64_t)max(I, J);
            key[e] = (a << 32) | b;
            we[e] = w ? (double)w[p] : 1.0;
        }
}

__global__ void k_gather_keys(const uint64_t *key, const int64_t *idx, int64_t n, uint64_t *out) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t < n) out[t] = key[idx[t]];
}

__global__ void k_first_flags(const uint64_t *key, int64_t n, uint8_t *first) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t < n) first[t] = (t == 0 || key[t] != key[t - 1]) ? 1 : 0;
}

// one thread per coarse edge: FP64 sum of its fine weights in fine-edge order
__global__ void k_segment_sum(const uint64_t *key, const int64_t *fine, const int64_t *seg, int64_t mc, int64_t total,
                              const double *we, int64_t *f2c, int32_t *ca, int32_t *cb, float *cw) {
    const int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= mc) return;
    const int64_t b0 = seg[s], b1 = s + 1 < mc ? seg[s + 1] : total;
    double sum = 0.0;
    for (int64_t t = b0; t < b1; ++t) {
        sum += we[fine[t]];
        f2c[fine[t]] = s;
    }
    ca[s] = (int32_t)(key[b0] >> 32);
    cb[s] = (int32_t)(key[b0] & 0xffffffffu);
    cw[s] = (float)sum;
}

// lanes with the same end add once (ca is sorted, so a warp mostly shares one)
__global__ void k_count_ends(const int32_t *ca, const int32_t *cb, int64_t mc, unsigned long long *cnt_up,
                             unsigned long long *cnt_lo) {
    const int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const unsigned lower = (1u << (threadIdx.x & 31)) - 1u;
    const int32_t a = s < mc ? ca[s] : -1, b = s < mc ? cb[s] : -1;
    const unsigned pa = __match_any_sync(0xffffffffu, a), pb = __match_any_sync(0xffffffffu, b);
    if (a >= 0 && (pa & lower) == 0) atomicAdd(cnt_up + a, (unsigned long long)__popc(pa));
    if (b >= 0 && (pb & lower) == 0) atomicAdd(cnt_lo + b, (unsigned long long)__popc(pb));
}

__global__ void k_add_counts(const unsigned long long *a, const unsigned long long *b, int64_t n, int64_t *out) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] = (int64_t)(a[i] + b[i]);
}

__device__ __forceinline__ int64_t lower_bound_i32(const int32_t *a, int64_t n, int32_t v) {
    int64_t lo = 0, hi = n;
    while (lo < hi) {
        const int64_t mid = (lo + hi) >> 1;
        if (a[mid] < v) lo = mid + 1; else hi = mid;
    }
    return lo;
}
__device__ __forceinline__ int64_t lower_bound_u64(const uint64_t *a, int64_t n, uint64_t v) {
    int64_t lo = 0, hi = n;
    while (lo < hi) {
        const int64_t mid = (lo + hi) >> 1;
        if (a[mid] < v) lo = mid + 1; else hi = mid;
    }
    return lo;
}

// upper entries: row a holds b after its lower entries; the list is sorted by (a, b)
__global__ void k_fill_upper(const int32_t *ca, const int32_t *cb, const float *cw, int64_t mc, const int64_t *rp,
                             const unsigned long long *cnt_lo, int32_t *col, float *w) {
    const int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= mc) return;
    const int32_t a = ca[s];
    const int64_t rank = s - lower_bound_i32(ca, mc, a);
    const int64_t pos = rp[a] + (int64_t)cnt_lo[a] + rank;
    col[pos] = cb[s];
    w[pos] = cw[s];
}

// lower entries: (b, s) pairs sorted stably by b keep a ascending inside each b
__global__ void k_fill_lower(const uint64_t *bkey, const int64_t *sidx, int64_t mc, const int32_t *ca, const float *cw,
                             const int64_t *rp, int32_t *col, float *w) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= mc) return;
    const uint64_t b = bkey[t];
    const int64_t rank = t - lower_bound_u64(bkey, mc, b);
    const int64_t pos = rp[b] + rank;
    col[pos] = ca[sidx[t]];
    w[pos] = cw[sidx[t]];
}

__global__ void k_iota(int64_t *v, int64_t n) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) v[i] = i;
}
__global__ void k_widen_i32_u64(const int32_t *in, int64_t n, uint64_t *out) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] = (uint64_t)(uint32_t)in[i];
}

static std::vector<int> digit_shifts(int64_t maxval, int base) {
    std::vector<int> s;
    int bits = 1;
    while (bits < 62 && ((int64_t)1 << bits) <= maxval) ++bits;
    for (int b = 0; b < bits; b += 8) s.push_back(base + b);
    return s;
}

static inline int nblk(int64_t n) { return (int)((n + 255) / 256 > 0 ? (n + 255) / 256 : 1); }

// Seeds + Eq. (P) + Galerkin for one level.  agg[n] and f2c[m] are device
// arrays owned by g; *coarse receives a new handle (skipped when NULL).
static ad_status coarsen_level(ad_graph_t g, const float *score, double Q, int32_t *agg, int64_t *f2c, int64_t *n_coarse,
                               ad_graph_t *coarse) {
    AD_TRY(ensure_mirror(g));
    const int64_t n = g->n, m = g->m;
    int8_t *state = nullptr;
    int64_t *flag = nullptr, *cid = nullptr;
    unsigned long long *orphans = nullptr;
    AD_TRY(dalloc_t(g, n + 1, &state));
    AD_TRY(create_seeds(g, Q, state));
    AD_TRY(dalloc_t(g, n + 1, &flag));
    AD_TRY(dalloc_t(g, n + 1, &cid));
    AD_TRY(dalloc_t(g, 1, &orphans));
    AD_CUDA_TRY(cudaMemsetAsync(orphans, 0, sizeof(unsigned long long), g->stream));
    if (n > 0) AD_LAUNCH(k_seed_flags, nblk(n), 256, 0, g->stream, state, n, flag);
    int64_t nc = 0;
    AD_TRY(exclusive_scan_i64(g, flag, cid, n, &nc));
    const int64_t wblocks = std::min<int64_t>((n + 7) / 8 + 1, (int64_t)g->num_sms * 32);
    if (n > 0)
        AD_LAUNCH(k_aggregate, (int)wblocks, 256, 0, g->stream, g->rp, g->col, g->eid, score, state, cid, n, agg,
                  orphans);
    unsigned long long orph = 0;
    AD_TRY(copy_out(g, &orph, orphans, sizeof(orph)));
    dfree(g, state);
    dfree(g, flag);
    dfree(g, cid);
    dfree(g, orphans);
    if (orph) return fail(AD_ERR_STATE, std::to_string(orph) + " F vertices without a seed neighbour (Q >= 1?)");
    *n_coarse = nc;
    // ---- Galerkin: sort the inter-aggregate pairs (I < J), sum the weights per pair
    AD_CUDA_TRY(cudaMemsetAsync(f2c, 0xff, (m > 0 ? m : 1) * sizeof(int64_t), g->stream));
    uint8_t *inter = nullptr;
    uint64_t *key = nullptr;
    double *we = nullptr;
    AD_TRY(dalloc_t(g, m + 1, &inter));
    AD_TRY(dalloc_t(g, m + 1, &key));
    AD_TRY(dalloc_t(g, m + 1, &we));
    if (m > 0)
        AD_LAUNCH(k_coarse_pairs, (int)wblocks, 256, 0, g->stream, g->rp, g->col, g->w, g->upos, g->eoff, agg, n, inter,
                  key, we);
    int64_t *fine = nullptr;
    int64_t mi = 0;
    AD_TRY(compact_flags(g, inter, m, &fine, &mi));
    uint64_t *skey = nullptr;
    AD_TRY(dalloc_t(g, mi + 1, &skey));
    if (mi > 0) AD_LAUNCH(k_gather_keys, nblk(mi), 256, 0, g->stream, key, fine, mi, skey);
    std::vector<int> shifts = digit_shifts(nc, 0), hi = digit_shifts(nc, 32);
    shifts.insert(shifts.end(), hi.begin(), hi.end());
    AD_TRY(radix_sort_pairs(g, skey, fine, mi, shifts));
    uint8_t *first = nullptr;
    AD_TRY(dalloc_t(g, mi + 1, &first));
    if (mi > 0) AD_LAUNCH(k_first_flags, nblk(mi), 256, 0, g->stream, skey, mi, first);
    int64_t *seg = nullptr, mc = 0;
    AD_TRY(compact_flags(g, first, mi, &seg, &mc));
    int32_t *ca = nullptr, *cb = nullptr;
    float *cw = nullptr;
    AD_TRY(dalloc_t(g, mc + 1, &ca));
    AD_TRY(dalloc_t(g, mc + 1, &cb));
    AD_TRY(dalloc_t(g, mc + 1, &cw));
    if (mc > 0) AD_LAUNCH(k_segment_sum, nblk(mc), 256, 0, g->stream, skey, fine, seg, mc, mi, we, f2c, ca, cb, cw);
    if (coarse) {
        // ---- coarse symmetric CSR (rows sorted: lower entries, then upper entries)
        unsigned long long *cnt_up = nullptr, *cnt_lo = nullptr;
        int64_t *deg = nullptr, *rpc = nullptr;
        int32_t *colc = nullptr;
        float *wc = nullptr;
        AD_TRY(dalloc_t(g, nc + 1, &cnt_up));
        AD_TRY(dalloc_t(g, nc + 1, &cnt_lo));
        AD_TRY(dalloc_t(g, nc + 1, &deg));
        AD_TRY(dalloc_t(g, nc + 1, &rpc));
        AD_TRY(dalloc_t(g, 2 * mc + 1, &colc));
        AD_TRY(dalloc_t(g, 2 * mc + 1, &wc));
        AD_CUDA_TRY(cudaMemsetAsync(cnt_up, 0, (nc + 1) * sizeof(unsigned long long), g->stream));
        AD_CUDA_TRY(cudaMemsetAsync(cnt_lo, 0, (nc + 1) * sizeof(unsigned long long), g->stream));
        if (mc > 0) AD_LAUNCH(k_count_ends, nblk(mc), 256, 0, g->stream, ca, cb, mc, cnt_up, cnt_lo);
        if (nc > 0) AD_LAUNCH(k_add_counts, nblk(nc), 256, 0, g->stream, cnt_up, cnt_lo, nc, deg);
        int64_t nnzc = 0;
        AD_TRY(exclusive_scan_i64(g, deg, rpc, nc, &nnzc));
        AD_CUDA_TRY(cudaMemcpyAsync(rpc + nc, &nnzc, sizeof(int64_t), cudaMemcpyHostToDevice, g->stream));
        if (mc > 0) {
            AD_LAUNCH(k_fill_upper, nblk(mc), 256, 0, g->stream, ca, cb, cw, mc, rpc, cnt_lo, colc, wc);
            uint64_t *bkey = nullptr;
            int64_t *sidx = nullptr;
            AD_TRY(dalloc_t(g, mc, &bkey));
            AD_TRY(dalloc_t(g, mc, &sidx));
            AD_LAUNCH(k_widen_i32_u64, nblk(mc), 256, 0, g->stream, cb, mc, bkey);
            AD_LAUNCH(k_iota, nblk(mc), 256, 0, g->stream, sidx, mc);
            AD_TRY(radix_sort_pairs(g, bkey, sidx, mc, digit_shifts(nc, 0)));
            AD_LAUNCH(k_fill_lower, nblk(mc), 256, 0, g->stream, bkey, sidx, mc, ca, cw, rpc, colc, wc);
            AD_CUDA_TRY(cudaStreamSynchronize(g->stream));
            dfree(g, bkey);
            dfree(g, sidx);
        }
        AD_TRY(create_like(g, nc, rpc, colc, wc, coarse));
        dfree(g, cnt_up);
        dfree(g, cnt_lo);
        dfree(g, deg);
        dfree(g, rpc);
        dfree(g, colc);
        dfree(g, wc);
    }
    AD_CUDA_TRY(cudaStreamSynchronize(g->stream));
    dfree(g, inter);
    dfree(g, key);
    dfree(g, we);
    if (fine) dfree(g, fine);
    dfree(g, skey);
    dfree(g, first);
    if (seg) dfree(g, seg);
    dfree(g, ca);
    dfree(g, cb);
    dfree(g, cw);
    return AD_OK;
}

// ----------------------------------------------------------------------------
// Uncoarsening and sparsified subgraphs
// ----------------------------------------------------------------------------
__global__ void k_uncoarsen(const int64_t *f2c, const uint8_t *keep_c, int64_t m, uint8_t *keep_f) {
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e < m) keep_f[e] = f2c[e] < 0 ? 1 : keep_c[f2c[e]];
}

__global__ void k_sub_count(const int64_t *rp, const int64_t *eid, const uint8_t *keep, int64_t n, int64_t *cnt) {
    const int lane = threadIdx.x & 31;
    const int64_t W = (int64_t)gridDim.x * (blockDim.x >> 5);
    for (int64_t i = blockIdx.x * (int64_t)(blockDim.x >> 5) + (threadIdx.x >> 5); i < n; i += W) {
        int64_t c = 0;
        for (int64_t p = rp[i] + lane; p < rp[i + 1]; p += 32)
            c += keep[eid[p]] ? 1 : 0;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
        if (lane == 0) cnt[i] = c;
    }
}

__global__ void k_sub_fill(const int64_t *rp, const int32_t *col, const float *w, const int64_t *eid,
                           const uint8_t *keep, int64_t n, const int64_t *rps, int32_t *cols, float *ws) {
    const int lane = threadIdx.x & 31;
    const int64_t W = (int64_t)gridDim.x * (blockDim.x >> 5);
    for (int64_t i = blockIdx.x * (int64_t)(blockDim.x >> 5) + (threadIdx.x >> 5); i < n; i += W) {
        int64_t out = rps[i];
        for (int64_t base = rp[i]; base < rp[i + 1]; base += 32) {
            const int64_t p = base + lane;
            bool k = false;
            if (p < rp[i + 1]) k = keep[eid[p]] != 0;
            const unsigned b = __ballot_sync(0xffffffffu, k);
            if (k) {
                const int64_t q = out + __popc(b & ((1u << lane) - 1u));
                cols[q] = col[p];
                if (ws) ws[q] = w[p];
            }
            out += __popc(b);
        }
    }
}

__global__ void k_scatter_keep(const int64_t *s2f, const uint8_t *ks, int64_t ms, uint8_t *keep) {
    const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (q < ms) keep[s2f[q]] = ks[q];
}

__global__ void k_scatter_f32(const int64_t *s2f, const float *src, int64_t ms, float *dst) {
    const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (q < ms) dst[s2f[q]] = src[q];
}

__global__ void k_fill_nan(float *x, int64_t n) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        x[i] = __int_as_float(0x7fc00000);
}

// trace buffers of one level (allocated on first use, owned by the level's graph)
static ad_status trace_buffers(ad_ml_s::Level &v) {
    ad_graph_t g = v.g;
    if (!v.t_inh) AD_TRY(dalloc_t(g, g->m + 1, &v.t_inh));
    if (!v.t_keep) AD_TRY(dalloc_t(g, g->m + 1, &v.t_keep));
    if (!v.t_rho) AD_TRY(dalloc_t(g, g->m + 1, &v.t_rho));
    if (g->m > 0) AD_LAUNCH(k_fill_nan, std::max<int>(1, (int)std::min<int64_t>((g->m + 255) / 256, 4096)), 256, 0,
                            g->stream, v.t_rho, g->m);
    return AD_OK;
}

__global__ void k_count_u8(const uint8_t *f, int64_t n, unsigned long long *c) {
    unsigned long long s = 0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        s += f[i] ? 1 : 0;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0 && s) atomicAdd(c, s);
}

// Graph of the edges with keep[e] != 0 (same vertices) and the full id of each of its edges.
static ad_status kept_subgraph(ad_graph_t g, const uint8_t *keep, ad_graph_t *sub, int64_t **s2f, int64_t *ms) {
    AD_TRY(ensure_mirror(g));
    const int64_t n = g->n;
    int64_t *cnt = nullptr, *rps = nullptr;
    AD_TRY(dalloc_t(g, n + 1, &cnt));
    AD_TRY(dalloc_t(g, n + 1, &rps));
    const int64_t wblocks = std::min<int64_t>((n + 7) / 8 + 1, (int64_t)g->num_sms * 32);
    if (n > 0)
        AD_LAUNCH(k_sub_count, (int)wblocks, 256, 0, g->stream, g->rp, g->eid, keep, n, cnt);
    int64_t nnz = 0;
    AD_TRY(exclusive_scan_i64(g, cnt, rps, n, &nnz));
    AD_CUDA_TRY(cudaMemcpyAsync(rps + n, &nnz, sizeof(int64_t), cudaMemcpyHostToDevice, g->stream));
    int32_t *cols = nullptr;
    float *ws = nullptr;
    AD_TRY(dalloc_t(g, nnz + 1, &cols));
    if (g->w) AD_TRY(dalloc_t(g, nnz + 1, &ws));
    if (n > 0)
        AD_LAUNCH(k_sub_fill, (int)wblocks, 256, 0, g->stream, g->rp, g->col, g->w, g->eid, keep, n, rps, cols, ws);
    AD_TRY(create_like(g, n, rps, cols, ws, sub));
    AD_TRY(compact_flags(g, keep, g->m, s2f, ms));
    dfree(g, cnt);
    dfree(g, rps);
    dfree(g, cols);
    if (ws) dfree(g, ws);
    return AD_OK;
}

static ad_status count_kept(ad_graph_t g, const uint8_t *keep, int64_t m, int64_t *out) {
    unsigned long long *c = nullptr;
    AD_TRY(dalloc_t(g, 1, &c));
    AD_CUDA_TRY(cudaMemsetAsync(c, 0, sizeof(unsigned long long), g->stream));
    if (m > 0) AD_LAUNCH(k_count_u8, g->num_sms * 8, 256, 0, g->stream, keep, m, c);
    unsigned long long v = 0;
    AD_TRY(copy_out(g, &v, c, sizeof(v)));
    dfree(g, c);
    *out = (int64_t)v;
    return AD_OK;
}

// Upward half of Alg. 6 with per-level keep fractions (index = level, 0 finest;
// < 0 = level not sparsified).  keep0: device array [m_0].
static ad_status ml_upward(ad_ml_t ml, const std::vector<double> &r, uint8_t *keep0, int64_t *kept) {
    const int L = (int)ml->lv.size();
    uint8_t *keep_c = nullptr;
    ad_graph_t owner_c = nullptr;
    for (int l = L - 1; l >= 0; --l) {
        ad_graph_t g = ml->lv[l].g;
        ad_ml_s::Level &tv = ml->lv[l];
        uint8_t *keep = l == 0 ? keep0 : nullptr;
        if (!keep) AD_TRY(dalloc_t(g, g->m + 1, &keep));
        if (ml->trace) AD_TRY(trace_buffers(tv));
        if (l == L - 1) {
            AD_CUDA_TRY(cudaMemsetAsync(keep, 1, g->m > 0 ? g->m : 1, g->stream));
            if (ml->trace && g->m > 0)
                AD_CUDA_TRY(cudaMemcpyAsync(tv.t_inh, keep, g->m, cudaMemcpyDeviceToDevice, g->stream));
            if (r[l] >= 0.0 && g->m > 0) {
                int64_t k = 0;
                double e = 0;
                AD_TRY(select_per_node_fit(g, ml->lv[l].rho, r[l], ml->p.mode, keep, &k, &e));
            }
        } else {
            if (g->m > 0) AD_LAUNCH(k_uncoarsen, nblk(g->m), 256, 0, g->stream, ml->lv[l].f2c, keep_c, g->m, keep);
            if (ml->trace && g->m > 0)
                AD_CUDA_TRY(cudaMemcpyAsync(tv.t_inh, keep, g->m, cudaMemcpyDeviceToDevice, g->stream));
            if (r[l] >= 0.0 && g->m > 0) {
                // ComputeAlgDist(G_f^s), then Sparsify(G_f^s)
                ad_graph_t sub = nullptr;
                int64_t *s2f = nullptr, ms = 0;
                AD_TRY(kept_subgraph(g, keep, &sub, &s2f, &ms));
                ad_status st = AD_OK;
                if (ms > 0) {
                    if (!sub->rho) st = dalloc_t(sub, sub->m + 1, &sub->rho);
                    if (st == AD_OK)
                        st = algebraic_distance(sub, ml->p.R, ml->p.k, ml->p.omega, ml->p.seed, (uint32_t)(2 * l + 1),
                                                ml->p.storage, AD_DIST_PERSISTENT, sub->rho);
                    uint8_t *ks = nullptr;
                    if (st == AD_OK) st = dalloc_t(sub, sub->m + 1, &ks);
                    int64_t k = 0;
                    double e = 0;
                    if (st == AD_OK) st = select_per_node_fit(sub, sub->rho, r[l], ml->p.mode, ks, &k, &e);
                    if (st == AD_OK) {
                        AD_CUDA_TRY(cudaMemsetAsync(keep, 0, g->m, g->stream));
                        AD_CUDA_TRY(cudaStreamSynchronize(sub->stream));
                        AD_LAUNCH(k_scatter_keep, nblk(ms), 256, 0, g->stream, s2f, ks, ms, keep);
                        if (ml->trace) AD_LAUNCH(k_scatter_f32, nblk(ms), 256, 0, g->stream, s2f, sub->rho, ms, tv.t_rho);
                        AD_CUDA_TRY(cudaStreamSynchronize(g->stream));
                    }
                }
                ad_graph_destroy(sub);
                if (s2f) dfree(g, s2f);
                AD_TRY(st);
            }
        }
        if (ml->trace && g->m > 0)
            AD_CUDA_TRY(cudaMemcpyAsync(tv.t_keep, keep, g->m, cudaMemcpyDeviceToDevice, g->stream));
        if (keep_c) dfree(owner_c, keep_c);
        keep_c = l == 0 ? nullptr : keep;
        owner_c = g;
    }
    ml->have_trace = ml->trace;
    return count_kept(ml->lv[0].g, keep0, ml->lv[0].g->m, kept);
}

static void ml_free(ad_ml_t ml) {
    if (!ml) return;
    for (auto &v : ml->lv) {
        if (v.owned) {
            ad_graph_destroy(v.g);
        } else if (v.g) {
            if (v.agg) dfree(v.g, v.agg);
            if (v.f2c) dfree(v.g, v.f2c);
            for (void *b : {(void *)v.t_inh, (void *)v.t_keep, (void *)v.t_rho})
                if (b) dfree(v.g, b);
            // level 0's rho is the handle's own score buffer and stays with it
        }
    }
    delete ml;
}

}  // namespace ad

using namespace ad;

extern "C" ad_status ad_ml_build(ad_graph_t g, const ad_ml_params *params, ad_ml_t *out) {
    if (out) *out = nullptr;
    if (!g || !params || !out) return fail(AD_ERR_INVALID_ARG, "NULL argument");
    const ad_ml_params &p = *params;
    if (p.R < 1 || p.R > 256 || p.k < 0 || !(p.omega > 0.0 && p.omega <= 1.0) || !(p.Q >= 0.0 && p.Q < 1.0) ||
        p.max_levels < 1 || p.max_levels > 64 || p.coarsest_n < 1 || (p.mode != AD_MODE_LOCAL && p.mode != AD_MODE_GLOBAL) ||
        p.storage < AD_STORAGE_FP32 || p.storage > AD_STORAGE_Q16)
        return fail(AD_ERR_INVALID_ARG, "bad multilevel parameters");
    if (g->G != 1) return fail(AD_ERR_INVALID_ARG, "multilevel needs a single graph, not a batch");
    ad_ml_t ml = new ad_ml_s();
    ml->g0 = g;
    ml->p = p;
    ad_graph_t cur = g;
    ad_status st = AD_OK;
    for (int l = 0;; ++l) {
        ad_ml_s::Level lev;
        lev.g = cur;
        lev.owned = l > 0;
        ml->lv.push_back(lev);
        ad_ml_s::Level &v = ml->lv.back();
        if (!cur->rho) { if ((st = dalloc_t(cur, cur->m + 1, &cur->rho)) != AD_OK) break; }
        // every level is relaxed in one persistent launch (init, k sweeps, distances)
        if ((st = algebraic_distance(cur, p.R, p.k, p.omega, p.seed, (uint32_t)(2 * l), p.storage, AD_DIST_PERSISTENT,
                                     cur->rho)) != AD_OK)
            break;
        cur->have_rho = true;
        cur->rho_version++;
        v.rho = cur->rho;
        if (cur->n <= p.coarsest_n || l + 1 >= p.max_levels) break;      // small enough
        if ((st = dalloc_t(cur, cur->n + 1, &v.agg)) != AD_OK) break;
        if ((st = dalloc_t(cur, cur->m + 1, &v.f2c)) != AD_OK) break;
        int64_t nc = 0;
        ad_graph_t coarse = nullptr;
        if ((st = coarsen_level(cur, cur->rho, p.Q, v.agg, v.f2c, &nc, &coarse)) != AD_OK) break;
        if ((double)nc > 0.9 * (double)cur->n) {                         // coarsening stalled
            ad_graph_destroy(coarse);
            dfree(cur, v.agg);
            dfree(cur, v.f2c);
            v.agg = nullptr;
            v.f2c = nullptr;
            break;
        }
        cur = coarse;
    }
    if (st != AD_OK) {
        std::string msg = ad_last_error();
        ml_free(ml);
        set_error(msg);
        return st;
    }
    *out = ml;
    return AD_OK;
}

extern "C" ad_status ad_ml_levels(ad_ml_t ml, int32_t *n_levels) {
    if (!ml || !n_levels) return fail(AD_ERR_INVALID_ARG, "NULL argument");
    *n_levels = (int32_t)ml->lv.size();
    return AD_OK;
}

extern "C" ad_status ad_ml_level_size(ad_ml_t ml, int32_t level, int64_t *n, int64_t *m) {
    if (!ml) return fail(AD_ERR_INVALID_ARG, "NULL hierarchy");
    if (level < 0 || level >= (int32_t)ml->lv.size()) return fail(AD_ERR_INVALID_ARG, "level out of range");
    if (n) *n = ml->lv[level].g->n;
    if (m) *m = ml->lv[level].g->m;
    return AD_OK;
}

// Inspection of one level (see include/ad.h): its graph, the distances of the
// downward pass, and the maps to the next coarser level.
extern "C" ad_status ad_ml_level_export(ad_ml_t ml, int32_t level, int64_t *row_ptr, int32_t *col, float *weight,
                                        int32_t *has_weight, float *rho, int32_t *agg, int64_t *fine_to_coarse) {
    if (!ml) return fail(AD_ERR_INVALID_ARG, "NULL hierarchy");
    if (level < 0 || level >= (int32_t)ml->lv.size()) return fail(AD_ERR_INVALID_ARG, "level out of range");
    const ad_ml_s::Level &v = ml->lv[level];
    ad_graph_t g = v.g;
    if ((agg || fine_to_coarse) && !v.agg) return fail(AD_ERR_STATE, "the coarsest level has no coarser level");
    AD_TRY(ad_graph_export(g, row_ptr, col, weight, has_weight));
    if (rho && g->m > 0) AD_TRY(copy_out(g, rho, v.rho, g->m * sizeof(float)));
    if (agg && g->n > 0) AD_TRY(copy_out(g, agg, v.agg, g->n * sizeof(int32_t)));
    if (fine_to_coarse && g->m > 0) AD_TRY(copy_out(g, fine_to_coarse, v.f2c, g->m * sizeof(int64_t)));
    return AD_OK;
}

extern "C" ad_status ad_ml_set_trace(ad_ml_t ml, int32_t enable) {
    if (!ml) return fail(AD_ERR_INVALID_ARG, "NULL hierarchy");
    ml->trace = enable != 0;
    return AD_OK;
}

extern "C" ad_status ad_ml_level_trace(ad_ml_t ml, int32_t level, uint8_t *inherited, uint8_t *kept, float *rho_up) {
    if (!ml) return fail(AD_ERR_INVALID_ARG, "NULL hierarchy");
    if (level < 0 || level >= (int32_t)ml->lv.size()) return fail(AD_ERR_INVALID_ARG, "level out of range");
    if (!ml->have_trace) return fail(AD_ERR_STATE, "no traced ad_ml_sparsify call");
    const ad_ml_s::Level &v = ml->lv[level];
    ad_graph_t g = v.g;
    if (g->m == 0) return AD_OK;
    if (inherited) AD_TRY(copy_out(g, inherited, v.t_inh, g->m));
    if (kept) AD_TRY(copy_out(g, kept, v.t_keep, g->m));
    if (rho_up) AD_TRY(copy_out(g, rho_up, v.t_rho, g->m * sizeof(float)));
    return AD_OK;
}

extern "C" ad_status ad_ml_sparsify(ad_ml_t ml, const double *ratios, int32_t n_ratios, double target_fraction,
                                    uint8_t *keep_out, int64_t *n_kept, double *r_used) {
    if (!ml || !ratios) return fail(AD_ERR_INVALID_ARG, "NULL argument");
    const int L = (int)ml->lv.size();
    if (n_ratios != L) return fail(AD_ERR_INVALID_ARG, "need one ratio per level (" + std::to_string(L) + ")");
    for (int t = 0; t < L; ++t)
        if (std::isnan(ratios[t]) || ratios[t] > 1.0) return fail(AD_ERR_INVALID_ARG, "ratios must be <= 1");
    if (std::isnan(target_fraction) || target_fraction > 1.0)
        return fail(AD_ERR_INVALID_ARG, "target_fraction must be <= 1");
    ad_graph_t g0 = ml->lv[0].g;
    if (!keep_out && g0->m > 0) return fail(AD_ERR_INVALID_ARG, "keep_out is NULL");
    const bool dev_out = is_device_ptr(keep_out);
    uint8_t *kd = keep_out;
    if (!dev_out) AD_TRY(dalloc_t(g0, g0->m + 16, &kd));
    std::vector<double> r(L);
    int64_t kept = 0;
    double used = -1.0;
    ad_status st = AD_OK;
    if (target_fraction < 0.0) {
        for (int l = 0; l < L; ++l) r[l] = ratios[L - 1 - l];
        st = ml_upward(ml, r, kd, &kept);
    } else {
        const int64_t K = (int64_t)std::floor(target_fraction * (double)g0->m + 0.5);
        double lo = 0.0, hi = 1.0;
        for (int it = 0; it < 20 && st == AD_OK; ++it) {
            const double mid = 0.5 * (lo + hi);
            for (int l = 0; l < L; ++l) r[l] = ratios[L - 1 - l] >= 0.0 ? mid : -1.0;
            int64_t c = 0;
            st = ml_upward(ml, r, kd, &c);
            if (c >= K) hi = mid; else lo = mid;
        }
        if (st == AD_OK) {
            for (int l = 0; l < L; ++l) r[l] = ratios[L - 1 - l] >= 0.0 ? hi : -1.0;
            st = ml_upward(ml, r, kd, &kept);
            used = hi;
        }
    }
    if (st == AD_OK && !dev_out) st = copy_out(g0, keep_out, kd, g0->m);
    if (!dev_out) dfree(g0, kd);
    AD_TRY(st);
    if (n_kept) *n_kept = kept;
    if (r_used) *r_used = used;
    return AD_OK;
}

// MLSparsify(G_f, ratios) of Alg. 6 in one call: the downward half
// (ad_ml_build), the upward half with the ratio vector (ad_ml_sparsify) and
// the release of the hierarchy.  ratios[l] belongs to the l-th coarsest level;
// levels past the end of the vector are not sparsified.
extern "C" ad_status ad_multilevel(ad_graph_t g, const ad_ml_params *params, const double *ratios, int32_t n_ratios,
                                   double target_fraction, uint8_t *keep_out, int32_t *n_levels_out) {
    if (!g || !params) return fail(AD_ERR_INVALID_ARG, "NULL argument");
    if (n_ratios < 0 || (n_ratios > 0 && !ratios)) return fail(AD_ERR_INVALID_ARG, "bad ratio vector");
    for (int32_t t = 0; t < n_ratios; ++t)
        if (std::isnan(ratios[t]) || ratios[t] > 1.0) return fail(AD_ERR_INVALID_ARG, "ratios must be <= 1");
    if (std::isnan(target_fraction) || target_fraction > 1.0)
        return fail(AD_ERR_INVALID_ARG, "target_fraction must be <= 1");
    if (!keep_out && g->m > 0) return fail(AD_ERR_INVALID_ARG, "keep_out is NULL");
    ad_ml_t ml = nullptr;
    AD_TRY(ad_ml_build(g, params, &ml));
    const int32_t L = (int32_t)ml->lv.size();
    std::vector<double> r(L, -1.0);
    for (int32_t l = 0; l < L && l < n_ratios; ++l) r[l] = ratios[l];
    const ad_status st = ad_ml_sparsify(ml, r.data(), L, target_fraction, keep_out, nullptr, nullptr);
    ad_ml_destroy(ml);
    if (st == AD_OK && n_levels_out) *n_levels_out = L;
    return st;
}

extern "C" ad_status ad_ml_segment_ratios(int32_t n_levels, int32_t segment, int32_t level_span, double value,
                                          double *ratios_out) {
    if (n_levels < 1 || level_span < 1 || segment < 1 || segment > 3 || !ratios_out)
        return fail(AD_ERR_INVALID_ARG, "bad segment arguments");
    const int32_t s = level_span < n_levels ? level_span : n_levels;
    const int32_t start = segment == 1 ? 0 : (segment == 2 ? (n_levels - s) / 2 : n_levels - s);
    for (int32_t t = 0; t < n_levels; ++t) ratios_out[t] = (t >= start && t < start + s) ? value : -1.0;
    return AD_OK;
}

extern "C" ad_status ad_ml_destroy(ad_ml_t ml) {
    ml_free(ml);
    return AD_OK;
}

extern "C" ad_status ad_coarsen(ad_graph_t g, const float *score, double Q, int32_t *agg_out, int64_t *n_coarse,
                                ad_graph_t *coarse_out, int64_t *fine_to_coarse_out) {
    if (coarse_out) *coarse_out = nullptr;
    if (!g) return fail(AD_ERR_INVALID_ARG, "NULL graph");
    if (!(Q >= 0.0 && Q < 1.0)) return fail(AD_ERR_INVALID_ARG, "Q must be in [0, 1)");
    if (g->G != 1) return fail(AD_ERR_INVALID_ARG, "coarsening needs a single graph");
    const float *sd = g->rho;
    float *tmp_s = nullptr;
    if (score) {
        if (is_device_ptr(score)) sd = score;
        else {
            AD_TRY(dalloc_t(g, g->m + 1, &tmp_s));
            AD_TRY(copy_in(g, tmp_s, score, g->m * sizeof(float)));
            sd = tmp_s;
        }
        AD_TRY(check_scores(g, sd));
    } else if (!g->have_rho) {
        return fail(AD_ERR_STATE, "no distances: call ad_algebraic_distance first or pass scores");
    }
    int32_t *agg = nullptr;
    int64_t *f2c = nullptr;
    AD_TRY(dalloc_t(g, g->n + 1, &agg));
    AD_TRY(dalloc_t(g, g->m + 1, &f2c));
    int64_t nc = 0;
    AD_TRY(coarsen_level(g, sd, Q, agg, f2c, &nc, coarse_out));
    if (agg_out) AD_TRY(copy_out(g, agg_out, agg, g->n * sizeof(int32_t)));
    if (fine_to_coarse_out) AD_TRY(copy_out(g, fine_to_coarse_out, f2c, g->m * sizeof(int64_t)));
    if (n_coarse) *n_coarse = nc;
    dfree(g, agg);
    dfree(g, f2c);
    if (tmp_s) dfree(g, tmp_s);
    return AD_OK;
}
