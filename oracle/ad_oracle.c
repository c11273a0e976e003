/*
 * ad_oracle.c -- plain FP64 CPU oracle for sparsification by algebraic distance
 * (John & Safro, "Single- and Multi-level Network Sparsification by Algebraic
 * Distance", arXiv 1601.05527).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the slow, obviously-correct
 * definition that the CUDA path is checked against.  Only the test suite, the
 * smoke check and the CPU-baseline leg of the benchmark may load it; the
 * product library never links, calls or falls back to it.  It shares no code,
 * header, table or helper with the CUDA sources.
 *
 * Every quantity is IEEE double.  Loops follow the paper's statement order:
 *   - Alg. 1 (ComputeAlgDist): test vectors r outermost, k JOR sweeps each,
 *     rescale, accumulate (x_i - x_j)^2, distance = sqrt of the sum.
 *   - Alg. 2 (Sparsify): per node, sort incident edges by algebraic distance,
 *     keep the top ceil(d_i^e) of them, union over nodes.
 *   - Sec. 5 / Alg. 6 (MLSparsify): seeds, restriction P of Eq. (P), Galerkin
 *     coarse graph P^T L P, recursion, uncoarsening, recomputed distances.
 *
 * Readings of points the paper leaves open (each one is also listed in the
 * design notes of the repository):
 *   R1  Damping.  The paper writes x <- alpha x + (1-alpha) avg (Alg. 1).
 *       Callers pass alpha; the CUDA library takes omega = 1 - alpha.
 *   R2  Random init.  rand(-0.5, 0.5) of Alg. 1 is the half-open grid value
 *       (u >> 8) * 2^-24 - 0.5 of a Philox4x32-10 word (Salmon et al., SC'11),
 *       counter = (i_lo, i_hi, r / 4, stream), key = (seed_lo, seed_hi),
 *       word r % 4.  Exactly representable in binary32 and binary64.
 *   R3  Rescale.  Alg. 1 rescales once after the k sweeps; the per-sweep form
 *       rescales after every sweep.  Both are provided (they agree in exact
 *       arithmetic because the JOR operator commutes with affine maps of a
 *       vector).  Rescale maps [lo, hi] onto [-0.5, 0.5]; when hi == lo the
 *       vector becomes 0.
 *   R4  Vertices of degree 0 take no part: never updated, never in min/max.
 *   R5  The returned edge score is rho = sqrt(R_ij), the L2 distance over the
 *       test vectors.  delta = 1/sqrt(R_ij + eps) of Alg. 1 is a strictly
 *       decreasing function of rho, so "sort by delta descending" is "sort by
 *       rho ascending".  Optional normalisation (last line of Alg. 1) divides
 *       delta by sqrt(D_i D_j) (weighted degrees); with eps = 0 that is the
 *       score rho * sqrt(D_i D_j).
 *   R6  Ties in every ordering are broken by ascending edge id; edge ids
 *       enumerate the pairs (i < j) in CSR row-major order.
 *   R7  "top d_i^e" of Alg. 2 is T(d, e) = min(d, max(1, ceil(d^e - 1e-9))).
 *   R8  A target edge fraction f is met by bisection on e (Sec. 6.2 fits e by
 *       binary search): K = floor(f m + 1/2), 40 halvings of [0, 1], result =
 *       the upper end, the smallest grid point whose kept count is >= K.
 *   R9  Seeds (Sec. 5 "The Coarsening"): visit active vertices by decreasing
 *       weighted degree (ties: smaller id first) and move i to C when the
 *       weight from i to the seeds chosen so far is <= Q * D_i.  The paper
 *       states no coupling rule, so parity with its own hierarchy is
 *       unpinned; this rule is pinned by the condition that determines it.
 *   R10 Eq. (P): an F vertex joins the seed neighbour of largest delta, that
 *       is smallest rho; ties go to the smaller seed id.  Coarse ids number
 *       the seeds by increasing vertex id.
 *   R11 Coarsening stops when n_c <= coarsest_n, when n_c > 0.9 n_f, or at
 *       max_levels.  The coarsest level is sparsified with Alg. 2 (SparsifyB
 *       of Alg. 3 is cut off in the text).
 *   R12 Level ratios (Alg. 6 input, Sec. 6 example): index 0 is the coarsest
 *       level, -1 means no sparsification at that level, otherwise the value
 *       is the fraction of that level's current edges to keep, met by fitting
 *       e with the bisection of R8.  Philox stream of level l is 2l on
 *       the way down and 2l+1 for the recomputation on the way up.  A span
 *       of levels in the middle of L levels starts floor((L - span) / 2)
 *       levels from the coarsest (the paper's example has L - span even).
 *   R13 SparsifyB (Alg. 3; its text stops mid-sentence).  Per node, sigma is
 *       the population standard deviation of its incident distances; the bin
 *       width is h = 3.5 sigma / cbrt(d) and the bin of a distance is
 *       floor((rho - min) / h) (one bin when sigma = 0).  "Randomly select
 *       bins and edges up to d^e" is read as a stratified draw: entries of a
 *       bin in random order, bins in random order, then round robin over the
 *       bins until T(d, e) entries are taken (reading R7), so every bin
 *       contributes before any contributes twice.  Random order = ascending
 *       word 0 of Philox4x32-10 with key = the selection seed and counter
 *       (edge id lo, hi, 0, 0xB1000000) for an entry, (vertex lo, hi, 1 + bin,
 *       0xB1000000) for a bin; ties by position / bin index.  Mean, sigma,
 *       h and the bin index are FP64, sums sequential in CSR order.  Union
 *       over the two ends of an edge and the fit of e are those of Alg. 2 (R8).
 *   R14 Local Degree (the comparison method of Sec. 1.1 and Sec. 6): node i
 *       ranks its neighbours by their degree, largest first, ties by CSR
 *       position (smaller id first), and keeps the first T(d_i, e) (R7);
 *       union and fit of e as Alg. 2 (R8).
 *   R15 Reverse mode: L = sum over a subset S of rho_e^2 through the
 *       per-sweep form; the min and max of each rescale take their
 *       sub-gradient at the lowest-index argmin / argmax.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <math.h>
#include <time.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_OK 0
#define ORC_ERR_ARG 1
#define ORC_ERR_OOM 2

/* ------------------------------------------------------------------------ */
/* Threads.  Built with OpenMP, the loops over rows of Alg. 1 run on several */
/* host threads; every row is still computed by one thread with the same     */
/* operations in the same order, so results do not depend on the thread      */
/* count (min / max reductions are exact).                                   */
/* ------------------------------------------------------------------------ */
void orc_set_threads(int32_t n)
{
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
#else
    (void)n;
#endif
}

int32_t orc_max_threads(void)
{
#ifdef _OPENMP
    return (int32_t)omp_get_max_threads();
#else
    return 1;
#endif
}

/* Wall-clock seconds of the phases of the last orc_algebraic_distance call:
 * [0] degrees and init, [1] the k sweeps with their rescales, [2] distances. */
static double g_phase_s[3];

void orc_last_phase_seconds(double out[3])
{
    out[0] = g_phase_s[0]; out[1] = g_phase_s[1]; out[2] = g_phase_s[2];
}

static double now_s(void)
{
    struct timespec ts;
    clock_gettime(CLOCK_MONOTONIC, &ts);
    return (double)ts.tv_sec + 1e-9 * (double)ts.tv_nsec;
}

/* ------------------------------------------------------------------------ */
/* Philox4x32-10, from the definition in Salmon, Moraes, Dror, Shaw,        */
/* "Parallel Random Numbers: As Easy as 1, 2, 3" (SC'11): ten rounds of     */
/* two 32x32->64 multiplies, key schedule bumped by the Weyl constants.     */
/* ------------------------------------------------------------------------ */
void orc_philox4x32_10(const uint32_t ctr_in[4], const uint32_t key_in[2], uint32_t out[4])
{
    const uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u;
    const uint32_t W0 = 0x9E3779B9u, W1 = 0xBB67AE85u;
    uint32_t c0 = ctr_in[0], c1 = ctr_in[1], c2 = ctr_in[2], c3 = ctr_in[3];
    uint32_t k0 = key_in[0], k1 = key_in[1];
    for (int round = 0; round < 10; ++round) {
        if (round > 0) { k0 += W0; k1 += W1; }
        uint64_t p0 = (uint64_t)M0 * (uint64_t)c0;
        uint64_t p1 = (uint64_t)M1 * (uint64_t)c2;
        uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        uint32_t n0 = hi1 ^ c1 ^ k0;
        uint32_t n1 = lo1;
        uint32_t n2 = hi0 ^ c3 ^ k1;
        uint32_t n3 = lo0;
        c0 = n0; c1 = n1; c2 = n2; c3 = n3;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/* x_i^r at iteration 0 (Alg. 1, "x_i <- rand(-0.5, 0.5)"), reading R2. */
double orc_test_value(uint64_t seed, uint32_t stream, int64_t i, int32_t r)
{
    uint32_t ctr[4], key[2], out[4];
    ctr[0] = (uint32_t)((uint64_t)i & 0xffffffffu);
    ctr[1] = (uint32_t)((uint64_t)i >> 32);
    ctr[2] = (uint32_t)(r / 4);
    ctr[3] = stream;
    key[0] = (uint32_t)(seed & 0xffffffffu);
    key[1] = (uint32_t)(seed >> 32);
    orc_philox4x32_10(ctr, key, out);
    uint32_t u = out[r % 4];
    return (double)(u >> 8) * (1.0 / 16777216.0) - 0.5;
}

/* All initial test vectors, layout x[i * R + r]. */
void orc_init_vectors(int64_t n, int32_t R, uint64_t seed, uint32_t stream, double *x)
{
    for (int64_t i = 0; i < n; ++i)
        for (int32_t r = 0; r < R; ++r)
            x[i * R + r] = orc_test_value(seed, stream, i, r);
}

/* ------------------------------------------------------------------------ */
/* Graph helpers.  G = (V, E, w): undirected, no self loops, no multi-edges */
/* (Sec. 2).  Stored as a symmetric CSR with sorted columns.                */
/* ------------------------------------------------------------------------ */

/* Number of undirected edges = CSR entries with col > row. */
int64_t orc_count_edges(int64_t n, const int64_t *rp, const int32_t *ci)
{
    int64_t m = 0;
    for (int64_t i = 0; i < n; ++i)
        for (int64_t p = rp[i]; p < rp[i + 1]; ++p)
            if (ci[p] > i) ++m;
    return m;
}

/* Edge list in edge-id order (reading R6): e-th pair (eu[e] < ev[e]). */
void orc_edge_list(int64_t n, const int64_t *rp, const int32_t *ci, int32_t *eu, int32_t *ev)
{
    int64_t e = 0;
    for (int64_t i = 0; i < n; ++i)
        for (int64_t p = rp[i]; p < rp[i + 1]; ++p)
            if (ci[p] > i) { eu[e] = (int32_t)i; ev[e] = ci[p]; ++e; }
}

/* Position of column j in row i (binary search; rows are sorted), or -1. */
static int64_t find_entry(const int64_t *rp, const int32_t *ci, int64_t i, int32_t j)
{
    int64_t lo = rp[i], hi = rp[i + 1];
    while (lo < hi) {
        int64_t mid = lo + (hi - lo) / 2;
        if (ci[mid] < j) lo = mid + 1; else hi = mid;
    }
    return (lo < rp[i + 1] && ci[lo] == j) ? lo : -1;
}

/* Edge id of every CSR entry (both directions of an edge share one id). */
void orc_entry_edge_ids(int64_t n, const int64_t *rp, const int32_t *ci, int64_t *eid)
{
    int64_t e = 0;
    for (int64_t i = 0; i < n; ++i)
        for (int64_t p = rp[i]; p < rp[i + 1]; ++p) {
            int32_t j = ci[p];
            if (j > i) eid[p] = e++;
            else eid[p] = eid[find_entry(rp, ci, j, (int32_t)i)];  /* row j < i already numbered */
        }
}

/* Weighted degree D_i = sum_j w_ij, the denominator of the JOR update (Alg. 1). */
void orc_weighted_degree(int64_t n, const int64_t *rp, const double *w, double *D)
{
    for (int64_t i = 0; i < n; ++i) {
        double s = 0.0;
        for (int64_t p = rp[i]; p < rp[i + 1]; ++p) s += (w ? w[p] : 1.0);
        D[i] = s;
    }
}

/* Rescale one vector back to (-0.5, 0.5) over the active vertices (R3, R4). */
static void rescale_vector(int64_t n, const double *D, double *x)
{
    double lo = INFINITY, hi = -INFINITY;
#pragma omp parallel for reduction(min:lo) reduction(max:hi) schedule(static)
    for (int64_t i = 0; i < n; ++i) {
        if (!(D[i] > 0.0)) continue;
        if (x[i] < lo) lo = x[i];
        if (x[i] > hi) hi = x[i];
    }
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; ++i) {
        if (!(D[i] > 0.0)) continue;
        x[i] = (hi > lo) ? (x[i] - lo) / (hi - lo) - 0.5 : 0.0;
    }
}

/*
 * ComputeAlgDist (Alg. 1).
 *   alpha          JOR damping of Alg. 1 (omega = 1 - alpha)
 *   rescale_mode   0: rescale after every sweep; 1: once after the k sweeps
 *   normalize      0: score rho; 1: rho * sqrt(D_i D_j) (optional last line)
 *   x0             optional [n][R] initial vectors replacing the Philox init
 *   x_final        optional [n][R] output: the rescaled vectors after sweep k
 *   rho            [m] output, edge-id order
 */
int orc_algebraic_distance(int64_t n, const int64_t *rp, const int32_t *ci, const double *w,
                           int32_t R, int32_t k, double alpha, uint64_t seed, uint32_t stream,
                           int32_t rescale_mode, int32_t normalize,
                           const double *x0, double *x_final, double *rho)
{
    if (n < 0 || R < 1 || k < 0) return ORC_ERR_ARG;
    const double t0 = now_s();
    double t_sweeps = 0.0, t_dist = 0.0, t_init = 0.0;
    int64_t m = orc_count_edges(n, rp, ci);
    double *D = (double *)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
    double *x = (double *)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
    double *y = (double *)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
    double *acc = (double *)calloc((size_t)(m > 0 ? m : 1), sizeof(double));
    int64_t *e0 = (int64_t *)malloc(sizeof(int64_t) * (size_t)(n + 1));   /* first edge id of row i */
    if (!D || !x || !y || !acc || !e0) { free(D); free(x); free(y); free(acc); free(e0); return ORC_ERR_OOM; }
    orc_weighted_degree(n, rp, w, D);
    e0[0] = 0;
    for (int64_t i = 0; i < n; ++i) {
        int64_t up = 0;
        for (int64_t p = rp[i]; p < rp[i + 1]; ++p) up += ci[p] > i;
        e0[i + 1] = e0[i] + up;
    }
    t_init += now_s() - t0;

    for (int64_t e = 0; e < m; ++e) acc[e] = 0.0;                       /* R_ij = 0 */
    for (int32_t r = 0; r < R; ++r) {                                   /* test vectors */
        double ta = now_s();
#pragma omp parallel for schedule(static)
        for (int64_t i = 0; i < n; ++i)                                 /* x <- rand */
            x[i] = x0 ? x0[i * R + r] : orc_test_value(seed, stream, i, r);
        double tb = now_s();
        t_init += tb - ta;
        for (int32_t t = 0; t < k; ++t) {                               /* JOR sweeps */
#pragma omp parallel for schedule(dynamic, 1024)
            for (int64_t i = 0; i < n; ++i) {
                if (!(D[i] > 0.0)) { y[i] = x[i]; continue; }
                double s = 0.0;
                for (int64_t p = rp[i]; p < rp[i + 1]; ++p)
                    s += (w ? w[p] : 1.0) * x[ci[p]];
                y[i] = alpha * x[i] + (1.0 - alpha) * s / D[i];
            }
            double *tmp = x; x = y; y = tmp;
            if (rescale_mode == 0) rescale_vector(n, D, x);
        }
        if (rescale_mode == 1) rescale_vector(n, D, x);                 /* rescale back */
        ta = now_s();
        t_sweeps += ta - tb;
        if (x_final)
            for (int64_t i = 0; i < n; ++i) x_final[i * R + r] = x[i];
#pragma omp parallel for schedule(dynamic, 1024)
        for (int64_t i = 0; i < n; ++i) {                               /* R_ij += (x_i-x_j)^2 */
            int64_t e = e0[i];
            for (int64_t p = rp[i]; p < rp[i + 1]; ++p)
                if (ci[p] > i) { double d = x[i] - x[ci[p]]; acc[e] += d * d; ++e; }
        }
        t_dist += now_s() - ta;
    }
    const double tc = now_s();
#pragma omp parallel for schedule(dynamic, 1024)
    for (int64_t i = 0; i < n; ++i) {
        int64_t e = e0[i];
        for (int64_t p = rp[i]; p < rp[i + 1]; ++p)
            if (ci[p] > i) {
                double s = sqrt(acc[e]);
                if (normalize) s *= sqrt(D[i] * D[ci[p]]);
                rho[e] = s;
                ++e;
            }
    }
    t_dist += now_s() - tc;
    g_phase_s[0] = t_init;
    g_phase_s[1] = t_sweeps;
    g_phase_s[2] = t_dist;
    free(D); free(x); free(y); free(acc); free(e0);
    return ORC_OK;
}

/* ------------------------------------------------------------------------ */
/* Ranking and sampling (Sec. 4, Alg. 2).                                    */
/* mode 0 "local": keep delta-strong edges = ascending rho.                  */
/* mode 1 "global": keep delta-weak edges = descending rho.  Ties: edge id.  */
/* ------------------------------------------------------------------------ */
typedef struct { double s; int64_t e; } scored_edge;

static int cmp_ascending(const void *a, const void *b)
{
    const scored_edge *x = (const scored_edge *)a, *y = (const scored_edge *)b;
    if (x->s < y->s) return -1;
    if (x->s > y->s) return 1;
    return (x->e < y->e) ? -1 : (x->e > y->e);
}

static int cmp_descending(const void *a, const void *b)
{
    const scored_edge *x = (const scored_edge *)a, *y = (const scored_edge *)b;
    if (x->s > y->s) return -1;
    if (x->s < y->s) return 1;
    return (x->e < y->e) ? -1 : (x->e > y->e);
}

/* Whole-graph ranking: keep the first K edges of the mode's order. */
int64_t orc_select_whole_graph(int64_t m, const double *score, int32_t mode, int64_t K, uint8_t *keep)
{
    scored_edge *a = (scored_edge *)malloc(sizeof(scored_edge) * (size_t)(m > 0 ? m : 1));
    if (!a) return -1;
    for (int64_t e = 0; e < m; ++e) { a[e].s = score[e]; a[e].e = e; keep[e] = 0; }
    qsort(a, (size_t)m, sizeof(scored_edge), mode ? cmp_descending : cmp_ascending);
    if (K > m) K = m;
    for (int64_t t = 0; t < K; ++t) keep[a[t].e] = 1;
    free(a);
    return K;
}

/* Number of edges node of degree d keeps at exponent e (reading R7). */
int64_t orc_degree_target(int64_t d, double e)
{
    if (d <= 0) return 0;
    double t = ceil(pow((double)d, e) - 1e-9);
    if (t < 1.0) t = 1.0;
    if (t > (double)d) t = (double)d;
    return (int64_t)t;
}

/* Per node: incident edge ids in the mode's order (the sort of Alg. 2). */
static int sort_incidence(int64_t n, const int64_t *rp, const int32_t *ci, const double *score,
                          int32_t mode, int64_t *sorted_e)
{
    int64_t nnz = rp[n];
    int64_t *eid = (int64_t *)malloc(sizeof(int64_t) * (size_t)(nnz > 0 ? nnz : 1));
    if (!eid) return ORC_ERR_OOM;
    orc_entry_edge_ids(n, rp, ci, eid);
    int64_t maxd = 0;
    for (int64_t i = 0; i < n; ++i) if (rp[i + 1] - rp[i] > maxd) maxd = rp[i + 1] - rp[i];
    scored_edge *a = (scored_edge *)malloc(sizeof(scored_edge) * (size_t)(maxd > 0 ? maxd : 1));
    if (!a) { free(eid); return ORC_ERR_OOM; }
    for (int64_t i = 0; i < n; ++i) {
        int64_t d = rp[i + 1] - rp[i];
        for (int64_t t = 0; t < d; ++t) { a[t].e = eid[rp[i] + t]; a[t].s = score[a[t].e]; }
        qsort(a, (size_t)d, sizeof(scored_edge), mode ? cmp_descending : cmp_ascending);
        for (int64_t t = 0; t < d; ++t) sorted_e[rp[i] + t] = a[t].e;
    }
    free(a); free(eid);
    return ORC_OK;
}

/* Add the top T(d_i, e) edges of every node; returns the size of the union. */
static int64_t union_of_tops(int64_t n, const int64_t *rp, const int64_t *sorted_e, int64_t m,
                             double e, uint8_t *keep)
{
    for (int64_t q = 0; q < m; ++q) keep[q] = 0;
    for (int64_t i = 0; i < n; ++i) {
        int64_t T = orc_degree_target(rp[i + 1] - rp[i], e);
        for (int64_t t = 0; t < T; ++t) keep[sorted_e[rp[i] + t]] = 1;
    }
    int64_t c = 0;
    for (int64_t q = 0; q < m; ++q) c += keep[q];
    return c;
}

/* Sparsify(G) of Alg. 2 at a given exponent e.  Returns |E_sparse|. */
int64_t orc_select_per_node(int64_t n, const int64_t *rp, const int32_t *ci, const double *score,
                            int32_t mode, double e, uint8_t *keep)
{
    int64_t nnz = rp[n], m = orc_count_edges(n, rp, ci);
    int64_t *sorted_e = (int64_t *)malloc(sizeof(int64_t) * (size_t)(nnz > 0 ? nnz : 1));
    if (!sorted_e) return -1;
    if (sort_incidence(n, rp, ci, score, mode, sorted_e) != ORC_OK) { free(sorted_e); return -1; }
    int64_t c = union_of_tops(n, rp, sorted_e, m, e, keep);
    free(sorted_e);
    return c;
}

/* K = floor(f m + 1/2) (reading R8). */
int64_t orc_target_count(int64_t m, double fraction)
{
    return (int64_t)floor(fraction * (double)m + 0.5);
}

/*
 * Sparsify to a target fraction.  scope 0 = per node (Alg. 2, e bisected,
 * reading R8); scope 1 = whole graph (one global ranking, keep K).
 */
int orc_sparsify(int64_t n, const int64_t *rp, const int32_t *ci, const double *score,
                 int32_t mode, int32_t scope, double fraction, uint8_t *keep,
                 int64_t *n_kept, double *e_used)
{
    if (fraction < 0.0 || fraction > 1.0) return ORC_ERR_ARG;
    int64_t m = orc_count_edges(n, rp, ci);
    int64_t K = orc_target_count(m, fraction);
    if (scope == 1) {
        *n_kept = orc_select_whole_graph(m, score, mode, K, keep);
        *e_used = -1.0;
        return *n_kept < 0 ? ORC_ERR_OOM : ORC_OK;
    }
    int64_t nnz = rp[n];
    int64_t *sorted_e = (int64_t *)malloc(sizeof(int64_t) * (size_t)(nnz > 0 ? nnz : 1));
    if (!sorted_e) return ORC_ERR_OOM;
    if (sort_incidence(n, rp, ci, score, mode, sorted_e) != ORC_OK) { free(sorted_e); return ORC_ERR_OOM; }
    double lo = 0.0, hi = 1.0;
    for (int it = 0; it < 40; ++it) {
        double mid = 0.5 * (lo + hi);
        if (union_of_tops(n, rp, sorted_e, m, mid, keep) >= K) hi = mid; else lo = mid;
    }
    *n_kept = union_of_tops(n, rp, sorted_e, m, hi, keep);
    *e_used = hi;
    free(sorted_e);
    return ORC_OK;
}

/* ------------------------------------------------------------------------ */
/* Alg. 3 (SparsifyB): per node, the incident distances are put into bins    */
/* whose width follows the rule quoted in Sec. 4, h = 3.5 sigma / d^(1/3),   */
/* and edges are drawn from all bins (reading R13).                          */
/* ------------------------------------------------------------------------ */
#define ORC_BIN_STREAM 0xB1000000u

static uint32_t bin_word(uint64_t seed, uint64_t a, uint32_t z)
{
    const uint32_t ctr[4] = {(uint32_t)a, (uint32_t)(a >> 32), z, ORC_BIN_STREAM};
    const uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    uint32_t out[4];
    orc_philox4x32_10(ctr, key, out);
    return out[0];
}

typedef struct { int64_t bin; uint32_t u; int64_t t; } binned_entry;

static int cmp_binned(const void *a, const void *b)
{
    const binned_entry *x = (const binned_entry *)a, *y = (const binned_entry *)b;
    if (x->bin != y->bin) return x->bin < y->bin ? -1 : 1;
    if (x->u != y->u) return x->u < y->u ? -1 : 1;
    return (x->t < y->t) ? -1 : (x->t > y->t);
}

typedef struct { uint32_t v; int64_t bin; } bin_key;

static int cmp_bin_key(const void *a, const void *b)
{
    const bin_key *x = (const bin_key *)a, *y = (const bin_key *)b;
    if (x->v != y->v) return x->v < y->v ? -1 : 1;
    return (x->bin < y->bin) ? -1 : (x->bin > y->bin);
}

/*
 * Selection rank of every CSR entry under SparsifyB; node i keeps its entries
 * of rank < T(d_i, e).  For row i with distances rho_1..rho_d (CSR order):
 *   mean and sigma (population) by sequential FP64 sums in CSR order;
 *   sigma == 0: one bin; else h = 3.5 sigma / cbrt(d), bin = floor((rho - min) / h),
 *   all in FP64;
 *   entries of a bin in order of (Philox word of the edge id, position);
 *   bins in order of (Philox word of (i, 1 + bin), bin);
 *   selection order = round robin over the bins: round r takes the r-th entry
 *   of every bin that has one, bins in their order.
 * bin (nullable) receives the bin of every CSR entry.  Returns ORC_OK or ORC_ERR_OOM.
 */
int orc_binned_ranks(int64_t n, const int64_t *rp, const int32_t *ci, const double *score, uint64_t seed,
                     int64_t *rank, int64_t *bin)
{
    int64_t nnz = rp[n];
    int64_t *eid = (int64_t *)malloc(sizeof(int64_t) * (size_t)(nnz > 0 ? nnz : 1));
    int64_t maxd = 0;
    for (int64_t i = 0; i < n; ++i) if (rp[i + 1] - rp[i] > maxd) maxd = rp[i + 1] - rp[i];
    size_t md = (size_t)(maxd > 0 ? maxd : 1);
    binned_entry *a = (binned_entry *)malloc(sizeof(binned_entry) * md);
    bin_key *bk = (bin_key *)malloc(sizeof(bin_key) * md);
    int64_t *size = (int64_t *)malloc(sizeof(int64_t) * md);
    int64_t *order = (int64_t *)malloc(sizeof(int64_t) * md);   /* position of a bin in the bin order */
    int64_t *within = (int64_t *)malloc(sizeof(int64_t) * md);
    if (!eid || !a || !bk || !size || !order || !within) {
        free(eid); free(a); free(bk); free(size); free(order); free(within);
        return ORC_ERR_OOM;
    }
    orc_entry_edge_ids(n, rp, ci, eid);
    for (int64_t i = 0; i < n; ++i) {
        const int64_t p0 = rp[i], d = rp[i + 1] - p0;
        if (d == 0) continue;
        double sum = 0.0, lo = score[eid[p0]], hi = lo;
        for (int64_t t = 0; t < d; ++t) {
            const double x = score[eid[p0 + t]];
            sum += x;
            if (x < lo) lo = x;
            if (x > hi) hi = x;
        }
        const double mean = sum / (double)d;
        double q = 0.0;
        for (int64_t t = 0; t < d; ++t) {
            const double dx = score[eid[p0 + t]] - mean;
            q += dx * dx;
        }
        const double sigma = sqrt(q / (double)d);
        const double h = 3.5 * sigma / cbrt((double)d);
        int64_t nbins = 1;
        for (int64_t t = 0; t < d; ++t) {
            int64_t b = 0;
            if (sigma > 0.0 && hi > lo) b = (int64_t)floor((score[eid[p0 + t]] - lo) / h);
            a[t].bin = b;
            a[t].u = bin_word(seed, (uint64_t)eid[p0 + t], 0u);
            a[t].t = t;
            if (b + 1 > nbins) nbins = b + 1;
        }
        qsort(a, (size_t)d, sizeof(binned_entry), cmp_binned);
        for (int64_t b = 0; b < nbins; ++b) size[b] = 0;
        for (int64_t s = 0; s < d; ++s) {
            within[s] = size[a[s].bin];
            size[a[s].bin] += 1;
        }
        for (int64_t b = 0; b < nbins; ++b) {
            bk[b].v = bin_word(seed, (uint64_t)i, (uint32_t)(1 + b));
            bk[b].bin = b;
        }
        qsort(bk, (size_t)nbins, sizeof(bin_key), cmp_bin_key);
        for (int64_t o = 0; o < nbins; ++o) order[bk[o].bin] = o;
        for (int64_t s = 0; s < d; ++s) {
            const int64_t r = within[s], b = a[s].bin;
            int64_t rk = 0;
            for (int64_t c = 0; c < nbins; ++c) {
                rk += size[c] < r ? size[c] : r;                 /* entries of earlier rounds */
                if (size[c] > r && order[c] < order[b]) ++rk;   /* this round, earlier bins */
            }
            rank[p0 + a[s].t] = rk;
            if (bin) bin[p0 + a[s].t] = b;
        }
    }
    free(eid); free(a); free(bk); free(size); free(order); free(within);
    return ORC_OK;
}

/* SparsifyB to a target fraction: e bisected as in orc_sparsify (reading R8). */
int orc_sparsify_binned(int64_t n, const int64_t *rp, const int32_t *ci, const double *score, uint64_t seed,
                        double fraction, uint8_t *keep, int64_t *n_kept, double *e_used)
{
    if (fraction < 0.0 || fraction > 1.0) return ORC_ERR_ARG;
    int64_t m = orc_count_edges(n, rp, ci), nnz = rp[n];
    int64_t K = orc_target_count(m, fraction);
    int64_t *rank = (int64_t *)malloc(sizeof(int64_t) * (size_t)(nnz > 0 ? nnz : 1));
    int64_t *eid = (int64_t *)malloc(sizeof(int64_t) * (size_t)(nnz > 0 ? nnz : 1));
    int64_t *sorted_e = (int64_t *)malloc(sizeof(int64_t) * (size_t)(nnz > 0 ? nnz : 1));
    if (!rank || !eid || !sorted_e) { free(rank); free(eid); free(sorted_e); return ORC_ERR_OOM; }
    if (orc_binned_ranks(n, rp, ci, score, seed, rank, NULL) != ORC_OK) {
        free(rank); free(eid); free(sorted_e);
        return ORC_ERR_OOM;
    }
    orc_entry_edge_ids(n, rp, ci, eid);
    for (int64_t i = 0; i < n; ++i)   /* ranks of a row are 0 .. d-1: the row in selection order */
        for (int64_t p = rp[i]; p < rp[i + 1]; ++p) sorted_e[rp[i] + rank[p]] = eid[p];
    double lo = 0.0, hi = 1.0;
    for (int it = 0; it < 40; ++it) {
        double mid = 0.5 * (lo + hi);
        if (union_of_tops(n, rp, sorted_e, m, mid, keep) >= K) hi = mid; else lo = mid;
    }
    *n_kept = union_of_tops(n, rp, sorted_e, m, hi, keep);
    *e_used = hi;
    free(rank); free(eid); free(sorted_e);
    return ORC_OK;
}

/* ------------------------------------------------------------------------ */
/* Local Degree, the comparison method of Sec. 6 (Lindner et al.): node i    */
/* keeps the edges to its T(d_i, e) neighbours of largest degree (ties: the  */
/* smaller neighbour id, i.e. CSR position); union and fit of e as Alg. 2.   */
/* ------------------------------------------------------------------------ */
typedef struct { int64_t d; int64_t t; int64_t e; } ld_entry;

static int cmp_ld(const void *a, const void *b)
{
    const ld_entry *x = (const ld_entry *)a, *y = (const ld_entry *)b;
    if (x->d != y->d) return x->d > y->d ? -1 : 1;
    return (x->t < y->t) ? -1 : (x->t > y->t);
}

int orc_sparsify_local_degree(int64_t n, const int64_t *rp, const int32_t *ci, double fraction, uint8_t *keep,
                              int64_t *n_kept, double *e_used)
{
    if (fraction < 0.0 || fraction > 1.0) return ORC_ERR_ARG;
    int64_t m = orc_count_edges(n, rp, ci), nnz = rp[n];
    int64_t K = orc_target_count(m, fraction);
    int64_t maxd = 0;
    for (int64_t i = 0; i < n; ++i) if (rp[i + 1] - rp[i] > maxd) maxd = rp[i + 1] - rp[i];
    int64_t *eid = (int64_t *)malloc(sizeof(int64_t) * (size_t)(nnz > 0 ? nnz : 1));
    int64_t *sorted_e = (int64_t *)malloc(sizeof(int64_t) * (size_t)(nnz > 0 ? nnz : 1));
    ld_entry *a = (ld_entry *)malloc(sizeof(ld_entry) * (size_t)(maxd > 0 ? maxd : 1));
    if (!eid || !sorted_e || !a) { free(eid); free(sorted_e); free(a); return ORC_ERR_OOM; }
    orc_entry_edge_ids(n, rp, ci, eid);
    for (int64_t i = 0; i < n; ++i) {
        const int64_t d = rp[i + 1] - rp[i];
        for (int64_t t = 0; t < d; ++t) {
            const int32_t j = ci[rp[i] + t];
            a[t].d = rp[j + 1] - rp[j];
            a[t].t = t;
            a[t].e = eid[rp[i] + t];
        }
        qsort(a, (size_t)d, sizeof(ld_entry), cmp_ld);
        for (int64_t t = 0; t < d; ++t) sorted_e[rp[i] + t] = a[t].e;
    }
    double lo = 0.0, hi = 1.0;
    for (int it = 0; it < 40; ++it) {
        double mid = 0.5 * (lo + hi);
        if (union_of_tops(n, rp, sorted_e, m, mid, keep) >= K) hi = mid; else lo = mid;
    }
    *n_kept = union_of_tops(n, rp, sorted_e, m, hi, keep);
    *e_used = hi;
    free(eid); free(sorted_e); free(a);
    return ORC_OK;
}

/* ------------------------------------------------------------------------ */
/* Multilevel framework (Sec. 5, Alg. 6).                                    */
/* ------------------------------------------------------------------------ */

typedef struct { double D; int64_t i; } vertex_by_degree;

static int cmp_degree_desc(const void *a, const void *b)
{
    const vertex_by_degree *x = (const vertex_by_degree *)a, *y = (const vertex_by_degree *)b;
    if (x->D > y->D) return -1;
    if (x->D < y->D) return 1;
    return (x->i < y->i) ? -1 : (x->i > y->i);
}

/* createSeeds (Sec. 5 "The Coarsening", reading R9).  is_seed[i] in {0,1}. */
int orc_create_seeds(int64_t n, const int64_t *rp, const int32_t *ci, const double *w, double Q,
                     uint8_t *is_seed)
{
    double *D = (double *)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
    vertex_by_degree *order = (vertex_by_degree *)malloc(sizeof(vertex_by_degree) * (size_t)(n > 0 ? n : 1));
    if (!D || !order) { free(D); free(order); return ORC_ERR_OOM; }
    orc_weighted_degree(n, rp, w, D);
    int64_t na = 0;
    for (int64_t i = 0; i < n; ++i) {
        is_seed[i] = 0;
        if (D[i] > 0.0) { order[na].D = D[i]; order[na].i = i; ++na; }
    }
    qsort(order, (size_t)na, sizeof(vertex_by_degree), cmp_degree_desc);
    for (int64_t t = 0; t < na; ++t) {                 /* traversal of F */
        int64_t i = order[t].i;
        double to_seeds = 0.0;
        for (int64_t p = rp[i]; p < rp[i + 1]; ++p)
            if (is_seed[ci[p]]) to_seeds += (w ? w[p] : 1.0);
        if (to_seeds <= Q * D[i]) is_seed[i] = 1;     /* not strongly coupled to C */
    }
    free(D); free(order);
    return ORC_OK;
}

/*
 * Restriction P of Eq. (P), order-1 interpolation (reading R10).
 * score[e] = rho of edge e.  agg[i] = coarse id of i's aggregate, -1 for
 * inactive vertices.  Returns n_c = |C|, or -1 if an F vertex has no seed
 * neighbour (impossible for seeds from orc_create_seeds with Q < 1).
 */
int64_t orc_aggregate(int64_t n, const int64_t *rp, const int32_t *ci, const double *score,
                      const uint8_t *is_seed, int32_t *agg)
{
    int64_t nnz = rp[n];
    int64_t *eid = (int64_t *)malloc(sizeof(int64_t) * (size_t)(nnz > 0 ? nnz : 1));
    if (!eid) return -1;
    orc_entry_edge_ids(n, rp, ci, eid);
    int64_t nc = 0;
    for (int64_t i = 0; i < n; ++i) agg[i] = is_seed[i] ? (int32_t)(nc++) : -1;   /* I_c */
    for (int64_t i = 0; i < n; ++i) {
        if (is_seed[i] || rp[i + 1] == rp[i]) continue;
        int64_t best = -1;
        double best_s = 0.0;
        for (int64_t p = rp[i]; p < rp[i + 1]; ++p) {
            int32_t j = ci[p];
            if (!is_seed[j]) continue;
            double s = score[eid[p]];
            if (best < 0 || s < best_s || (s == best_s && j < best)) { best = j; best_s = s; }
        }
        if (best < 0) { free(eid); return -1; }
        agg[i] = agg[best];
    }
    free(eid);
    return nc;
}

typedef struct { int32_t a, b; int64_t fe; double w; } coarse_pair;

static int cmp_pair(const void *x_, const void *y_)
{
    const coarse_pair *x = (const coarse_pair *)x_, *y = (const coarse_pair *)y_;
    if (x->a != y->a) return x->a < y->a ? -1 : 1;
    if (x->b != y->b) return x->b < y->b ? -1 : 1;
    return (x->fe < y->fe) ? -1 : (x->fe > y->fe);
}

/*
 * Galerkin coarse graph L_c = P^T L_f P (Sec. 5).  Off-diagonal coarse
 * weight W_c[I,J] = sum of w_pq over fine edges with agg(p)=I, agg(q)=J;
 * edges inside an aggregate vanish.  Outputs a symmetric sorted CSR
 * (rp_c[n_c+1], ci_c, w_c with capacity nnz_f) and, for each fine edge,
 * the coarse edge id it is bundled into (-1 inside an aggregate).
 * Returns nnz_c, or -1 on failure.
 */
int64_t orc_galerkin(int64_t n, const int64_t *rp, const int32_t *ci, const double *w,
                     const int32_t *agg, int64_t nc,
                     int64_t *rp_c, int32_t *ci_c, double *w_c, int64_t *fine_to_coarse)
{
    int64_t m = orc_count_edges(n, rp, ci);
    coarse_pair *pairs = (coarse_pair *)malloc(sizeof(coarse_pair) * (size_t)(m > 0 ? m : 1));
    if (!pairs) return -1;
    int64_t np = 0, e = 0;
    for (int64_t i = 0; i < n; ++i)
        for (int64_t p = rp[i]; p < rp[i + 1]; ++p) {
            int32_t j = ci[p];
            if (j <= i) continue;
            int32_t I = agg[i], J = agg[j];
            if (I == J) { fine_to_coarse[e] = -1; }
            else {
                pairs[np].a = I < J ? I : J; pairs[np].b = I < J ? J : I;
                pairs[np].fe = e; pairs[np].w = w ? w[p] : 1.0; ++np;
            }
            ++e;
        }
    qsort(pairs, (size_t)np, sizeof(coarse_pair), cmp_pair);
    /* unique coarse edges in (a, b) order = coarse edge ids */
    int64_t mc = 0;
    int32_t *ua = (int32_t *)malloc(sizeof(int32_t) * (size_t)(np > 0 ? np : 1));
    int32_t *ub = (int32_t *)malloc(sizeof(int32_t) * (size_t)(np > 0 ? np : 1));
    double *uw = (double *)malloc(sizeof(double) * (size_t)(np > 0 ? np : 1));
    if (!ua || !ub || !uw) { free(pairs); free(ua); free(ub); free(uw); return -1; }
    for (int64_t t = 0; t < np; ++t) {
        if (t == 0 || pairs[t].a != pairs[t - 1].a || pairs[t].b != pairs[t - 1].b) {
            ua[mc] = pairs[t].a; ub[mc] = pairs[t].b; uw[mc] = 0.0; ++mc;
        }
        uw[mc - 1] += pairs[t].w;
        fine_to_coarse[pairs[t].fe] = mc - 1;
    }
    /* symmetric CSR: row I holds J for both (I,J) and (J,I), sorted by J */
    for (int64_t I = 0; I <= nc; ++I) rp_c[I] = 0;
    for (int64_t t = 0; t < mc; ++t) { rp_c[ua[t] + 1]++; rp_c[ub[t] + 1]++; }
    for (int64_t I = 0; I < nc; ++I) rp_c[I + 1] += rp_c[I];
    int64_t *fill = (int64_t *)malloc(sizeof(int64_t) * (size_t)(nc > 0 ? nc : 1));
    if (!fill) { free(pairs); free(ua); free(ub); free(uw); return -1; }
    for (int64_t I = 0; I < nc; ++I) fill[I] = rp_c[I];
    /* Lower entries (J < I) of row I come from pairs (J, I), visited in J order;
       upper entries from pairs (I, J) in J order.  Two passes keep rows sorted. */
    for (int64_t t = 0; t < mc; ++t) {          /* lower part of row b: column a */
        int32_t I = ub[t];
        ci_c[fill[I]] = ua[t]; w_c[fill[I]] = uw[t]; fill[I]++;
    }
    for (int64_t t = 0; t < mc; ++t) {          /* upper part of row a: column b */
        int32_t I = ua[t];
        ci_c[fill[I]] = ub[t]; w_c[fill[I]] = uw[t]; fill[I]++;
    }
    int64_t nnz_c = rp_c[nc];
    free(pairs); free(ua); free(ub); free(uw); free(fill);
    return nnz_c;
}

/* Uncoarsening (Sec. 5): a fine edge bundled into a removed coarse edge is removed. */
void orc_uncoarsen(int64_t m_f, const int64_t *fine_to_coarse, const uint8_t *keep_c, uint8_t *keep_f)
{
    for (int64_t e = 0; e < m_f; ++e)
        keep_f[e] = (fine_to_coarse[e] < 0) ? 1 : keep_c[fine_to_coarse[e]];
}

/* Subgraph with the kept edges only (same vertex set), weights carried over. */
static int64_t kept_subgraph(int64_t n, const int64_t *rp, const int32_t *ci, const double *w,
                             const uint8_t *keep, int64_t *rp_s, int32_t *ci_s, double *w_s,
                             int64_t *sub_to_full /* [m_s] */)
{
    int64_t nnz = rp[n];
    int64_t *eid = (int64_t *)malloc(sizeof(int64_t) * (size_t)(nnz > 0 ? nnz : 1));
    if (!eid) return -1;
    orc_entry_edge_ids(n, rp, ci, eid);
    int64_t q = 0, es = 0;
    rp_s[0] = 0;
    for (int64_t i = 0; i < n; ++i) {
        for (int64_t p = rp[i]; p < rp[i + 1]; ++p) {
            if (!keep[eid[p]]) continue;
            ci_s[q] = ci[p]; w_s[q] = w ? w[p] : 1.0; ++q;
            if (ci[p] > i) sub_to_full[es++] = eid[p];
        }
        rp_s[i + 1] = q;
    }
    free(eid);
    return es;
}

typedef struct {
    int64_t n, m;
    int64_t *rp; int32_t *ci; double *w;
    double *rho;              /* distances computed on the way down */
    int32_t *agg;             /* to the next coarser level (NULL at the coarsest) */
    int64_t *f2c;             /* fine edge -> coarse edge id */
} orc_level;

typedef struct {
    int32_t L;
    orc_level lv[64];
    int32_t R, k; double alpha; uint64_t seed; int32_t mode;
} orc_ml;

void orc_ml_free(orc_ml *h)
{
    if (!h) return;
    for (int l = 0; l < h->L; ++l) {
        orc_level *v = &h->lv[l];
        if (l > 0) { free(v->rp); free(v->ci); free(v->w); }
        free(v->rho); free(v->agg); free(v->f2c);
    }
    free(h);
}

/*
 * Downward half of Alg. 6: ComputeAlgDist at each level, seeds, P, Galerkin,
 * until the graph is small enough (reading R11).  The input arrays are
 * borrowed for level 0 and must outlive the handle.
 */
orc_ml *orc_ml_build(int64_t n, const int64_t *rp, const int32_t *ci, const double *w,
                     int32_t R, int32_t k, double alpha, uint64_t seed, double Q,
                     int64_t coarsest_n, int32_t max_levels, int32_t mode)
{
    if (max_levels < 1 || max_levels > 64) return NULL;
    orc_ml *h = (orc_ml *)calloc(1, sizeof(orc_ml));
    if (!h) return NULL;
    h->R = R; h->k = k; h->alpha = alpha; h->seed = seed; h->mode = mode;
    int64_t cn = n; int64_t *crp = (int64_t *)rp; int32_t *cci = (int32_t *)ci; double *cw = (double *)w;
    for (int32_t l = 0; ; ++l) {
        orc_level *v = &h->lv[l];
        v->n = cn; v->rp = crp; v->ci = cci; v->w = cw;
        v->m = orc_count_edges(cn, crp, cci);
        h->L = l + 1;
        v->rho = (double *)malloc(sizeof(double) * (size_t)(v->m > 0 ? v->m : 1));
        if (!v->rho) goto fail;
        if (orc_algebraic_distance(cn, crp, cci, cw, R, k, alpha, seed, (uint32_t)(2 * l),
                                   0, 0, NULL, NULL, v->rho) != ORC_OK) goto fail;
        if (cn <= coarsest_n || l + 1 >= max_levels) break;               /* small enough */
        uint8_t *is_seed = (uint8_t *)malloc((size_t)(cn > 0 ? cn : 1));
        v->agg = (int32_t *)malloc(sizeof(int32_t) * (size_t)(cn > 0 ? cn : 1));
        if (!is_seed || !v->agg) { free(is_seed); goto fail; }
        if (orc_create_seeds(cn, crp, cci, cw, Q, is_seed) != ORC_OK) { free(is_seed); goto fail; }
        int64_t nc = orc_aggregate(cn, crp, cci, v->rho, is_seed, v->agg);
        free(is_seed);
        if (nc < 0) goto fail;
        if ((double)nc > 0.9 * (double)cn) { free(v->agg); v->agg = NULL; break; }   /* stall */
        int64_t nnz = crp[cn];
        int64_t *rpc = (int64_t *)malloc(sizeof(int64_t) * (size_t)(nc + 1));
        int32_t *cic = (int32_t *)malloc(sizeof(int32_t) * (size_t)(nnz > 0 ? nnz : 1));
        double *wc = (double *)malloc(sizeof(double) * (size_t)(nnz > 0 ? nnz : 1));
        v->f2c = (int64_t *)malloc(sizeof(int64_t) * (size_t)(v->m > 0 ? v->m : 1));
        if (!rpc || !cic || !wc || !v->f2c) { free(rpc); free(cic); free(wc); goto fail; }
        if (orc_galerkin(cn, crp, cci, cw, v->agg, nc, rpc, cic, wc, v->f2c) < 0) {
            free(rpc); free(cic); free(wc); goto fail;
        }
        cn = nc; crp = rpc; cci = cic; cw = wc;
    }
    return h;
fail:
    orc_ml_free(h);
    return NULL;
}

int32_t orc_ml_levels(const orc_ml *h) { return h->L; }
void orc_ml_level_size(const orc_ml *h, int32_t l, int64_t *n, int64_t *m)
{
    *n = h->lv[l].n; *m = h->lv[l].m;
}

/*
 * Upward half of Alg. 6 for per-level keep fractions r_by_level[l]
 * (index = level, 0 finest; -1 = no sparsification at that level).  A
 * sparsified level keeps floor(r m_s + 1/2) of its m_s current edges, with
 * e fitted per level as in orc_sparsify (reading R8).  Writes keep0[m_0]
 * and returns its count, or -1.
 */
static int64_t ml_upward(const orc_ml *h, const double *r_by_level, uint8_t *keep0)
{
    int32_t L = h->L;
    uint8_t *keep_c = NULL;
    for (int32_t l = L - 1; l >= 0; --l) {
        const orc_level *v = &h->lv[l];
        uint8_t *keep = (uint8_t *)malloc((size_t)(v->m > 0 ? v->m : 1));
        if (!keep) { free(keep_c); return -1; }
        int64_t kept; double e_used;
        if (l == L - 1) {
            for (int64_t e = 0; e < v->m; ++e) keep[e] = 1;
            if (r_by_level[l] >= 0.0 &&                                      /* coarsest level */
                orc_sparsify(v->n, v->rp, v->ci, v->rho, h->mode, 0, r_by_level[l], keep,
                             &kept, &e_used) != ORC_OK) {
                free(keep); return -1;
            }
        } else {
            orc_uncoarsen(v->m, v->f2c, keep_c, keep);                       /* Uncoarsen */
            if (r_by_level[l] >= 0.0) {
                /* ComputeAlgDist(G_f^s), then Sparsify(G_f^s) */
                int64_t nnz = v->rp[v->n];
                int64_t *rps = (int64_t *)malloc(sizeof(int64_t) * (size_t)(v->n + 1));
                int32_t *cis = (int32_t *)malloc(sizeof(int32_t) * (size_t)(nnz > 0 ? nnz : 1));
                double *ws = (double *)malloc(sizeof(double) * (size_t)(nnz > 0 ? nnz : 1));
                int64_t *s2f = (int64_t *)malloc(sizeof(int64_t) * (size_t)(v->m > 0 ? v->m : 1));
                double *rhos = (double *)malloc(sizeof(double) * (size_t)(v->m > 0 ? v->m : 1));
                uint8_t *ks = (uint8_t *)malloc((size_t)(v->m > 0 ? v->m : 1));
                int ok = rps && cis && ws && s2f && rhos && ks;
                int64_t ms = ok ? kept_subgraph(v->n, v->rp, v->ci, v->w, keep, rps, cis, ws, s2f) : -1;
                ok = ok && ms >= 0 &&
                     orc_algebraic_distance(v->n, rps, cis, ws, h->R, h->k, h->alpha, h->seed,
                                            (uint32_t)(2 * l + 1), 0, 0, NULL, NULL, rhos) == ORC_OK &&
                     orc_sparsify(v->n, rps, cis, rhos, h->mode, 0, r_by_level[l], ks,
                                  &kept, &e_used) == ORC_OK;
                if (ok) {
                    for (int64_t e = 0; e < v->m; ++e) keep[e] = 0;
                    for (int64_t q = 0; q < ms; ++q) keep[s2f[q]] = ks[q];
                }
                free(rps); free(cis); free(ws); free(s2f); free(rhos); free(ks);
                if (!ok) { free(keep); free(keep_c); return -1; }
            }
        }
        free(keep_c);
        keep_c = keep;
    }
    int64_t c = 0;
    for (int64_t e = 0; e < h->lv[0].m; ++e) { keep0[e] = keep_c[e]; c += keep_c[e]; }
    free(keep_c);
    return c;
}

/*
 * MLSparsify with a vector of sparsification ratios (reading R12:
 * ratios[0] = coarsest level, n_ratios must equal the number of levels,
 * -1 = level not sparsified).  With target_fraction < 0 each ratio is that
 * level's keep fraction.  Otherwise every level with a ratio >= 0 uses one
 * shared keep fraction r, fitted by 20 halvings of [0, 1] to the smallest
 * grid point whose final count is >= floor(f m_0 + 1/2); *r_used returns it.
 */
int orc_ml_sparsify(const orc_ml *h, const double *ratios, int32_t n_ratios, double target_fraction,
                    uint8_t *keep0, int64_t *n_kept, double *r_used)
{
    int32_t L = h->L;
    if (n_ratios != L) return ORC_ERR_ARG;
    double r_by_level[64];
    if (target_fraction < 0.0) {
        for (int32_t l = 0; l < L; ++l) r_by_level[l] = ratios[L - 1 - l];
        *n_kept = ml_upward(h, r_by_level, keep0);
        *r_used = -1.0;
        return *n_kept < 0 ? ORC_ERR_OOM : ORC_OK;
    }
    int64_t K = orc_target_count(h->lv[0].m, target_fraction);
    double lo = 0.0, hi = 1.0;
    for (int it = 0; it < 20; ++it) {
        double mid = 0.5 * (lo + hi);
        for (int32_t l = 0; l < L; ++l) r_by_level[l] = (ratios[L - 1 - l] >= 0.0) ? mid : -1.0;
        int64_t c = ml_upward(h, r_by_level, keep0);
        if (c < 0) return ORC_ERR_OOM;
        if (c >= K) hi = mid; else lo = mid;
    }
    for (int32_t l = 0; l < L; ++l) r_by_level[l] = (ratios[L - 1 - l] >= 0.0) ? hi : -1.0;
    *n_kept = ml_upward(h, r_by_level, keep0);
    *r_used = hi;
    return *n_kept < 0 ? ORC_ERR_OOM : ORC_OK;
}

/* Level-span segments of Sec. 6: ratio vector (index 0 = coarsest) for L levels. */
void orc_ml_segment_ratios(int32_t L, int32_t segment, int32_t level_span, double value, double *ratios)
{
    int32_t s = level_span < L ? level_span : L;
    int32_t start = 0;
    if (segment == 1) start = 0;                    /* coarsest levels */
    else if (segment == 2) start = (L - s) / 2;     /* middle levels */
    else start = L - s;                             /* finest levels */
    for (int32_t t = 0; t < L; ++t) ratios[t] = (t >= start && t < start + s) ? value : -1.0;
}

/* ------------------------------------------------------------------------ */
/* Reverse mode of the per-sweep form of Alg. 1 for the loss                */
/*   L(w) = sum_{e in S} rho_e^2,  rho from k sweeps with per-sweep rescale  */
/* with respect to the undirected edge weights w_e (both CSR directions of  */
/* an edge carry w_e).  Written as the plain chain rule over stored         */
/* iterates; min/max use the lowest-index argmin/argmax.                     */
/* ------------------------------------------------------------------------ */
int orc_loss_grad(int64_t n, const int64_t *rp, const int32_t *ci, const double *w,
                  int32_t R, int32_t k, double alpha, uint64_t seed, uint32_t stream,
                  int64_t nS, const int64_t *S, double *loss, double *grad_e)
{
    int64_t nnz = rp[n];
    int64_t m = orc_count_edges(n, rp, ci);
    double omega = 1.0 - alpha;
    int32_t *eu = (int32_t *)malloc(sizeof(int32_t) * (size_t)(m > 0 ? m : 1));
    int32_t *ev = (int32_t *)malloc(sizeof(int32_t) * (size_t)(m > 0 ? m : 1));
    int64_t *eid = (int64_t *)malloc(sizeof(int64_t) * (size_t)(nnz > 0 ? nnz : 1));
    double *D = (double *)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
    /* xs[t] = rescaled iterate after sweep t (xs[0] = init); ys[t] = raw sweep output */
    double *xs = (double *)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1) * (size_t)(k + 1));
    double *ys = (double *)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1) * (size_t)(k + 1));
    int64_t *amin = (int64_t *)malloc(sizeof(int64_t) * (size_t)(k + 1));
    int64_t *amax = (int64_t *)malloc(sizeof(int64_t) * (size_t)(k + 1));
    double *a = (double *)malloc(sizeof(double) * (size_t)(k + 1));
    double *xbar = (double *)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
    double *ybar = (double *)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
    double *gentry = (double *)calloc((size_t)(nnz > 0 ? nnz : 1), sizeof(double));
    if (!eu || !ev || !eid || !D || !xs || !ys || !amin || !amax || !a || !xbar || !ybar || !gentry) {
        free(eu); free(ev); free(eid); free(D); free(xs); free(ys); free(amin); free(amax);
        free(a); free(xbar); free(ybar); free(gentry);
        return ORC_ERR_OOM;
    }
    orc_edge_list(n, rp, ci, eu, ev);
    orc_entry_edge_ids(n, rp, ci, eid);
    orc_weighted_degree(n, rp, w, D);
    double L = 0.0;
    for (int32_t r = 0; r < R; ++r) {
        /* forward, storing every iterate */
        double *x0 = xs;
        for (int64_t i = 0; i < n; ++i) x0[i] = orc_test_value(seed, stream, i, r);
        for (int32_t t = 1; t <= k; ++t) {
            const double *xp = xs + (size_t)(t - 1) * (size_t)n;
            double *y = ys + (size_t)t * (size_t)n, *x = xs + (size_t)t * (size_t)n;
            for (int64_t i = 0; i < n; ++i) {
                if (!(D[i] > 0.0)) { y[i] = xp[i]; continue; }
                double s = 0.0;
                for (int64_t p = rp[i]; p < rp[i + 1]; ++p) s += (w ? w[p] : 1.0) * xp[ci[p]];
                y[i] = alpha * xp[i] + omega * s / D[i];
            }
            int64_t imn = -1, imx = -1;
            for (int64_t i = 0; i < n; ++i) {
                if (!(D[i] > 0.0)) continue;
                if (imn < 0 || y[i] < y[imn]) imn = i;
                if (imx < 0 || y[i] > y[imx]) imx = i;
            }
            amin[t] = imn; amax[t] = imx;
            double lo = imn >= 0 ? y[imn] : 0.0, hi = imx >= 0 ? y[imx] : 0.0;
            a[t] = (hi > lo) ? 1.0 / (hi - lo) : 0.0;
            for (int64_t i = 0; i < n; ++i) {
                if (!(D[i] > 0.0)) { x[i] = xp[i]; continue; }
                x[i] = (hi > lo) ? (y[i] - lo) / (hi - lo) - 0.5 : 0.0;
            }
        }
        /* loss and dL/dx_k */
        const double *xk = xs + (size_t)k * (size_t)n;
        for (int64_t i = 0; i < n; ++i) xbar[i] = 0.0;
        for (int64_t s = 0; s < nS; ++s) {
            int64_t e = S[s];
            double d = xk[eu[e]] - xk[ev[e]];
            L += d * d;
            xbar[eu[e]] += 2.0 * d;
            xbar[ev[e]] -= 2.0 * d;
        }
        /* backward through sweeps t = k .. 1 */
        for (int32_t t = k; t >= 1; --t) {
            const double *x = xs + (size_t)t * (size_t)n;
            const double *xp = xs + (size_t)(t - 1) * (size_t)n;
            /* rescale: x_i = (y_i - y_amin) a - 1/2, a = 1/(y_amax - y_amin) */
            double A = 0.0, B = 0.0;
            for (int64_t i = 0; i < n; ++i) {
                if (!(D[i] > 0.0)) continue;
                A += xbar[i] * (x[i] - 0.5);   /* d x_i / d lo = a (x_i - 1/2) */
                B += xbar[i] * (x[i] + 0.5);   /* d x_i / d hi = -a (x_i + 1/2) */
            }
            for (int64_t i = 0; i < n; ++i) ybar[i] = (D[i] > 0.0) ? a[t] * xbar[i] : 0.0;
            if (a[t] > 0.0) {
                ybar[amin[t]] += a[t] * A;
                ybar[amax[t]] -= a[t] * B;
            }
            /* sweep: y_i = alpha xp_i + omega (sum_j w_ij xp_j) / D_i,  D_i = sum_j w_ij */
            for (int64_t i = 0; i < n; ++i) {
                if (!(D[i] > 0.0)) continue;
                double s = 0.0;
                for (int64_t p = rp[i]; p < rp[i + 1]; ++p) s += (w ? w[p] : 1.0) * xp[ci[p]];
                double avg = s / D[i];
                for (int64_t p = rp[i]; p < rp[i + 1]; ++p)   /* d y_i / d w_ij */
                    gentry[p] += ybar[i] * omega * (xp[ci[p]] - avg) / D[i];
            }
            for (int64_t j = 0; j < n; ++j) {                  /* d L / d xp_j */
                if (!(D[j] > 0.0)) { xbar[j] = 0.0; continue; }
                double s = 0.0;
                for (int64_t p = rp[j]; p < rp[j + 1]; ++p) {
                    int32_t i = ci[p];                        /* w_ij = w_ji */
                    s += ybar[i] * omega * (w ? w[p] : 1.0) / D[i];
                }
                xbar[j] = alpha * ybar[j] + s;
            }
        }
    }
    for (int64_t e = 0; e < m; ++e) grad_e[e] = 0.0;
    for (int64_t p = 0; p < nnz; ++p) grad_e[eid[p]] += gentry[p];
    *loss = L;
    free(eu); free(ev); free(eid); free(D); free(xs); free(ys); free(amin); free(amax);
    free(a); free(xbar); free(ybar); free(gentry);
    return ORC_OK;
}
