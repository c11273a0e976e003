/*
 * ad.h -- C ABI of the GB300 (sm_103a) library for network sparsification by
 * algebraic distance (John & Safro, arXiv 1601.05527).
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 * Graph.  G = (V, E, w) is undirected with positive finite weights, no self
 *   loops and no multi-edges (Sec. 2).  It is passed as a symmetric CSR:
 *   row_ptr int64[n+1] (row_ptr[0] = 0), col int32[nnz] strictly increasing
 *   inside each row, weight float[nnz] with weight(i,j) == weight(j,i), or
 *   NULL for unit weights.
 * Edge ids.  Edge e is the e-th pair (i < j) in CSR row-major order, i.e. the
 *   e-th CSR entry whose column exceeds its row.  Every per-edge array
 *   (rho, keep, scores, gradients) has m entries in this order.
 * Host or device pointers.  Every array argument may live in host memory
 *   (pageable or pinned) or in device memory of the current device; the
 *   library detects which and copies as needed.  Results written to host
 *   memory are complete when the call returns; results written to device
 *   memory are ordered on the graph's stream (complete after that stream is
 *   synchronised).
 * Ownership.  The caller owns every array it passes.  A graph handle owns a
 *   device copy of the CSR and all scratch memory; nothing the caller passes
 *   is retained after a call returns.
 * Streams.  All device work of a handle is issued on the CUDA stream given at
 *   creation (NULL = the legacy default stream).  A handle is not thread safe.
 * Errors.  Every entry point returns an ad_status.  On an error, no output
 *   array has been written unless stated otherwise, and ad_last_error()
 *   returns a message for the calling thread.  Device faults are reported as
 *   AD_ERR_CUDA; the handle should then be destroyed.
 * Random numbers.  Test vector r of vertex i starts at
 *   (u >> 8) * 2^-24 - 1/2, u = word (r mod 4) of Philox4x32-10 (Salmon et al.,
 *   SC'11) with counter (lo32(i), hi32(i), r / 4, stream) and key
 *   (lo32(seed), hi32(seed)): a value of rand(-0.5, 0.5) of Alg. 1.
 */
#ifndef AD_H
#define AD_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    AD_OK = 0,
    AD_ERR_INVALID_ARG = 1,     /* a size, range or pointer argument is invalid */
    AD_ERR_NOT_SYMMETRIC = 2,   /* entry (i,j) without (j,i), or unequal weights */
    AD_ERR_SELF_LOOP = 3,       /* entry (i,i) (Sec. 2 excludes self loops) */
    AD_ERR_DUPLICATE_EDGE = 4,  /* repeated or unsorted column inside a row */
    AD_ERR_BAD_WEIGHT = 5,      /* weight <= 0, NaN or infinite */
    AD_ERR_OOM = 6,             /* device memory allocation failed */
    AD_ERR_CUDA = 7,            /* a CUDA runtime call or kernel failed */
    AD_ERR_TIMEOUT = 8,         /* a bounded device-side wait ran out */
    AD_ERR_STATE = 9,           /* call order: e.g. sparsify before distances */
    AD_ERR_BAD_CSR = 10         /* row_ptr not monotone / col out of range */
} ad_status;

/* Sec. 4 / Fig. 1: which edges a sparsification keeps. */
typedef enum {
    AD_MODE_LOCAL = 0,          /* keep delta-strong (short-range) edges: ascending rho */
    AD_MODE_GLOBAL = 1          /* keep delta-weak (long-range) edges: descending rho */
} ad_mode;

/* Ranking scope. */
typedef enum {
    AD_SCOPE_PER_NODE = 0,      /* Alg. 2: each node keeps its top ceil(d_i^e) edges, union over nodes */
    AD_SCOPE_WHOLE_GRAPH = 1    /* one ranking of all edges (the global-threshold filtering of Sec. 1.1) */
} ad_scope;

/*
 * Storage type of the R test vectors between sweeps; sweeps always
 * accumulate in FP32.  Every stored iterate lies in [-1/2, 1/2] (a sweep
 * output is a convex combination of rescaled values), so besides IEEE
 * formats a 16-bit fixed-point code with step 2^-16 is offered: the same
 * bytes as BF16/FP16 with a uniform absolute error <= 2^-17.
 */
typedef enum {
    AD_STORAGE_FP32 = 0,
    AD_STORAGE_BF16 = 1,
    AD_STORAGE_FP16 = 2,
    AD_STORAGE_Q16 = 3          /* int16 q, value q * 2^-16 */
} ad_storage;

/* ad_graph_create flags */
#define AD_CREATE_SKIP_VALIDATION 0x1   /* trust the caller: no symmetry / sortedness checks */

/* ad_algebraic_distance flags */
#define AD_DIST_NORMALIZE 0x1           /* score rho * sqrt(D_i D_j): the optional last line of Alg. 1 */
#define AD_DIST_KEEP_STATE 0x2          /* keep the iterates ad_algebraic_distance_backward needs */
#define AD_DIST_PERSISTENT 0x4          /* init, all sweeps and distances in one persistent launch (single graphs) */
#define AD_DIST_SQRT_CHECKPOINTS 0x8    /* with AD_DIST_KEEP_STATE: only every ceil(sqrt k)-th iterate */

typedef struct ad_graph_s *ad_graph_t;
typedef struct ad_ml_s *ad_ml_t;

/* ------------------------------------------------------------------------ */
/* Library                                                                   */
/* ------------------------------------------------------------------------ */

/* Version string of the library ("major.minor.patch"). */
const char *ad_version(void);

/* Static text for a status code. */
const char *ad_status_string(ad_status s);

/* Message describing the last error raised on the calling thread ("" if none). */
const char *ad_last_error(void);

/*
 * Device memory hooks.  alloc(bytes, stream, ctx) returns device memory or
 * NULL; release(ptr, bytes, stream, ctx) frees it.  Both are called on the
 * thread that called into the library, with the handle's stream.  Passing
 * NULL hooks restores the default (cudaMallocAsync / cudaFreeAsync on the
 * handle's stream).  Handles created before the call keep freeing their
 * memory with the hooks they were created with.
 */
typedef void *(*ad_alloc_fn)(size_t bytes, void *stream, void *ctx);
typedef void (*ad_free_fn)(void *ptr, size_t bytes, void *stream, void *ctx);
ad_status ad_set_allocator(ad_alloc_fn alloc, ad_free_fn release, void *ctx);

/* Number of kernels this library has launched in the process so far. */
uint64_t ad_kernel_launch_count(void);

/*
 * Per-phase device timing of one handle with CUDA events recorded on the
 * handle's stream around each launch (off by default; while on, every
 * timed launch waits for its end event, so use it for measurement only).
 */
ad_status ad_graph_set_profiling(ad_graph_t g, int32_t enable);

/*
 * Accumulated event time in milliseconds and number of launches of one
 * phase since profiling was enabled: phase is "init", "sweep" (one JOR sweep
 * of Alg. 1 with its fused rescale reduction), "distance" or "select".
 * reset != 0 clears the counters after reading.
 */
ad_status ad_graph_phase_time(ad_graph_t g, const char *phase, double *total_ms, int64_t *launches, int32_t reset);

/*
 * Self-test of the bounded grid-wide wait used by the persistent relaxation:
 * a cooperative launch of two CTAs on stream whose barrier waits for an
 * arrival that never comes, polling at most `polls` times.  *status_out
 * receives the status the waiting kernel recorded (AD_ERR_TIMEOUT when the
 * limit works); the context stays usable.  The paper has no counterpart: this
 * checks the failure path of the library itself.  Errors: AD_ERR_INVALID_ARG,
 * AD_ERR_CUDA, AD_ERR_STATE (a CTA passed the barrier).
 */
ad_status ad_selftest_barrier_timeout(void *stream, uint32_t polls, int32_t *status_out);

/* ------------------------------------------------------------------------ */
/* Graphs                                                                    */
/* ------------------------------------------------------------------------ */

/*
 * Create a graph handle from a symmetric CSR (Sec. 2: undirected, w > 0, no
 * self loops, no multi-edges).  n >= 0 vertices; row_ptr/col/weight as in the
 * conventions above (weight may be NULL = unit weights).  The CSR is copied
 * to device memory owned by the handle and validated unless
 * AD_CREATE_SKIP_VALIDATION is set.  stream: a cudaStream_t (NULL = default
 * stream).  Errors: AD_ERR_INVALID_ARG (n < 0, NULL out, nnz >= 2^31),
 * AD_ERR_BAD_CSR, AD_ERR_SELF_LOOP, AD_ERR_DUPLICATE_EDGE,
 * AD_ERR_NOT_SYMMETRIC, AD_ERR_BAD_WEIGHT, AD_ERR_OOM, AD_ERR_CUDA; *out is
 * left NULL and nothing is leaked.
 */
ad_status ad_graph_create(int64_t n, const int64_t *row_ptr, const int32_t *col, const float *weight,
                          int32_t flags, void *stream, ad_graph_t *out);

/*
 * Create one handle over a batch of n_graphs independent graphs stored as a
 * block-diagonal CSR: graph g owns vertices [vertex_offset[g],
 * vertex_offset[g+1]) (host array of n_graphs + 1 entries, vertex_offset[0] =
 * 0, vertex_offset[n_graphs] = n) and no edge may join two graphs
 * (AD_ERR_INVALID_ARG otherwise).  Edge ids are global; the edges of graph g
 * are a contiguous id range.  Every operation then runs on each graph as if
 * it were alone (its own rescale, its own sparsification target), in one
 * pass over the batch.
 */
ad_status ad_graph_create_batched(int32_t n_graphs, const int64_t *vertex_offset, int64_t n,
                                  const int64_t *row_ptr, const int32_t *col, const float *weight,
                                  int32_t flags, void *stream, ad_graph_t *out);

/* Release a handle and all device memory it owns (NULL is accepted). */
ad_status ad_graph_destroy(ad_graph_t g);

/* Sizes: vertices, undirected edges, CSR entries, vertices of degree > 0, graphs in the batch. */
ad_status ad_graph_info(ad_graph_t g, int64_t *n, int64_t *m, int64_t *nnz, int64_t *n_active,
                        int32_t *n_graphs);

/*
 * Copy the handle's CSR into caller arrays: row_ptr[n+1], col[nnz] and, when
 * the graph has explicit weights, weight[nnz] (each may be NULL to skip; host
 * or device memory).  *has_weight (may be NULL) is set to 0 for unit weights,
 * in which case weight is left untouched.  Used to read coarse graphs.
 */
ad_status ad_graph_export(ad_graph_t g, int64_t *row_ptr, int32_t *col, float *weight, int32_t *has_weight);

/* First edge id of each graph of a batch: edge_offset[n_graphs + 1] (host array). */
ad_status ad_graph_edge_offsets(ad_graph_t g, int64_t *edge_offset);

/*
 * Replace the weights: w_edge[m] holds one positive finite weight per
 * undirected edge (edge-id order); both CSR directions receive it and the
 * weighted degrees are recomputed.  A graph created with unit weights gains
 * explicit weights.  Errors: AD_ERR_BAD_WEIGHT, AD_ERR_INVALID_ARG.
 */
ad_status ad_graph_set_edge_weights(ad_graph_t g, const float *w_edge);

/* ------------------------------------------------------------------------ */
/* Algebraic distance (Sec. 3, Alg. 1)                                       */
/* ------------------------------------------------------------------------ */

/*
 * ComputeAlgDist (Alg. 1) with a rescale after every sweep.  R test vectors
 * (1 <= R <= 256), k >= 0 Jacobi over-relaxation sweeps
 *     x_i <- (1 - omega) x_i + omega (sum_j w_ij x_j) / (sum_j w_ij)
 * (omega = 1 - alpha of the paper; 0 < omega <= 1), each vector rescaled to
 * [-1/2, 1/2] over the vertices of degree > 0 after every sweep (a vector
 * whose values are all equal becomes 0), then for every edge
 *     rho_ij = sqrt(sum_r (x_i^r - x_j^r)^2),
 * the quantity R_ij of Alg. 1 under its square root: delta_ij = 1/sqrt(R_ij + eps)
 * is a decreasing function of rho_ij.  With AD_DIST_NORMALIZE the score is
 * rho_ij * sqrt(D_i D_j) (weighted degrees), the reciprocal of the normalised
 * delta of Alg. 1's last line with eps = 0.  Vertices of degree 0 take no part.
 * stream_id selects an independent random stream (the fourth counter word).
 * storage: FP32 or BF16 storage of the vectors between sweeps (FP32
 * accumulation either way).  rho_out[m] may be NULL; the scores are kept in
 * the handle for ad_sparsify either way.  With AD_DIST_KEEP_STATE the
 * iterates needed by ad_algebraic_distance_backward are kept: all k + 1 of
 * them when they take at most half of the device's free memory (the backward
 * then recomputes none), otherwise -- or with AD_DIST_SQRT_CHECKPOINTS --
 * every ceil(sqrt k)-th one, from which the backward recomputes the others.
 * The gradient is bit-identical either way (the sweep is deterministic).  With AD_DIST_PERSISTENT a single graph (not a batch) is
 * computed in one persistent cooperative launch: init, the k sweeps separated
 * by grid-wide barriers (each rescale needs the min/max over all vertices),
 * then the distances, with bit-identical results; a barrier waits at most a
 * few seconds and then ends the launch with AD_ERR_TIMEOUT (reported by calls
 * made outside a stream capture).  The multilevel functions relax every
 * level this way.
 * Errors: AD_ERR_INVALID_ARG, AD_ERR_OOM, AD_ERR_CUDA, AD_ERR_TIMEOUT.
 */
ad_status ad_algebraic_distance(ad_graph_t g, int32_t R, int32_t k, double omega, uint64_t seed,
                                uint32_t stream_id, ad_storage storage, int32_t flags, float *rho_out);

/*
 * Vector-Jacobian product of the last ad_algebraic_distance call (which must
 * have used AD_DIST_KEEP_STATE, FP32 storage and no normalisation):
 * given rho_bar[m] = dL/drho, writes w_bar[m] = dL/dw_e for every undirected
 * edge weight.  The rescale's min/max are differentiated at the lowest-index
 * argmin/argmax; d rho / d x is taken as 0 where rho = 0.  Errors:
 * AD_ERR_STATE (no kept state), AD_ERR_INVALID_ARG, AD_ERR_OOM, AD_ERR_CUDA.
 */
ad_status ad_algebraic_distance_backward(ad_graph_t g, const float *rho_bar, float *w_bar);

/* ------------------------------------------------------------------------ */
/* Ranking and sampling (Sec. 4, Alg. 2)                                     */
/* ------------------------------------------------------------------------ */

/*
 * Sparsify with the scores of the last ad_algebraic_distance call.
 * Orders: AD_MODE_LOCAL ranks edges by ascending score (delta-strong first),
 * AD_MODE_GLOBAL by descending score (delta-weak first); ties by ascending
 * edge id.  Target K = floor(fraction * m + 1/2) edges (per graph of a batch).
 *   AD_SCOPE_WHOLE_GRAPH: keep the first K edges of the order.
 *   AD_SCOPE_PER_NODE (Alg. 2): node i keeps its first
 *     T(d_i, e) = min(d_i, max(1, ceil(d_i^e - 1e-9))) incident edges
 *     (d_i = unweighted degree), the sparse graph is the union over nodes,
 *     and e is the smallest point of the 2^-40 grid of [0, 1] whose union
 *     has >= K edges (binary search, Sec. 6.2).  With a batch, e is fitted
 *     per graph.
 * keep_out[m] (uint8 0/1) receives the kept set; n_kept (total) and e_used
 * (per-node scope: the exponent, for a batch the one of graph 0; whole-graph
 * scope: -1) may be NULL.  0 <= fraction <= 1.  Errors: AD_ERR_STATE (no
 * scores yet), AD_ERR_INVALID_ARG, AD_ERR_OOM, AD_ERR_CUDA.
 */
ad_status ad_sparsify(ad_graph_t g, double fraction, ad_mode mode, ad_scope scope, uint8_t *keep_out,
                      int64_t *n_kept, double *e_used);

/*
 * Alg. 2 (per-node scope) in both orders at once on the scores of the last
 * ad_algebraic_distance call: keep_local[m] receives the AD_MODE_LOCAL
 * selection and keep_global[m] the AD_MODE_GLOBAL one, each exactly as
 * ad_sparsify with AD_SCOPE_PER_NODE would give it.  The per-node ranking is
 * taken once for both orders and the two exponent searches run as one
 * two-problem search.  n_kept[2] and e_used[2] (local, global; for a batch
 * the totals and graph 0's exponents) may be NULL.  keep_local and
 * keep_global may each be host or device memory.  0 <= fraction <= 1.
 * Errors: as ad_sparsify.
 */
ad_status ad_sparsify_local_global(ad_graph_t g, double fraction, uint8_t *keep_local, uint8_t *keep_global,
                                   int64_t *n_kept, double *e_used);

/*
 * As ad_sparsify, with caller-supplied scores score[m] (non-negative and
 * finite, e.g. precomputed distances) instead of the kept ones.  The scores
 * are compared as FP32 values.  Errors: as ad_sparsify, plus
 * AD_ERR_INVALID_ARG for negative or non-finite scores.
 */
ad_status ad_sparsify_scores(ad_graph_t g, const float *score, double fraction, ad_mode mode,
                             ad_scope scope, uint8_t *keep_out, int64_t *n_kept, double *e_used);

/*
 * Alg. 2 at a given exponent e in [0, 1] (per-node scope, no fitting) on
 * score[m] (NULL = the kept scores).  keep_out[m], n_kept may be NULL.
 */
ad_status ad_select_per_node(ad_graph_t g, const float *score, double e, ad_mode mode, uint8_t *keep_out,
                             int64_t *n_kept);

/*
 * Picks the launch shape of the JOR sweep (Alg. 1) for this graph, R and
 * storage by timing the candidates on the handle: lanes per row (the natural
 * 16-byte-chunk layout, and half as many lanes with two chunks each) x
 * resident CTAs per SM (as many as fit, 5, 4).  Each candidate runs a short
 * distance computation (k = 4) three times; the fastest shape is kept on the
 * handle and used by every later call with this R and storage.  The result
 * depends only on the shape through the order of FP32 additions.
 *   lanes_per_row, chunks_per_lane, ctas_per_sm (0 = as many as fit): the
 *   chosen shape; each may be NULL.
 * Errors: AD_ERR_INVALID_ARG, AD_ERR_OOM, AD_ERR_CUDA.
 */
ad_status ad_graph_autotune(ad_graph_t g, int32_t R, ad_storage storage, int32_t *lanes_per_row,
                            int32_t *chunks_per_lane, int32_t *ctas_per_sm);

/*
 * SparsifyB, the binned ("mixture") single-level sparsification of Alg. 3
 * (Sec. 4): for every node, the distances of its incident edges are put into
 * bins of width h = 3.5 sigma / d^(1/3) (sigma: their population standard
 * deviation; one bin when sigma = 0), and the node takes T(d, e) of its edges
 * by drawing from all bins in turn -- entries of a bin and the bins themselves
 * in random order, round robin over the bins -- so that short- and long-range
 * connections are both kept.  An edge is kept when either end takes it; e is
 * fitted to reach K = floor(fraction * m + 1/2) edges exactly as in
 * ad_sparsify's per-node scope.  The random order comes from Philox4x32-10 with
 * key = seed: word 0 of counter (edge id, 0, 0xB1000000) for an edge and of
 * (vertex, 1 + bin, 0xB1000000) for a bin of that vertex.
 *   score     [m] FP32 scores (non-negative, finite), host or device; NULL =
 *             the distances of the last ad_algebraic_distance call.
 *   keep_out  [m] uint8, host or device; n_kept, e_used may be NULL.
 * Errors: AD_ERR_INVALID_ARG (fraction outside [0, 1], bad scores, a row with
 * 2^24 bins or more), AD_ERR_STATE (score NULL and no distances), AD_ERR_OOM,
 * AD_ERR_CUDA.
 */
ad_status ad_sparsify_binned(ad_graph_t g, const float *score, double fraction, uint64_t seed, uint8_t *keep_out,
                             int64_t *n_kept, double *e_used);

/*
 * The per-entry quantities behind ad_sparsify_binned (Alg. 3, Sec. 4), for
 * inspection and testing: rank_out[nnz] receives the SparsifyB selection rank
 * of every CSR entry inside its row (node i keeps its entries of rank <
 * T(d_i, e)), bin_out[nnz] (may be NULL) the bin floor((rho - min) / h) of the
 * entry in its row.  Both are uint32 in CSR order, host or device memory.
 * score and seed as in ad_sparsify_binned.  The per-row mean and sigma are
 * FP64 sums over the lanes of a warp, so a bin can differ from one computed
 * with sequential FP64 sums only when (rho - min) / h lies within a few units
 * in the last place of an integer.  Errors: as ad_sparsify_binned.
 */
ad_status ad_binned_ranks(ad_graph_t g, const float *score, uint64_t seed, uint32_t *rank_out, uint32_t *bin_out);

/*
 * Local Degree, the method the paper compares against (Sec. 1.1, Sec. 6;
 * Lindner et al.): every node takes the edges to its T(d, e) neighbours of
 * largest degree (ties: smaller neighbour position in the row), an edge is
 * kept when either end takes it, and e is fitted to reach
 * K = floor(fraction * m + 1/2) edges as in ad_sparsify's per-node scope.  No
 * distances are needed.  keep_out[m] uint8, host or device; n_kept, e_used may
 * be NULL.  Errors: AD_ERR_INVALID_ARG, AD_ERR_OOM, AD_ERR_CUDA.
 */
ad_status ad_sparsify_local_degree(ad_graph_t g, double fraction, uint8_t *keep_out, int64_t *n_kept,
                                   double *e_used);

/*
 * Whole-graph ranking (as ad_sparsify_scores with AD_SCOPE_WHOLE_GRAPH on a
 * single graph whose edge ids are 0..m-1) for callers that cannot let a
 * library allocate device memory -- a process whose device memory is all
 * pre-reserved by its own allocator or arena, or a latency-critical service
 * that must not reach the allocator on its request path.  The paper has no
 * counterpart; this is an operational variant.
 * score[m] (FP32, >= 0, finite) and keep[m] (uint8 output) must be device
 * arrays; K = floor(fraction m + 1/2) edges are kept in the order of mode
 * (ties by index); *n_kept (may be NULL) receives K.  stream: a cudaStream_t.
 * No cudaMalloc, cudaFree or allocating library routine is called: all
 * scratch lives in one fixed device array of about 600 KB that every GPU
 * loading the library holds until exit, which limits m to 2^26
 * (AD_ERR_INVALID_ARG beyond).  The first call on a device looks the array
 * up (cudaGetSymbolAddress) and should come before any stream capture.  All
 * calls on a device share the array: each call rewrites what it reads, and
 * calls that overlap on the GPU race, so the caller must order them.  Every
 * call checks the scores on the device and then waits on the host for the
 * result (a device-to-host copy followed by cudaStreamSynchronize(stream)),
 * so that it can return an error before any selection work is queued; the
 * selection itself is then queued on stream and is complete after the stream
 * is synchronised.  *n_kept is written only when the call succeeds.
 * Errors: AD_ERR_INVALID_ARG (size, fraction, mode, host pointers, negative
 * or non-finite scores), AD_ERR_CUDA.
 */
ad_status ad_select_whole_graph_noalloc(const float *score, int64_t m, double fraction, ad_mode mode, uint8_t *keep,
                                        int64_t *n_kept, void *stream);

/* ------------------------------------------------------------------------ */
/* Multilevel sparsification (Sec. 5, Alg. 6)                                */
/* ------------------------------------------------------------------------ */

typedef struct {
    int32_t R;              /* test vectors per level (Alg. 1) */
    int32_t k;              /* JOR sweeps per level */
    double omega;           /* 1 - alpha */
    uint64_t seed;          /* level l uses Philox stream 2l down, 2l+1 up */
    double Q;               /* seed coupling threshold: i becomes a seed when its weight to earlier seeds <= Q D_i */
    int64_t coarsest_n;     /* stop coarsening at n <= coarsest_n (Alg. 6 "small enough") */
    int32_t max_levels;     /* 1..64 */
    ad_mode mode;           /* local or global filtering at every sparsified level */
    ad_storage storage;     /* storage of the test vectors */
} ad_ml_params;

/*
 * Downward half of Alg. 6: at each level ComputeAlgDist, createSeeds
 * (vertices by decreasing weighted degree, ties by id; i joins C when its
 * weight to the seeds already chosen is <= Q D_i), the restriction P of
 * Eq. (P) (an F vertex joins its seed neighbour of smallest rho, ties to the
 * smaller seed id; coarse ids number the seeds by vertex id) and the
 * Galerkin coarse graph L_c = P^T L_f P, until n <= coarsest_n, n_c > 0.9
 * n_f, or max_levels.  The handle keeps the hierarchy; g must outlive it,
 * and the scores kept in g are replaced by the level-0 distances.
 * Errors: AD_ERR_INVALID_ARG (bad parameters, Q outside [0, 1), a batch),
 * AD_ERR_OOM, AD_ERR_CUDA.
 */
ad_status ad_ml_build(ad_graph_t g, const ad_ml_params *params, ad_ml_t *out);

/* Number of levels (level 0 = the input graph) and the size of one level. */
ad_status ad_ml_levels(ad_ml_t ml, int32_t *n_levels);
ad_status ad_ml_level_size(ad_ml_t ml, int32_t level, int64_t *n, int64_t *m);

/*
 * Upward half of Alg. 6.  ratios[n_levels] is the paper's vector of
 * sparsification ratios: ratios[0] belongs to the coarsest level, -1 means
 * "not sparsified", otherwise the fraction of that level's current edges to
 * keep with Alg. 2 (e fitted per level).  The coarsest level is sparsified
 * on its own distances; every finer level first inherits the removals of
 * the coarser one (a fine edge bundled into a removed coarse edge is
 * removed; edges inside an aggregate are kept), then, if sparsified,
 * recomputes the distances on its remaining graph and sparsifies it.  With
 * target_fraction >= 0 every level whose ratio is >= 0 uses one shared
 * fraction r, the smallest point of the 2^-20 grid of [0, 1] whose final
 * edge count reaches floor(target_fraction * m + 1/2); r_used returns it
 * (-1 otherwise).  keep_out[m] for the finest graph; n_kept may be NULL.
 */
ad_status ad_ml_sparsify(ad_ml_t ml, const double *ratios, int32_t n_ratios, double target_fraction,
                         uint8_t *keep_out, int64_t *n_kept, double *r_used);

/*
 * MLSparsify(G_f, ratios) of Alg. 6 in one call: builds the hierarchy as
 * ad_ml_build does, runs the upward half as ad_ml_sparsify does, writes the
 * kept set of the input graph and releases the hierarchy.  ratios[l]
 * (l = 0 .. n_ratios - 1, host memory) is the ratio of the l-th coarsest
 * level in ad_ml_sparsify's convention (-1: not sparsified, otherwise the
 * fraction of that level's edges to keep, or with target_fraction >= 0 a
 * marker of the levels that share the fitted ratio); levels past the end of
 * the vector are not sparsified, so the caller need not know the number of
 * levels in advance.  ratios may be NULL when n_ratios = 0 (nothing is
 * sparsified: every edge is kept).  keep_out[m] uint8, host or device;
 * *n_levels_out (may be NULL) receives the number of levels built.  g must
 * not be a batch; its kept scores are replaced by the level-0 distances.
 * Errors: those of ad_ml_build and ad_ml_sparsify.
 */
ad_status ad_multilevel(ad_graph_t g, const ad_ml_params *params, const double *ratios, int32_t n_ratios,
                        double target_fraction, uint8_t *keep_out, int32_t *n_levels_out);

/*
 * Inspection of level `level` of a hierarchy, for checking Alg. 6 level by
 * level: the level's graph as ad_graph_export writes it (row_ptr[n_l + 1],
 * col[nnz_l], weight[nnz_l] FP32 or *has_weight = 0 for unit weights), the
 * distances of the downward pass rho[m_l] (Alg. 1 with Philox stream 2 level),
 * and the maps to level + 1: agg[n_l] (coarse vertex of each vertex under
 * Eq. (P), -1 for degree-0 vertices) and fine_to_coarse[m_l] (coarse edge of
 * each edge, -1 inside an aggregate).  Every pointer may be NULL; host or
 * device memory.  Errors: AD_ERR_INVALID_ARG (level), AD_ERR_STATE (agg or
 * fine_to_coarse asked of the coarsest level).
 */
ad_status ad_ml_level_export(ad_ml_t ml, int32_t level, int64_t *row_ptr, int32_t *col, float *weight,
                             int32_t *has_weight, float *rho, int32_t *agg, int64_t *fine_to_coarse);

/*
 * Upward trace: with enable != 0, later ad_ml_sparsify calls (and, for a
 * fitted target fraction, their final pass) record per level the edges left
 * after the coarser level's removals, the edges kept at the level and the
 * distances recomputed on the kept subgraph G_f^s of Alg. 6 (NaN where an
 * edge is not in it or the level is not sparsified); ad_ml_level_trace reads
 * them (inherited[m_l], kept[m_l] uint8; rho_up[m_l] FP32; each may be NULL;
 * host or device memory).  Tracing holds 6 bytes per edge of every level.
 * Errors: AD_ERR_INVALID_ARG, AD_ERR_STATE (no traced call yet).
 */
ad_status ad_ml_set_trace(ad_ml_t ml, int32_t enable);
ad_status ad_ml_level_trace(ad_ml_t ml, int32_t level, uint8_t *inherited, uint8_t *kept, float *rho_up);

/* Ratio vector of the level-span experiments of Sec. 6 for an n_levels
 * hierarchy: segment 1 = coarsest, 2 = middle, 3 = finest levels;
 * level_span levels of the segment get value, the others -1. */
ad_status ad_ml_segment_ratios(int32_t n_levels, int32_t segment, int32_t level_span, double value,
                               double *ratios_out);

/* Release a hierarchy (NULL is accepted). */
ad_status ad_ml_destroy(ad_ml_t ml);

/*
 * Coarsening components on caller scores, for one level: seeds and the
 * aggregate map of Eq. (P) (agg_out[n], -1 for degree-0 vertices), the number
 * of coarse vertices, and the Galerkin coarse graph as a new handle
 * (coarse_out, may be NULL) with fine_to_coarse_out[m] (coarse edge id of
 * each fine edge, -1 inside an aggregate; may be NULL).
 */
ad_status ad_coarsen(ad_graph_t g, const float *score, double Q, int32_t *agg_out, int64_t *n_coarse,
                     ad_graph_t *coarse_out, int64_t *fine_to_coarse_out);

#ifdef __cplusplus
}
#endif

#endif /* AD_H */
