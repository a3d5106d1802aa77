/*
 * ubt.h -- C ABI of libubt: exact counting and enumeration of t-balanced and
 * t-unbalanced triangles on uncertain signed graphs, on one GB300 GPU.
 *
 * Paper: "Counting Balanced Triangles on Social Networks With Uncertain Edge
 * Signs" (arXiv 2602.14084).  The operations and their defining passages:
 *   - uncertain signed graph G = (V, E, P+)                (Def. 1, Sec. 3)
 *   - triangle; balanced iff an odd number of its edges are positive
 *                                                      (Defs. 2-3, Sec. 3)
 *   - P_bal = sum over the classes T3 and T1 of products of independent
 *     P+ / P-; P_unbal = 1 - P_bal                     (equation in Sec. 3)
 *   - t-balanced: P_bal >= t; t-unbalanced: P_unbal > t  (Defs. 4-5, Sec. 3)
 *   - counting / enumeration problems UBTC / UBTE      (Defs. 7-8, Sec. 3)
 *   - exact algorithms: forward iteration under Node Order (Alg. 1, Sec. 4)
 *     and probability pruning (Lemma 2, Lemma 3, Alg. 2, Sec. 5)
 *
 * Conventions
 *   - Every function returns ubt_status: 0 = UBT_OK, negative = error.
 *     Nothing throws or aborts across this boundary.
 *   - Pointers named d_* are device pointers, h_* host pointers.  All device
 *     memory is owned by the caller; the library never allocates or frees
 *     device memory.  Sizes are queried with the *_workspace_size calls.
 *   - Calls marked ASYNC only enqueue work on the given stream and write
 *     their outputs when that work completes; they do not synchronise and may
 *     be captured into a CUDA graph.  Calls marked SYNC synchronise `stream`
 *     before returning.
 *   - Calls on the same graph must not overlap in time (issue them on one
 *     stream): each graph carries one query scratch area.
 *   - Fixed point: P+(e) = k_e / 65536 with integer k_e in [0, 65536].  With
 *     q_e = 32768 - k_e (so 1 - 2 P+(e) = q_e / 2^15) every test is exact in
 *     int64; counts and enumeration records are bit-exact.
 *   - Thresholds t must lie in [0.5, 1] (the paper assumes t >= 0.5, Sec. 3);
 *     t is used exactly as the given IEEE double.
 *   - The stream is a cudaStream_t passed as void* (0 = legacy default).
 */
#ifndef UBT_H
#define UBT_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef int32_t ubt_status;

#define UBT_OK 0
#define UBT_ERR_INVALID_ARG (-1)          /* null pointer, bad size, bad flag */
#define UBT_ERR_SELF_LOOP (-2)            /* an edge (v, v) */
#define UBT_ERR_DUPLICATE_EDGE (-3)       /* the same unordered pair twice */
#define UBT_ERR_VERTEX_OOB (-4)           /* an endpoint >= n */
#define UBT_ERR_PROB_OOB (-5)             /* k > 65536, or p outside [0,1] / NaN */
#define UBT_ERR_TAU_OOB (-6)              /* t outside [0.5, 1] or NaN */
#define UBT_ERR_CAPACITY (-7)             /* enumeration output too small */
#define UBT_ERR_WORKSPACE_TOO_SMALL (-8)  /* workspace below the queried size */
#define UBT_ERR_TIMEOUT (-9)              /* reserved: a bounded device wait gave up */
#define UBT_ERR_CUDA (-10)                /* a CUDA runtime call failed */
#define UBT_ERR_UNSUPPORTED (-11)         /* operation not defined for this graph kind */
#define UBT_ERR_SCRATCH_LIMIT (-12)       /* request larger than a fixed scratch array */

/* Graph kinds (the `flags` of ubt_graph_workspace_size / ubt_create_graph). */
#define UBT_GRAPH_FIXED 0   /* probabilities given as k (uint32, 0..65536) */
#define UBT_GRAPH_REAL 1    /* probabilities given as p (float32, [0,1]) */

typedef struct ubt_graph ubt_graph;   /* opaque */

/* One enumeration record (24 bytes): the triangle's vertex ids (as given,
 * u < v < w), its class (1 = t-balanced, 2 = t-unbalanced) and its exact
 * balance probability P_bal = N / 2^46 (exact in double). */
typedef struct {
    uint32_t u, v, w;
    uint32_t cls;
    double p_bal;
} ubt_tri_rec;

/* Sizes of the built graph, filled by ubt_graph_get_info. */
typedef struct {
    int64_t n;                /* vertices */
    int64_t m;                /* undirected edges */
    int64_t max_out_degree;   /* largest forward list under Node Order */
    int64_t hub_vertices;     /* vertices handled by a whole thread block */
    int64_t wedges;           /* sum over forward edges (u,v) of |N>(v)|: the
                                 entries Alg. 1 probes */
    int64_t kind;             /* UBT_GRAPH_FIXED or UBT_GRAPH_REAL */
    int64_t probes;           /* entries the traversal probes without pruning:
                                 sum over pairs of the streamed list's length */
} ubt_graph_info;

/* Optional extras for ubt_create_graph (pass NULL for none). */
typedef struct {
    /* Philox key of every edge (device, m entries); NULL = the edge index.
     * Sub-graphs cut from a parent pass the parent's edge ids here so that
     * their sign worlds agree with the parent's. */
    const uint32_t* d_edge_key;
    /* Batches of disjoint graphs: d_vertex_offsets[g] .. [g+1] is the vertex
     * range of graph g (device, n_graphs + 1 entries, int64, ascending,
     * first 0, last n).  Edges must not cross graphs.  NULL = one graph. */
    const int64_t* d_vertex_offsets;
    int64_t n_graphs;
    /* UBT_OPT_UNDIRECTED: also build the undirected adjacency in Absolute
     * Edge Order (FIXED graphs only), which ubt_count_aeo, ubt_enumerate_aeo,
     * ubt_edge_local_counts and ubt_vertex_local_counts need.
     * UBT_OPT_EDGE_INDEX (with UBT_OPT_UNDIRECTED): also build a hash index
     * of the edges ({u, w} -> edge value; 16 bytes per slot, the power of two
     * >= 4m slots).  Same results, different work: ubt_vertex_local_counts
     * and ubt_vertex_topk look a neighbour pair up in it instead of streaming
     * a neighbour's row when that row is much longer than the pairs left to
     * check; ubt_count_aeo and ubt_enumerate_aeo stream, for each edge, the
     * shorter of its two Lemma 3 windows and look the closing edge up, with
     * no owner tables (knob "edge_index" = 0 keeps the table forms). */
    int64_t flags;
} ubt_graph_opts;

#define UBT_OPT_UNDIRECTED 1
#define UBT_OPT_EDGE_INDEX 2

/* Human-readable name of a status code (static string). */
const char* ubt_status_str(ubt_status s);

/* Library version as MAJOR*10000 + MINOR*100 + PATCH. */
int32_t ubt_version(void);

/*
 * ubt_graph_workspace_size -- bytes of device workspace a graph of n vertices
 * and m edges of the given kind needs (the built forward CSR, its edge ids,
 * temporaries of the build and the per-graph query scratch).  With opts
 * describing a batch, pass the same opts to ubt_create_graph.
 * Errors: UBT_ERR_INVALID_ARG (n or m negative or >= 2^32 - 1, bad flags).
 */
ubt_status ubt_graph_workspace_size(int64_t n, int64_t m, int32_t flags,
                                    const ubt_graph_opts* opts, size_t* h_bytes);

/*
 * ubt_create_graph -- SYNC.  Validates the edge list and builds the graph the
 * exact algorithms traverse (Def. 1; Node Order, Sec. 4):
 *   - each undirected edge {a, b} is kept once and oriented from the endpoint
 *     earlier in Node Order (degree, then id) to the later one;
 *   - the forward lists N>(u) are stored as CSR, each list sorted by
 *     |1 - 2 P+| descending (ties by neighbour id), so that the edges a
 *     threshold prunes (Lemma 2) form a suffix of every list.
 * Arguments:
 *   n, m           vertex and edge counts (0 allowed).
 *   d_src, d_dst   device uint32[m] endpoints, any order, ids < n.
 *   d_k            device uint32[m], k in [0, 65536]   (flags FIXED), or NULL
 *   d_p            device float[m], p in [0, 1]         (flags REAL), or NULL
 *   flags          UBT_GRAPH_FIXED or UBT_GRAPH_REAL.
 *   opts           NULL, or the extras above.
 *   d_workspace    device buffer of >= ubt_graph_workspace_size bytes,
 *                  256-byte aligned; owned by the caller and used by the
 *                  graph until ubt_destroy_graph (do not free it earlier).
 *   stream         cudaStream_t as void*.
 *   h_out          receives the graph handle (host memory, owned by the
 *                  library; release with ubt_destroy_graph).
 * The input arrays may be freed after the call returns.
 * Errors: UBT_ERR_INVALID_ARG, UBT_ERR_SELF_LOOP, UBT_ERR_DUPLICATE_EDGE,
 *   UBT_ERR_VERTEX_OOB, UBT_ERR_PROB_OOB, UBT_ERR_WORKSPACE_TOO_SMALL,
 *   UBT_ERR_CUDA.  On error no handle is returned.
 */
ubt_status ubt_create_graph(int64_t n, int64_t m, const uint32_t* d_src, const uint32_t* d_dst,
                            const uint32_t* d_k, const float* d_p, int32_t flags,
                            const ubt_graph_opts* opts, void* d_workspace, size_t ws_bytes,
                            void* stream, ubt_graph** h_out);

/* ubt_destroy_graph -- releases the handle (not the caller's workspace). */
ubt_status ubt_destroy_graph(ubt_graph* g);

/* ubt_graph_get_info -- SYNC-free; copies the sizes recorded at build time. */
ubt_status ubt_graph_get_info(const ubt_graph* g, ubt_graph_info* h_info);

/*
 * ubt_count_threshold -- ASYNC.  Counting problem (UBTC, Def. 8): for each of
 * n_tau thresholds t_i, the number of triangles with P_bal >= t_i and the
 * number with P_unbal > t_i (Defs. 4-5; Alg. 1 and Alg. 2).  All thresholds
 * are answered in one traversal.
 *   h_tau     host double[n_tau], each in [0.5, 1], any order, 1 <= n_tau <= 64.
 *   prune     0: visit every triangle (Alg. 1).  1: skip edges and triangles
 *             that cannot reach the smallest threshold (Lemma 2 per edge;
 *             the order-free form of Lemma 3 per pair of edges, applied to
 *             the streamed lists only when 2t - 1 >= 1/10 for the smallest
 *             t: below that it removes too few entries to pay for itself);
 *             results are identical either way.
 *   d_counts  device int64[2 * n_tau]: [0, n_tau) balanced counts,
 *             [n_tau, 2 n_tau) unbalanced counts, in the order of h_tau.
 * Graph kind: FIXED only (UBT_ERR_UNSUPPORTED otherwise).
 * Errors: UBT_ERR_INVALID_ARG, UBT_ERR_TAU_OOB, UBT_ERR_UNSUPPORTED, UBT_ERR_CUDA.
 */
ubt_status ubt_count_threshold(ubt_graph* g, const double* h_tau, int32_t n_tau, int32_t prune,
                               int64_t* d_counts, void* stream);

/*
 * ubt_count_threshold_noalloc -- ASYNC after its first call on a device.  The
 * same counts as ubt_count_threshold, for callers that cannot allocate device
 * memory where they query (code that may only use buffers it is handed, or
 * that must not call an allocator): the per-call scratch -- task counters,
 * self-check word and per-threshold accumulators -- lives in a fixed 2 KiB
 * array in the library's own device memory, which every GPU that loads the
 * library holds until the process exits.  The paper has no counterpart; this
 * is an interface for such callers.
 *   Arguments as ubt_count_threshold, with 1 <= n_tau <= 8; more thresholds
 *   return UBT_ERR_SCRATCH_LIMIT (the fixed array has room for 8).
 *   No device memory is allocated or freed (no cudaMalloc, no allocating
 *   library call); the array is cleared on `stream` at every call.
 *   The first call on a device looks up the array's device address (once per
 *   device, with that device current); make that first call before any
 *   stream capture.  The current device must be the one the graph was built
 *   on (else UBT_ERR_INVALID_ARG): the array used is that device's.
 *   All calls share the one array: calls that overlap on the GPU (on
 *   different streams, or on different graphs at the same time) race and
 *   give wrong counts.  Issue them one after another on one stream.
 *   A failed self-check of the traversal is copied into the graph's own
 *   self-check word at the end of the call, so ubt_query_guard sees it.
 */
ubt_status ubt_count_threshold_noalloc(ubt_graph* g, const double* h_tau, int32_t n_tau, int32_t prune,
                                       int64_t* d_counts, void* stream);

/*
 * ubt_enumerate -- SYNC.  Enumeration problem (UBTE, Def. 7) at threshold t:
 * writes one ubt_tri_rec per t-balanced (which & 1) and/or t-unbalanced
 * (which & 2) triangle into d_out, in no particular order.
 *   d_out       device ubt_tri_rec[capacity] (may be NULL if capacity == 0).
 *   h_n_found   receives the total number of records (even when it exceeds
 *               capacity; then only `capacity` records are written and the
 *               call returns UBT_ERR_CAPACITY).
 *   prune       as in ubt_count_threshold.
 * Graph kind: FIXED only.
 */
ubt_status ubt_enumerate(ubt_graph* g, double tau, int32_t which, int32_t prune,
                         ubt_tri_rec* d_out, int64_t capacity, int64_t* h_n_found, void* stream);

/*
 * ubt_expected_counts -- ASYNC.  Expected numbers of balanced and unbalanced
 * triangles, E_bal = sum_t P_bal(t) = (T - sum_t S_t) / 2 and
 * E_unbal = (T + sum_t S_t) / 2 with S_t the product of (1 - 2 P+) over the
 * triangle's edges (from the equation in Sec. 3; not in the paper).
 *   d_out    device double[2] = {E_bal, E_unbal}.
 *   d_exact  device int64[4] or NULL: {T, sum_lo, sum_hi, 0}: T triangles
 *            and sum_hi:sum_lo a two's-complement 128-bit integer.  FIXED
 *            graph: the exact sum of q_e q_f q_g over all triangles, so
 *            E_bal = (T 2^45 - sum) / 2^46 exactly.  REAL graph: the sum of
 *            S_t * 2^32, each term rounded to an integer.
 * Arithmetic: FIXED graphs are exact (int64 products, 128-bit sums).  REAL
 * graphs hold s = 1 - 2p as s * 2^30 rounded to an int32 (exact for
 * p >= 2^-7, within 2^-31 otherwise); the products are exact int64 products
 * of these, rounded once to 2^-30 and once to 2^-32 per triangle; the sum is
 * exact in 128 bits and converted to double at the end.
 */
ubt_status ubt_expected_counts(ubt_graph* g, double* d_out, int64_t* d_exact, void* stream);

/*
 * ubt_expected_counts_backward -- ASYNC.  Adjoint of ubt_expected_counts:
 *   d_grad_p[e] = (g_bal - g_unbal) * sum over triangles t containing e of
 *                 (1 - 2 p_f)(1 - 2 p_g)     (f, g the other two edges of t)
 * i.e. the gradient of L = g_bal E_bal + g_unbal E_unbal with respect to p_e.
 *   d_gout    device double[2] = {g_bal, g_unbal} (upstream gradients).
 *   d_grad_p  device float[m], input edge order (overwritten).
 * Arithmetic: FIXED graphs exact in int64 before the final scaling; REAL
 * graphs exact int64 products of the 2^-30 fixed-point s values, rounded to
 * 2^-40 and accumulated in 64-bit integers, scaled to float at the end.
 * Limit: an edge's accumulator is a signed 64-bit integer and every triangle
 * adds a term of magnitude at most 2^30 (FIXED, units of 2^-30) or 2^40
 * (REAL, units of 2^-40), so the sum is exact while an edge lies in fewer
 * than 2^33 (FIXED) or 2^23 = 8,388,608 (REAL) triangles.  The sum of a REAL
 * edge in more triangles than that can wrap; no check is made.
 */
ubt_status ubt_expected_counts_backward(ubt_graph* g, const double* d_gout, float* d_grad_p,
                                        void* stream);

/*
 * ubt_set_edge_values -- ASYNC.  Replaces the probabilities of a REAL graph
 * with d_p (device float[m], input edge order, each in [0, 1]) without
 * rebuilding it: every stored s = 1 - 2p is recomputed from the new p, in the
 * arithmetic of ubt_create_graph.  Structure, orientation and work lists are
 * unchanged (REAL rows are ordered by neighbour id, which p does not affect),
 * so expected counts and their adjoint then answer for the new p (Sec. 3's
 * P_bal equation, with the new P+).  This is what a gradient step on p needs.
 * An entry outside [0, 1] or NaN keeps its old value, and the first such
 * input index is recorded in the self-check word (ubt_query_guard, code 6).
 * Graph kind: REAL only (UBT_ERR_UNSUPPORTED for FIXED: their rows are
 * ordered by |q|, which a new k would change).
 * Errors: UBT_ERR_INVALID_ARG, UBT_ERR_UNSUPPORTED, UBT_ERR_CUDA.
 */
ubt_status ubt_set_edge_values(ubt_graph* g, const float* d_p, void* stream);

/*
 * ubt_sample_worlds_workspace_size / ubt_sample_worlds -- ASYNC.  Monte-Carlo
 * sign worlds (not in the paper): W worlds (W a positive multiple of 64), each
 * an independent draw of every edge's sign with P(+) = k_e / 65536.  Returns
 * the number of balanced triangles (odd number of positive edges, Def. 3) in
 * every world.
 * Draws: world 64 w + j, edge with key K (ubt_graph_opts.d_edge_key, default
 * the edge index): sixteen 64-bit words r_0..r_15 from Philox4x64-10 with key
 * (seed, 0) and counters (K, w, c, 0), c = 0..3 (call c gives r_{4c..4c+3});
 * u_j = sum_b bit j of r_b * 2^b; the edge is positive iff u_j < k_e.
 *   d_bal_per_world  device int64[W].
 *   d_total          device int64[1]: sum over worlds (may be NULL).
 *   d_workspace      >= the queried bytes (sign table of one pass + counters).
 * Graph kind: FIXED only.
 */
ubt_status ubt_sample_worlds_workspace_size(const ubt_graph* g, int64_t W, size_t* h_bytes);
ubt_status ubt_sample_worlds(ubt_graph* g, uint64_t seed, int64_t W, int64_t* d_bal_per_world,
                             int64_t* d_total, void* d_workspace, size_t ws_bytes, void* stream);

/*
 * ubt_batch_query -- ASYNC.  For a graph created with opts.d_vertex_offsets
 * (a batch of disjoint graphs), answers per graph, in one launch:
 *   d_counts  device int64[n_graphs * 2 * n_tau]: graph g's balanced counts at
 *             [g*2*n_tau, g*2*n_tau + n_tau), unbalanced after them.
 *   d_expect  device double[n_graphs * 2] = {E_bal, E_unbal} per graph (exact
 *             for FIXED graphs), or NULL.
 *   d_worlds  device int64[n_graphs * 64]: balanced counts in the 64 worlds of
 *             world word 0 drawn with `seed` (as in ubt_sample_worlds), or NULL.
 *   h_tau     as in ubt_count_threshold (1 <= n_tau <= 8).
 * Graph kind: FIXED only.  Capturable into a CUDA graph.
 */
ubt_status ubt_batch_query(ubt_graph* g, const double* h_tau, int32_t n_tau, uint64_t seed,
                           int64_t* d_counts, double* d_expect, int64_t* d_worlds, void* stream);

/*
 * ubt_count_host -- SYNC, end to end from host memory.  Copies a FIXED graph
 * (h_src, h_dst, h_k: host uint32[m]) to the device, builds it, counts
 * (as ubt_count_threshold) and copies the counts back into h_counts
 * (host int64[2 * n_tau]).  d_workspace must hold
 * ubt_count_host_workspace_size bytes.
 */
ubt_status ubt_count_host_workspace_size(int64_t n, int64_t m, size_t* h_bytes);
ubt_status ubt_count_host(int64_t n, int64_t m, const uint32_t* h_src, const uint32_t* h_dst,
                          const uint32_t* h_k, const double* h_tau, int32_t n_tau, int32_t prune,
                          int64_t* h_counts, void* d_workspace, size_t ws_bytes, void* stream);

/*
 * ubt_traversal_stats -- SYNC.  Sizes of the traversal a query at these
 * thresholds performs (for roofline accounting; computes nothing else):
 *   h_out[0]  forward-list entries loaded into hash tables (sum of the pruned
 *             |N>(u)|, Lemma 2)
 *   h_out[1]  forward pairs (u, v) visited (same as h_out[0])
 *   h_out[2]  entries of N>(v) streamed and probed, summed over the pairs
 *             (pruned by Lemma 2 / the order-free Lemma 3 form when prune = 1,
 *             under the same rule as the query)
 *   h_out[3]  vertices with >= 2 forward entries (tasks)
 */
ubt_status ubt_traversal_stats(ubt_graph* g, const double* h_tau, int32_t n_tau, int32_t prune,
                               int64_t* h_out, void* stream);

/*
 * ubt_query_guard -- SYNC.  Reads and clears the self-check word of the
 * graph's traversals: 0 when every check since the last call passed, else
 * (code << 56 | detail) of the first failure (1/2 hash-table probe limit in
 * find/insert, 3 neighbour id >= n, 4 list offsets out of range, 5 table
 * larger than its region, 6 an edge value outside [0, 1] given to
 * ubt_set_edge_values, detail = its input index).  A failed check skips the
 * access it guards.  ubt_count_threshold_noalloc reports here too.
 */
ubt_status ubt_query_guard(ubt_graph* g, int64_t* h_word, void* stream);

/*
 * ubt_graph_export -- SYNC.  Copies the built graph to host memory for
 * inspection (any pointer may be NULL):
 *   h_row_ptr  uint32[n + 1] forward-list offsets
 *   h_adj      uint64[m] entries (low 32 bits neighbour id, high 32 bits the
 *              value: q = 32768 - k as int32 for FIXED graphs, round(s 2^30)
 *              as int32 for REAL graphs)
 *   h_eid      uint32[m] input edge index of every entry
 *   h_lists    uint32[tasks] the work lists: owners of giant, hub and
 *              medium tasks
 *   h_list_sizes int64[4] the three list sizes and 0
 */
ubt_status ubt_graph_export(const ubt_graph* g, uint32_t* h_row_ptr, uint64_t* h_adj, uint32_t* h_eid,
                            uint32_t* h_lists, int64_t* h_list_sizes, void* stream);

/*
 * ubt_graph_export_pairs -- SYNC.  Copies the pair partition to host memory
 * (any pointer may be NULL).  Every forward edge x-s is one pair of the
 * traversal, owned by the endpoint x whose list is the hash table while the
 * list of s is streamed: the earlier vertex u of the edge u -> v (Alg. 1) or,
 * with the "pull" tuning on and |N>(v)| > |N>(u)|, the later vertex v.  Both
 * intersect N>(u) and N>(v), so each triangle is found once either way.
 *   h_pair_ptr uint32[n + 1] pairs of owner x are [h_pair_ptr[x], h_pair_ptr[x + 1])
 *   h_pairs    uint64[m] streamed vertex s (low 32 bits) and CSR position of
 *              the edge (high 32 bits); order within an owner is unspecified
 */
ubt_status ubt_graph_export_pairs(const ubt_graph* g, uint32_t* h_pair_ptr, uint64_t* h_pairs, void* stream);

/*
 * ubt_count_aeo -- ASYNC.  The counting problem (Def. 8) answered by the
 * improved method's edge iteration (Alg. 2): edges in Absolute Edge Order
 * (Def. AEO: |P+ - 0.5| descending, ties by (min id, max id)), skipping every
 * edge below a(t) (Lemma 2) and every partner edge below Lemma 3's cutoff for
 * the smallest t; each triangle is found from its first edge in that order.
 * Same arguments and results as ubt_count_threshold with prune = 1.  Needs a
 * graph built with UBT_OPT_UNDIRECTED (else UBT_ERR_UNSUPPORTED); with
 * UBT_OPT_EDGE_INDEX each edge's partners come from the shorter of its two
 * windows and the edge index, else from the owner's table.
 */
ubt_status ubt_count_aeo(ubt_graph* g, const double* h_tau, int32_t n_tau, int64_t* d_counts, void* stream);

/*
 * ubt_enumerate_aeo -- SYNC.  The enumeration problem (Def. 7) by the same
 * iteration; arguments and results as ubt_enumerate with prune = 1.
 */
ubt_status ubt_enumerate_aeo(ubt_graph* g, double tau, int32_t which, ubt_tri_rec* d_out, int64_t capacity,
                             int64_t* h_n_found, void* stream);

/*
 * ubt_edge_local_counts -- ASYNC.  Edge sampling (Algs. 5-6, Sec. 6): for
 * each of k sampled edges, the number of t-balanced and t-unbalanced
 * triangles that contain it (the improved local search: lists in Absolute
 * Edge Order, stopped at the pruning cutoffs), and the estimator
 * |E| / 3 * mean over the samples, for every threshold.
 *   d_edges     device uint32[k] input edge indices (the caller's uniform
 *               draws, repeats allowed); each < m
 *   h_tau       host double[n_tau], 1 <= n_tau <= 64, each in [0.5, 1]
 *   d_bal, d_unbal  device int64[k * n_tau], [sample][t]
 *   d_estimate  device double[2 * n_tau] (balanced, then unbalanced), or NULL
 * Needs UBT_OPT_UNDIRECTED.  An edge index >= m sets the query's self-check
 * word (ubt_query_guard) and counts as no triangle.
 */
ubt_status ubt_edge_local_counts(ubt_graph* g, const uint32_t* d_edges, int64_t k, const double* h_tau,
                                 int32_t n_tau, int64_t* d_bal, int64_t* d_unbal, double* d_estimate, void* stream);

/*
 * ubt_vertex_local_counts -- ASYNC.  Vertex sampling (Algs. 3-4): the same
 * for k sampled vertices (triangles through each vertex; estimator |V| / 3 *
 * mean).  d_vertices: device uint32[k], each < n.
 */
ubt_status ubt_vertex_local_counts(ubt_graph* g, const uint32_t* d_vertices, int64_t k, const double* h_tau,
                                   int32_t n_tau, int64_t* d_bal, int64_t* d_unbal, double* d_estimate,
                                   void* stream);

/*
 * ubt_vertex_topk -- ASYNC.  Per-vertex top-k (Sec. 5, top-k "locally for
 * each node"): for each of k listed vertices, its K triangles of highest
 * balance (which = 1) or unbalance (which = 2) probability, sorted by that
 * probability (descending), ties by (u, v, w).  Where more than 1,024 - (the
 * triangles strictly better than the K-th) triangles tie at the K-th value,
 * an arbitrary subset of the ties completes the vertex's answer.
 *   d_vertices  device uint32[k], each < n (larger ids set the self-check word)
 *   K           1..256
 *   d_out       device ubt_tri_rec[k * K]: vertex i's records at [i K, i K + d_n_out[i])
 *   d_n_out     device int32[k]: min(K, triangles through the vertex)
 * Needs UBT_OPT_UNDIRECTED.
 */
ubt_status ubt_vertex_topk(ubt_graph* g, const uint32_t* d_vertices, int64_t k, int32_t K, int32_t which,
                           ubt_tri_rec* d_out, int32_t* d_n_out, void* stream);

/*
 * ubt_graph_export_undirected -- SYNC.  Copies the undirected adjacency of a
 * graph built with UBT_OPT_UNDIRECTED to host memory (any pointer may be
 * NULL; UBT_ERR_UNSUPPORTED without the option).  Row x holds every edge at x,
 * sorted by |q| descending then neighbour id (Absolute Edge Order restricted
 * to the edges at x), packed like h_adj of ubt_graph_export.
 *   h_uptr uint32[n+1]; h_uadj uint64[2m]; h_ueid uint32[2m] input edge index;
 *   h_umir uint32[2m] position of the same edge in the other endpoint's row;
 *   h_apair_ptr uint32[n+1], h_apairs uint64[m]: the edges ubt_count_aeo
 *   handles from x (the endpoint with the longer row, ties to the larger id):
 *   the other endpoint (low 32 bits), the edge's position in x's row (high).
 */
ubt_status ubt_graph_export_undirected(const ubt_graph* g, uint32_t* h_uptr, uint64_t* h_uadj, uint32_t* h_ueid,
                                       uint32_t* h_umir, uint32_t* h_apair_ptr, uint64_t* h_apairs, void* stream);

/*
 * ubt_topk_workspace_size / ubt_topk -- SYNC.  Top-k query (Sec. 5, "Adaption
 * to Top-k Search"): the K triangles of highest balance probability (which =
 * 1) or highest unbalance probability (which = 2), as records sorted by that
 * probability (descending), ties by (u, v, w).  Where ties at the K-th value
 * exceed the candidate buffer, an arbitrary subset of the tied triangles
 * completes the answer.  The threshold is raised as the search narrows: each
 * pass counts the triangle products at 64 cut points with pruning at the
 * level the current range allows, until the candidates fit; the candidates
 * are then enumerated and sorted on the device.
 *   K           1 <= K <= 2^26
 *   d_out       device ubt_tri_rec[K]
 *   h_n_out     number of records written (min(K, number of triangles))
 *   d_work      device workspace of ubt_topk_workspace_size(K) bytes
 */
ubt_status ubt_topk_workspace_size(int64_t K, size_t* h_bytes);
ubt_status ubt_topk(ubt_graph* g, int64_t K, int32_t which, ubt_tri_rec* d_out, int64_t* h_n_out, void* d_work,
                    size_t work_bytes, void* stream);

/*
 * ubt_set_tuning / ubt_get_tuning -- process-wide launch parameters that the
 * autotuner picks (they change speed, never results).  Unknown names return
 * UBT_ERR_INVALID_ARG.  Names:
 *   "count_visitor"   threshold counts: 0 (default) classify each triangle
 *                     in the lane that finds it (binned by a slice table);
 *                     1 queue products per warp and classify 32 at a time
 *                     (by binary search over the levels, or compared with
 *                     every threshold for at most 8)
 *   "pull"            1 (default): a pair is owned by the endpoint whose
 *                     list is longer, so the shorter list is streamed; 0:
 *                     always by the earlier vertex (Alg. 1 as written)
 *   "hub_threshold"   owners with longer lists than this are whole-block
 *                     tasks (default 128)
 *   "block_work"      owners whose pairs stream more entries than this are
 *                     whole-block tasks too (default 16384)
 *   "block_threads"   threads per block of the block-task kernel (64..512,
 *                     /32, default 512)
 *   "warp_threads"    threads per block of the warp-task kernel (64..512,
 *                     /32, default 128)
 *   "blocks_per_sm"   cap on resident blocks per SM (1..32; occupancy decides
 *                     below it)
 *   "smem_table_max"  hash-table slots kept in shared memory (power of two);
 *                     longer lists use a table in global scratch
 *   "block_unit"      pairs a warp takes at a time inside a block task (1..32,
 *                     default 16)
 *   "long_min"        streamed lists at least this long are streamed by the
 *                     whole warp, up to four entries per lane (default 64);
 *                     shorter ones are concatenated across the warp's pairs
 *   "long_tail"       1 (default): the last < 64 entries of a long list are
 *                     concatenated with the short lists; 0: the warp streams
 *                     them itself with idle lanes
 *   "edge_index"      on a graph with UBT_OPT_EDGE_INDEX: 0 never use the
 *                     index; 1 (default) vertex local counts / per-vertex
 *                     top-k use it for a neighbour whose row is more than 8
 *                     times longer than the pairs left to check, and the AEO
 *                     calls use its form; 2 as 1, the vertex queries for every
 *                     neighbour
 *   "vertex_split"    ubt_vertex_local_counts on a graph with the edge index:
 *                     samples whose pruned row is longer (default 64) are
 *                     spread over the warps of all blocks by a second launch
 *                     (at most 1,024 per call; the rest are counted by one
 *                     block each)
 *   "world_words_per_pass"  64-world words per traversal of ubt_sample_worlds
 *                     (1, 2, 4, 8, 16, 32 or 64)
 *   "small_batch"     warp tasks taken per grab of a task counter
 *   "sort_smem_max"   longest forward list sorted in shared memory during the
 *                     build (power of two, 64..4096); longer lists are sorted
 *                     in a global-memory slice
 *   "warp_sort_max"   longest forward list sorted by one warp in registers
 *                     during the build (128, 256 or 512; at most
 *                     sort_smem_max unless 128); longer lists up to
 *                     sort_smem_max are sorted by one block in shared memory
 * Build-time knobs (pull, hub_threshold, block_work, smem_table_max,
 * sort_smem_max, warp_sort_max) apply to graphs created afterwards; query the workspace size
 * after setting them.
 */
ubt_status ubt_set_tuning(const char* name, int64_t value);
ubt_status ubt_get_tuning(const char* name, int64_t* h_value);

#ifdef __cplusplus
}
#endif
#endif /* UBT_H */
