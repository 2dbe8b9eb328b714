/*
 * rp.h -- C ABI of the GB300 RP-Tuning library (librp.so).
 *
 * RP-Tuning (§3, "RP-Tuning" paragraph) re-runs RobustPrune (Algorithm 1) on
 * every node of an existing graph, each node reading only its own input
 * out-neighbour list, to lower alpha and/or the degree bound R without
 * rebuilding the index.  GreedySearch (Algorithm 2) from the medoid (§4.1)
 * queries the tuned graph.  Everything below runs in this library's own CUDA
 * kernels on one GPU.
 *
 * Conventions shared by every call
 * --------------------------------
 * - Every call returns an rp_status.  RP_OK is 0; errors are negative.  On an
 *   error, rp_last_error(ctx) returns a message owned by the context and valid
 *   until the next call on that context.  No C++ exception and no abort ever
 *   crosses this boundary.  A device-side problem found by a kernel (a bad
 *   index in an input graph, a canonical-tie run that could not be resolved)
 *   is reported as RP_EDEVICE with the first offending index in the message;
 *   kernels never trap.
 * - Vectors are row-major, n rows of d elements, element type RP_U8 (uint8)
 *   or RP_F32 (IEEE binary32).  Distances are squared Euclidean (the paper
 *   uses Euclidean distance for every dataset, §4.1); ordering by squared
 *   distance equals ordering by distance.
 * - Graphs are CSR: row_ptr int64[n+1] (row_ptr[0] = 0, non-decreasing),
 *   col int32[row_ptr[n]], ids in [0, n).  N_out(p) = col[row_ptr[p] ..
 *   row_ptr[p+1]).
 * - mem_flags = RP_MEM_HOST: pointers are host memory; the call copies inputs
 *   in, and copies outputs back before returning.  RP_MEM_DEVICE: pointers
 *   are device memory on the context's device; the call reads and writes them
 *   in order on the context's stream and may return before the work is done
 *   (rp_sync waits).  Input buffers are borrowed only for the duration of the
 *   call (until the stream reaches it, for device pointers).
 * - Graph handles (rp_graph) name device-resident graphs owned by the
 *   context.  They stay resident until rp_graph_free or rp_destroy.  A tuned
 *   graph shares the vectors of the graph it was tuned from.
 * - alpha must be >= 1 and a multiple of 0.001 (|1000 alpha - round(1000
 *   alpha)| < 1e-6); it is carried exactly as A = round(1000 alpha).  The
 *   domination test alpha * D(p*, v) <= D(p, v) of Algorithm 1 is evaluated
 *   as A^2 * d2(p*, v) <= 10^6 * d2(p, v): exactly in integers for RP_U8, and
 *   for RP_F32 with the same decision as the binary64 expression
 *   fl(A^2 * d2a) <= fl(1e6 * d2b) where d2 is summed in index order in
 *   binary64 without fused multiply-add (decisions whose single-precision
 *   margin is below a rigorous error bound are recomputed that way on the GPU).
 * - R >= 1; RP_R_INF (INT32_MAX) means no degree bound, as RP-Tuning is
 *   stated in §3.
 * - Calls on one context are serialised by the context; use one context per
 *   host thread for concurrency.
 */
#ifndef RP_H_
#define RP_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct rp_ctx rp_ctx;
typedef int32_t rp_status;
typedef int64_t rp_graph;

enum {
  RP_OK = 0,
  RP_EINVAL = -1,    /* bad argument or malformed input */
  RP_ENOMEM = -2,    /* the request would exceed the context's HBM budget */
  RP_ECUDA = -3,     /* a CUDA runtime call failed */
  RP_ETIMEOUT = -4,  /* a bounded wait ran out */
  RP_ENOTFOUND = -5, /* unknown graph handle */
  RP_EDEVICE = -6    /* a kernel reported a problem through its status word */
};

enum { RP_U8 = 1, RP_F32 = 2 };
enum { RP_SORTED = 0, RP_UNSORTED = 1 };
enum { RP_MEM_HOST = 0, RP_MEM_DEVICE = 1 };

#define RP_R_INF INT32_MAX
/* Largest out-degree a graph may have after cleaning (rp_load_graph). */
#define RP_MAX_DEGREE 8192
/* Largest beam width L accepted by rp_search. */
#define RP_MAX_L 1024

/*
 * rp_create: make a context on CUDA device `device`.
 *   hbm_budget_bytes: cap on the device memory the context may hold at once
 *     (vectors, graphs and scratch); 0 means "no cap beyond the device".
 *   cuda_stream: a cudaStream_t to order all work on (e.g. PyTorch's current
 *     stream), or NULL for a stream the context creates and owns.
 * Errors: RP_EINVAL (no such device, out == NULL), RP_ECUDA.
 */
rp_status rp_create(rp_ctx **out, int32_t device, uint64_t hbm_budget_bytes, void *cuda_stream);

/* rp_destroy: wait for outstanding work, free every graph and the context. */
rp_status rp_destroy(rp_ctx *ctx);

/* rp_last_error: message for the last failed call on ctx ("" if none). */
const char *rp_last_error(const rp_ctx *ctx);

/* rp_sync: block until all work enqueued on the context's stream is done,
 * then report any device status word raised since the last check. */
rp_status rp_sync(rp_ctx *ctx);

/*
 * rp_load_graph: make vectors and a graph resident (§2, a graph index
 * G = (P, E) over the dataset P; Algorithm 1's first step drops p from its
 * own candidate set and treats N_out(p) as a set).
 *   vectors: n x d elements of `dtype`, row-major.
 *   row_ptr, col: the graph in CSR; row_ptr == NULL loads the vectors with
 *     an empty graph (every out-degree 0), e.g. as the data source of
 *     rp_build_knn_base.
 *   start: the GreedySearch start vertex, or -1 for the medoid, read as the
 *     data point nearest (binary64, index-order sums) to the binary64 mean
 *     vector, ties to the smaller id (§4.1 names the medoid; this reading
 *     keeps it computable at n = 10^7).  The medoid takes two more passes
 *     over the vectors; a stored index passes the start vertex it was built
 *     with and skips them.
 * Cleaning: self loops are dropped and repeated ids keep their first
 * occurrence; the cleaned graph is what every later call sees.  Counts of
 * dropped entries are available through rp_stats.
 * Errors: RP_EINVAL (n < 1, d < 1, bad dtype, row_ptr not monotone, an id
 *   outside [0, n), a cleaned out-degree above RP_MAX_DEGREE, start >= n, a
 *   float value above 2^50 in magnitude: squared distances of such rows could
 *   leave the single-precision range the bounded tiers work in);
 *   RP_ENOMEM (over budget); RP_ECUDA.
 */
rp_status rp_load_graph(rp_ctx *ctx, const void *vectors, int32_t dtype, int64_t n, int32_t d,
                        const int64_t *row_ptr, const int32_t *col, int32_t start,
                        int32_t mem_flags, rp_graph *base_out);

/*
 * rp_tune: RP-Tuning (§3) of graph `src` to one target: for every node p,
 * N_out'(p) = RobustPrune(p, N_out(p), alpha, R) (Algorithm 1), computed from
 * src's lists only.  variant RP_SORTED takes p* = argmin D(p, .) with ties to
 * the smaller id; RP_UNSORTED (UnsortedRobustPrune, §3) takes the first
 * remaining candidate in src's stored order.  The new list of p holds the
 * kept points in the order they were added.  The result is a new graph
 * sharing src's vectors; *out receives its handle.
 * Errors: RP_ENOTFOUND, RP_EINVAL (alpha off the 0.001 grid or < 1, R < 1,
 *   bad variant), RP_ENOMEM, RP_ECUDA, RP_EDEVICE.
 */
rp_status rp_tune(rp_ctx *ctx, rp_graph src, double alpha, int32_t R, int32_t variant,
                  rp_graph *out);

/*
 * rp_tune_batch: T targets (alphas[t], Rs[t]) of the same source in one
 * persistent launch; each node's sort, pairwise distances and margins are
 * computed once and shared by all targets.  outs[t] receives the graph that
 * rp_tune(src, alphas[t], Rs[t], variant) would return (identical edges and
 * order).  1 <= T <= 16.  Repeated calls with the same (src, targets,
 * variant) replay a captured CUDA graph.
 * Errors: as rp_tune; RP_EINVAL for T outside [1, 16].
 */
rp_status rp_tune_batch(rp_ctx *ctx, rp_graph src, const double *alphas, const int32_t *Rs,
                        int32_t T, int32_t variant, rp_graph *outs);

/*
 * rp_debug_gram: test support, not part of the hot path.  The split-f16
 * tcgen05 Gram of float rows exactly as the prune kernel forms it (the same
 * operand stores, MMA sequence and combination of its two accumulators),
 * 128 rows at a time: out[(128 g + i) * 128 + j] = G~(y_i, y_j) for the rows
 * y_i = x[rows[128 g + i]] - c_i, where c_i = x[centres[2 g + i / 64]] (each
 * 64-row half centred on its own pivot, at the prune's scale for centred
 * rows), or c_i = 0 when centres is NULL.  Tests hold every entry against the
 * exact inner product and the error bound the float decision tiers assume.
 *   rows: host int32[nrows], nrows a multiple of 128, ids in [0, n);
 *   centres: host int32[nrows / 64], ids in [0, n), or NULL;
 *   out: host float[nrows * 128].
 * Errors: RP_ENOTFOUND, RP_EINVAL (uint8 vectors, a bad row count or id),
 *   RP_ENOMEM, RP_ECUDA, RP_EDEVICE.
 */
rp_status rp_debug_gram(rp_ctx *ctx, rp_graph g, const int32_t *rows, const int32_t *centres, int64_t nrows,
                        float *out);

/*
 * rp_graph_attach: a graph over the vectors (and start vertex) of graph `data`
 * from a CSR adjacency, cleaned as rp_load_graph cleans it (ids checked to lie
 * in [0, n), self loops and repeated ids dropped), without uploading the
 * vectors again.  A multi-GPU tuning assembles the node-range slices of the
 * ranks into one graph this way (each rank then searches it).
 *   row_ptr: int64[n + 1], col: int32[row_ptr[n]], host or device memory
 *     (mem_flags), borrowed for the call.
 * Errors: RP_ENOTFOUND, RP_EINVAL (a malformed CSR or an id out of range),
 *   RP_ENOMEM, RP_ECUDA.
 */
rp_status rp_graph_attach(rp_ctx *ctx, rp_graph data, const int64_t *row_ptr, const int32_t *col,
                          int32_t mem_flags, rp_graph *out);

/*
 * rp_tune_batch_async: rp_tune_batch on a stream of the lowest priority, the
 * prune cut into `chunks` launches over node ranges, so that work the context
 * runs meanwhile on its own stream (searches, which the context gives the
 * highest priority when it creates that stream) takes the GPU between them.
 * The graphs in outs[0..T) exist at once but must not be used (searched,
 * exported, tuned from or freed) until rp_tune_wait(ticket) has returned
 * RP_OK.  One job runs at a time: a call waits for the previous job to
 * finish.  Results equal rp_tune_batch's.  The paper has no counterpart; this
 * is the serving layer's way to keep searches running during a prune.
 *   chunks in [1, 4096]; *ticket receives the job's ticket (1, 2, ...).
 * Errors: as rp_tune_batch, and RP_EINVAL for a bad chunk count.
 */
rp_status rp_tune_batch_async(rp_ctx *ctx, rp_graph src, const double *alphas, const int32_t *Rs,
                              int32_t T, int32_t variant, int32_t chunks, rp_graph *outs,
                              int64_t *ticket);

/*
 * rp_tune_wait: wait up to timeout_ms (0 = do not wait) for tuning job
 * `ticket`.  RP_OK once its graphs are in place, RP_ETIMEOUT if not yet,
 * RP_ENOTFOUND for an unknown ticket, RP_EDEVICE if a kernel reported a
 * problem, RP_EINVAL for timeout_ms < 0.
 */
rp_status rp_tune_wait(rp_ctx *ctx, int64_t ticket, int32_t timeout_ms);

/*
 * rp_graph_info: n, number of edges, largest out-degree and start vertex of
 * a graph (waits for the graph to be complete).  Any output pointer may be
 * NULL.  Errors: RP_ENOTFOUND, RP_ECUDA.
 */
rp_status rp_graph_info(rp_ctx *ctx, rp_graph g, int64_t *n, int64_t *nnz, int32_t *max_deg,
                        int64_t *start);

/*
 * rp_graph_export: copy a graph out as CSR (row_ptr int64[n+1], col
 * int32[nnz]) into caller buffers; col_cap is the capacity of col in
 * elements.  Errors: RP_ENOTFOUND, RP_EINVAL (col_cap < nnz; call
 * rp_graph_info for nnz), RP_ECUDA.
 */
rp_status rp_graph_export(rp_ctx *ctx, rp_graph g, int64_t *row_ptr, int32_t *col,
                          int64_t col_cap, int32_t mem_flags);

/*
 * rp_search: GreedySearch(s, q, k, L) (Algorithm 2) on graph g for each of
 * the nq query rows (nq x d, the graph's dtype), s = the graph's start
 * vertex.  L is the search list size, L >= k (Algorithm 2's input condition).
 * The list is ordered by (distance, id); the loop ends when every member has
 * been expanded; the k closest members are returned.
 *   ids: int32[nq * k]; -1 where fewer than k points were reached.
 *   dists: float[nq * k] squared distances (exact integers for RP_U8; for
 *     RP_F32 single precision, with orderings decided as in binary64), +inf
 *     where ids is -1.  dists may be NULL.
 * Errors: RP_ENOTFOUND, RP_EINVAL (nq < 0, k < 1, L < k, L > RP_MAX_L),
 *   RP_ENOMEM, RP_ECUDA.
 */
rp_status rp_search(rp_ctx *ctx, rp_graph g, const void *queries, int64_t nq, int32_t L,
                    int32_t k, int32_t *ids, float *dists, int32_t mem_flags);

/*
 * rp_search_multi: one launch of GreedySearch (Algorithm 2) over queries that
 * address different graphs and list sizes -- the mixed batch a serving loop
 * collects.  The paper has no counterpart; each query's result is exactly what
 * rp_search(ctx, graphs[q_graph[i]], query i, q_L[i], k) returns, since every
 * query is searched on its own.
 *   graphs: ngraphs >= 1 resident graphs that share their vectors (tuned
 *     from one base, or the base itself).
 *   q_graph, q_L: int32[nq] host arrays: the graph index (in [0, ngraphs))
 *     and the list size (k <= q_L[i] <= RP_MAX_L) of each query.
 *   queries, ids, dists, mem_flags: as rp_search.
 * Errors: RP_ENOTFOUND, RP_EINVAL (an index or list size out of range, graphs
 *   with different vectors, k < 1), RP_ENOMEM, RP_ECUDA, RP_EDEVICE.
 */
rp_status rp_search_multi(rp_ctx *ctx, const rp_graph *graphs, int32_t ngraphs,
                          const int32_t *q_graph, const int32_t *q_L, const void *queries,
                          int64_t nq, int32_t k, int32_t *ids, float *dists, int32_t mem_flags);

/*
 * rp_search_noalloc: the GreedySearch of rp_search for callers that cannot
 * allocate device memory.  The paper has no counterpart: this entry point
 * exists for processes that reserve all device memory up front (an inference
 * engine's pool, an arena shared with other models) and for callers that must
 * not have allocations appear while they capture a stream.  It takes no
 * context, allocates nothing (no cudaMalloc, cudaMallocAsync or cudaFree, no
 * allocating library routine) and uses instead a fixed scratch array of
 * RP_NOALLOC_SCRATCH_BYTES (a status word and a query counter) that every GPU
 * loading this library holds until the process exits.
 *   vectors: n x d elements of dtype, device memory, rows packed (stride
 *     d * element size, which must be a multiple of 16 bytes; pointer
 *     16-byte aligned).  Float rows must be finite with |x| <= 2^50, as
 *     rp_load_graph requires; this call does not check them (the bounds of
 *     the float ordering tiers and the (distance, id) order rest on it).
 *   row_ptr, col: the graph in CSR on the device; ids must lie in [0, n) and
 *     rows must hold no repeated id (graphs from rp_graph_export qualify).
 *   start: the start vertex in [0, n).
 *   queries: nq x d elements of dtype, device memory, same stride rule.
 *   ids: int32[nq * k], dists: float[nq * k] or NULL (distances not
 *     written), device memory; same contents as rp_search's outputs.
 *   cuda_stream: the stream to run on (NULL: the legacy default stream).
 * The call is asynchronous on cuda_stream and runs on the current device.
 * Outside a stream capture every call looks up the scratch array's device
 * address (cudaGetSymbolAddress), so a device reset between calls is safe; a
 * call inside a capture reuses the address the last uncaptured call on that
 * device found, so make one call outside any capture first.
 * All calls share the one array and each clears it at its start, so calls
 * whose work overlaps on the GPU (other streams, other threads) race and must
 * be serialised by the caller.
 * Errors (checked on the host, before any work is enqueued): RP_EINVAL for a
 * bad argument or a stride or pointer alignment off 16 bytes; RP_ECUDA if
 * the symbol lookup or a launch fails.  Problems the kernel detects on the
 * device go to the status word of the scratch array: read them with
 * rp_search_noalloc_status.
 */
#define RP_NOALLOC_SCRATCH_BYTES 4096u
rp_status rp_search_noalloc(const void *vectors, int32_t dtype, int64_t n, int32_t d,
                            const int64_t *row_ptr, const int32_t *col, int64_t start,
                            const void *queries, int64_t nq, int32_t L, int32_t k, int32_t *ids,
                            float *dists, void *cuda_stream);

/*
 * rp_search_noalloc_status: the device status of the last rp_search_noalloc
 * call on the current device.  It waits for cuda_stream (the stream that call
 * ran on), then reads the status word of the scratch array into host memory
 * (no allocation).  Returns RP_OK if the kernel reported nothing, RP_EDEVICE if
 * it reported a problem (*info, if info is not NULL, receives the offending
 * query index), RP_EINVAL inside a stream capture (it must wait for the
 * stream), RP_ECUDA if the wait or the read fails.  A later rp_search_noalloc
 * call on the same device clears the word, so read it before the next call.
 */
rp_status rp_search_noalloc_status(void *cuda_stream, int64_t *info);

/*
 * rp_knn: exact k nearest neighbours by brute force over the vectors of
 * graph g, ordered by (distance, id) -- the ground truth of k-recall@k (§4).
 *   queries: nq x d rows of g's dtype, or NULL to use the base points
 *     0 .. nq-1 themselves, each excluded from its own list.
 *   ids int32[nq * k], dists float[nq * k] (dists may be NULL); -1 / +inf pad.
 * Errors: RP_ENOTFOUND, RP_EINVAL (k < 1 or k > 1024, nq > n when queries
 *   is NULL), RP_ENOMEM, RP_ECUDA, RP_EDEVICE.
 */
rp_status rp_knn(rp_ctx *ctx, rp_graph g, const void *queries, int64_t nq, int32_t k,
                 int32_t *ids, float *dists, int32_t mem_flags);

/*
 * rp_reachability: alpha-reachability of graph g (Definition 2.1), per node.
 * The term of node p is the min over q != p with (p, q) not an edge of the
 * max over p' in N_out(p) of D(p, q) / D(p', q), with D = Euclidean distance.
 * D(p', q) = 0 gives +inf. A node without out-neighbours gives 0; a node with
 * no such q gives +inf. g is alpha-reachable exactly for alpha <= alpha*(g),
 * the minimum of the terms over all nodes.
 * Distances: uint8 exact; float32 the canonical binary64 difference form; D
 * and the ratio in IEEE binary64, so the terms are exact.
 *   nodes: host int64[n_nodes], the nodes to measure, or NULL for every node
 *     (n_nodes is then ignored). Cost: about n * (deg + 1) * d per node, so
 *     at scale pass a sample.
 *   per_node: host double[n_nodes or n] receiving the terms (may be NULL).
 *   alpha_star: host double receiving their minimum, +inf for no node (may be
 *     NULL). Over a sample it is an upper bound of alpha*(g).
 * Errors: RP_ENOTFOUND, RP_EINVAL (both outputs NULL, n_nodes < 0, a node
 *   outside [0, n)), RP_ENOMEM, RP_ECUDA, RP_EDEVICE.
 */
rp_status rp_reachability(rp_ctx *ctx, rp_graph g, const int64_t *nodes, int64_t n_nodes, double *per_node,
                          double *alpha_star);

/*
 * rp_recall: k-recall@k (§4: the share of the true k nearest neighbours
 * found among the k returned).  found: int32[nq * ld_found], truth:
 * int32[nq * ld_truth]; the first k entries of each row are compared;
 * negative ids never match.  *hits receives the total number of matches,
 * so recall = hits / (nq * k).
 * Errors: RP_EINVAL (k < 1, ld < k), RP_ECUDA.
 */
rp_status rp_recall(rp_ctx *ctx, const int32_t *found, int32_t ld_found, const int32_t *truth,
                    int32_t ld_truth, int64_t nq, int32_t k, int64_t *hits, int32_t mem_flags);

/*
 * rp_build_knn_base: a base graph for tuning, built as RobustPrune(p, kNN(p),
 * alpha, R) for every p (Algorithm 1 over each point's exact `kcand` nearest
 * neighbours, excluding p).  The paper's base graphs are Vamana graphs
 * (§4.1); this kNN-candidate form stands in for them.  Uses the vectors of
 * graph `data`; *out shares them.  1 <= kcand <= 128.
 * Errors: as rp_knn and rp_tune.
 */
rp_status rp_build_knn_base(rp_ctx *ctx, rp_graph data, int32_t kcand, double alpha, int32_t R,
                            rp_graph *out);

/*
 * rp_build_knn_random_base: as rp_build_knn_base, with each point's
 * candidates being its exact kcand nearest neighbours followed by nrand ids
 * drawn uniformly from the other points (counter-based: splitmix64 of seed,
 * the point and the draw), repeats dropped.  The random candidates give the
 * base the long edges that a Vamana graph gets from its random start (§4.1),
 * which a pure kNN graph of well-separated clusters lacks (its search cannot
 * leave the start's cluster).  0 <= nrand <= 128.
 * Errors: as rp_build_knn_base.
 */
rp_status rp_build_knn_random_base(rp_ctx *ctx, rp_graph data, int32_t kcand, int32_t nrand,
                                   uint64_t seed, double alpha, int32_t R, rp_graph *out);

/*
 * rp_build_vamana: a Vamana graph, the "fast preprocessing" construction of
 * §2.1 with which §4.1 builds the paper's base indices (alpha1 = 1.2,
 * L_build = 75).  The paper does not open the construction; this is its
 * batched reading.  The graph starts empty; the points are inserted in the
 * order perm[0 .. n) in batches of 1, 2, 4, ... points, at most max_batch.
 * Every point p of a batch searches the graph as it stood when the batch
 * began (Algorithm 2 from the start vertex, list size L; its first vcap
 * visited points V_p, in expansion order), then N_out(p) <- RobustPrune(p,
 * V_p, alpha, R) (Algorithm 1, sorted; its first step adds the current
 * N_out(p)).  Then every point j kept by some batch point takes those points
 * as back edges, ascending by id and at most 512 of them (the smallest ids),
 * after its current list; a list that grows past R is pruned again,
 * RobustPrune(j, merged list, alpha, R).  Pass i
 * inserts every point with alpha = alphas[i] (the original construction runs
 * alpha = 1, then alpha1).  The result is fully determined by these rules.
 *   data: a graph whose vectors and start vertex are used (its edges are not).
 *   perm: host int32[n], a permutation of 0 .. n-1, or NULL for 0 .. n-1.
 *   npass in [1, 8]; alphas: host double[npass], each >= 1 on the 0.001 grid.
 *   R in [1, 1024]; L in [1, RP_MAX_L]; vcap in [1, 4096]; max_batch >= 1.
 *   visited_cut: if not NULL, receives how many searches expanded more than
 *     vcap points (their V_p was cut to the first vcap).
 *   out: receives the graph (CSR, each list in its stored order; vectors
 *     shared with data).
 * Errors: RP_ENOTFOUND, RP_EINVAL (a bad argument or perm), RP_ENOMEM,
 *   RP_ECUDA, RP_EDEVICE.
 */
rp_status rp_build_vamana(rp_ctx *ctx, rp_graph data, const int32_t *perm, int32_t npass, const double *alphas,
                          int32_t R, int32_t L, int32_t vcap, int64_t max_batch, int64_t *visited_cut,
                          rp_graph *out);

/*
 * rp_graph_slice: the part of graph g that one of several GPUs tunes when the
 * nodes are split by contiguous id ranges (RP-Tuning treats every node on its
 * own, §3).  *out keeps the rows of nodes lo .. hi-1 with their edges, in
 * order, and has no edges elsewhere; it shares g's vectors and start vertex.
 * Tuning it gives exactly the rows of lo .. hi-1 of tuning g, and empty rows
 * elsewhere.  Errors: RP_ENOTFOUND, RP_EINVAL (not 0 <= lo <= hi <= n),
 * RP_ENOMEM, RP_ECUDA.
 */
rp_status rp_graph_slice(rp_ctx *ctx, rp_graph g, int64_t lo, int64_t hi, rp_graph *out);

/*
 * rp_graph_shape: the vectors behind graph g (d and dtype) and the device
 * bytes of g's own adjacency (row_ptr and col capacity, vectors excluded).  A
 * graph tuned from g holds the same number of adjacency bytes.  Any output
 * pointer may be NULL.  Errors: RP_ENOTFOUND.
 */
rp_status rp_graph_shape(rp_ctx *ctx, rp_graph g, int32_t *d, int32_t *dtype, uint64_t *adj_bytes);

/* rp_graph_free: release a graph (its vectors are freed with the last graph
 * that uses them).  Errors: RP_ENOTFOUND. */
rp_status rp_graph_free(rp_ctx *ctx, rp_graph g);

/* Counters of the context since rp_create (or the last reset). */
typedef struct {
  int64_t nodes_pruned;        /* node x target pairs processed by the prune kernels */
  int64_t fp64_decisions;      /* domination tests settled by the binary64 recheck */
  int64_t fp64_sort_keys;      /* pivot keys recomputed in binary64 to order near-ties */
  int64_t fp64_search_dists;   /* search distances recomputed in binary64 for ordering */
  int64_t self_loops_dropped;  /* rp_load_graph cleaning */
  int64_t duplicates_dropped;  /* rp_load_graph cleaning */
  int64_t generic_nodes;       /* nodes handled by the large-degree path */
  int64_t graph_replays;       /* rp_tune_batch calls served from a captured CUDA graph */
  uint64_t bytes_in_use;       /* device bytes held by the context */
  uint64_t bytes_peak;
  int64_t kernel_launches;     /* kernels of this library launched (graph replays included) */
  float last_prune_ms;         /* device time of the prune kernels of the last tuning call */
  float last_emit_ms;          /* device time of its CSR emit (scan + compaction) */
  float last_search_ms;        /* device time of the last rp_search kernel */
  int32_t tile0;               /* prune configuration of the last tuning call (rp_set_tuning) */
  int32_t ctas_per_sm;
  int32_t knn_method;          /* path of the last rp_knn / rp_build_knn_base (RP_KNN_*) */
  int32_t pad_;
  int64_t f32_rechecks;        /* float domination tests redone in single-precision difference form */
} rp_stats_t;

rp_status rp_stats(rp_ctx *ctx, rp_stats_t *out, int32_t reset);

/*
 * rp_set_tuning: how the tensor-core prune kernels are configured.  The
 * paper fixes no kernel shape; these are this library's choices.
 *   tile0: 0 = two nodes of degree <= 64 share one 128-row Gram MMA,
 *          1 = one node per MMA (the shape of the 65..128 degree bucket).
 *   ctas_per_sm: CTAs per SM of those kernels, 0 = as many as fit (<= 4).
 * RP_TUNING_AUTO (the default): the first tuning call from a source graph
 * with at least 65,536 nodes of degree <= 64 times every (tile0, ctas_per_sm)
 * in {0, 1} x {all, 3, 2} on a 32,768-node sample and keeps the fastest for
 * that source, target-count class (1, 2, 4, 8, 16) and variant; smaller
 * sources use tile0 = 0 with all CTAs.  RP_TUNING_FIXED uses the given pair.
 * Results never depend on the configuration.  rp_stats reports the one used
 * by the last tuning call.  Errors: RP_EINVAL.
 */
enum { RP_TUNING_AUTO = 0, RP_TUNING_FIXED = 1 };
rp_status rp_set_tuning(rp_ctx *ctx, int32_t mode, int32_t tile0, int32_t ctas_per_sm);

/*
 * rp_set_knn_method: which exact kNN scan rp_knn and rp_build_knn_base use.
 * Both return the same lists (exact top k by (distance, id)).
 *   RP_KNN_CUDA_CORE: every pair's distance on CUDA cores.
 *   RP_KNN_TENSOR: a Gram on tcgen05 filters candidates with a rigorous
 *     error bound (uint8 rows of d <= 128: exact f16 products, no bound;
 *     float rows: each split into two f16 operands, hi and 2^11 times the
 *     remainder, bound near 2^-22 |q||p|), and the survivors are ranked
 *     exactly; needs k <= 128 and uint8 rows of d <= 128 or float rows of
 *     d <= 128 (RP_EINVAL otherwise).  Holds an f16 copy of the vectors
 *     (n x d x 2 bytes, twice that for float rows) for the call.
 *   RP_KNN_AUTO (default): RP_KNN_TENSOR where it applies.
 * Errors: RP_EINVAL.
 */
enum { RP_KNN_AUTO = 0, RP_KNN_CUDA_CORE = 1, RP_KNN_TENSOR = 2 };
rp_status rp_set_knn_method(rp_ctx *ctx, int32_t method);

/*
 * rp_set_search_config: the launch plan of rp_search and rp_search_multi.
 * The paper fixes none; results never depend on it.
 *   cache_bits: 8..12, a direct-mapped cache of 2^cache_bits recently met
 *     ids per query in shared memory (a miss only costs one more distance);
 *     0 = 256 or 512 entries, the larger if it keeps the most CTAs (of 4
 *     queries each) resident per SM that registers and shared memory allow.
 *   ctas_per_sm: at most this many CTAs per SM (0 = as many as one SM
 *     holds with the chosen cache, up to 16).
 * Errors: RP_EINVAL.
 */
rp_status rp_set_search_config(rp_ctx *ctx, int32_t cache_bits, int32_t ctas_per_sm);

/* ------------------------------------------------------------------------
 * Serving: a scheduler thread over one resident base graph that takes
 * prune-to-(alpha, R) jobs and query batches as they arrive (continuous
 * batching).  The paper tunes one graph at a time; serving many targets from
 * one base is this library's extension of §3's RP-Tuning (every tuned graph
 * is still computed from the base, never chained).
 *
 * Each scheduling round admits the waiting requests in arrival order while
 * (a) the distinct tuned graphs they address fit in the graph budget and
 * (b) their queries fit in max_batch_queries (the first waiting request is
 * always admitted).  Requests on graphs that are already resident (or on the
 * base) run first and complete at once: their searches in one mixed launch
 * per k (rp_search_multi).  The round then evicts least-recently-used tuned
 * graphs that none of its requests address until the new ones fit, tunes all
 * missing graphs in batched launches (up to 16 targets each), and runs the
 * remaining searches in one mixed launch per k.  Results depend only on each
 * request, never on the mix.  With an executor that tunes asynchronously
 * (rp_server_create's does), a round does not wait for its tuning: requests
 * on graphs being tuned are parked, rounds keep admitting arrivals and
 * running searches on resident graphs while the job runs (on the device the
 * searches take the SMs between the job's chunks), and the parked requests
 * run once their graphs are in; the next job starts when one finishes.  With
 * `serial` set the scheduler is the plain path instead: one request per
 * round, one target per tuning launch, each waited for.
 * ---------------------------------------------------------------------- */
typedef struct rp_server rp_server;

/* The operations a server runs, with their rp_ctx counterparts: tune_batch
 * ~ rp_tune_batch (RP_SORTED), search_multi ~ rp_search_multi (host
 * memory), graph_free ~ rp_graph_free.  rp_server_create supplies these for
 * a context; rp_server_create_ex takes any implementation, e.g. one on a
 * host without a GPU.  The callbacks run on the scheduler thread, one at a
 * time. */
typedef struct {
  void *user;
  rp_status (*tune_batch)(void *user, rp_graph src, const double *alphas, const int32_t *Rs,
                          int32_t T, rp_graph *outs);
  rp_status (*search_multi)(void *user, const rp_graph *graphs, int32_t ngraphs,
                            const int32_t *q_graph, const int32_t *q_L, const void *queries,
                            int64_t nq, int32_t k, int32_t *ids, float *dists);
  rp_status (*graph_free)(void *user, rp_graph g);
  /* Optional (NULL: the scheduler tunes with tune_batch and waits).  tune_start
   * begins what tune_batch does without waiting, returning a ticket; the
   * graphs in outs may be used once tune_ready(ticket) returns RP_OK
   * (RP_ETIMEOUT while the job runs, another code if it failed).  With both,
   * a non-serial server keeps searching resident graphs while a tuning job
   * runs (~ rp_tune_batch_async / rp_tune_wait). */
  rp_status (*tune_start)(void *user, rp_graph src, const double *alphas, const int32_t *Rs,
                          int32_t T, rp_graph *outs, int64_t *ticket);
  rp_status (*tune_ready)(void *user, int64_t ticket, int32_t timeout_ms);
} rp_executor;

typedef struct {
  rp_graph base;               /* the graph every target is tuned from */
  int32_t d;                   /* vector dimension */
  int32_t dtype;               /* RP_U8 or RP_F32 */
  uint64_t graph_bytes;        /* device bytes of one tuned graph (the budget's unit) */
  uint64_t graph_budget_bytes; /* bytes for resident tuned graphs; 0 = unlimited */
  int64_t max_batch_queries;   /* queries admitted per round; 0 = 65536 */
  int32_t serial;              /* 1 = plain serial path */
} rp_server_config;

/* rp_server_create: a server over base graph `base` of ctx.  The ctx must
 * outlive the server; other calls on the ctx may run meanwhile (calls are
 * serialised by the ctx).  Errors: RP_EINVAL, RP_ENOTFOUND. */
rp_status rp_server_create(rp_ctx *ctx, rp_graph base, uint64_t graph_budget_bytes,
                           int64_t max_batch_queries, int32_t serial, rp_server **out);

/* rp_server_create_ex: a server over an executor; *ex is copied.
 * Errors: RP_EINVAL (missing callback, d < 1, bad dtype). */
rp_status rp_server_create_ex(const rp_executor *ex, const rp_server_config *cfg, rp_server **out);

/* rp_server_destroy: finish every submitted request, stop the scheduler and
 * free the tuned graphs it holds (the base stays). */
rp_status rp_server_destroy(rp_server *srv);

/* rp_submit_tune: ask for the graph tuned to (alpha, R) to be resident.
 * alpha >= 1 on the 0.001 grid, R >= 1 (RP_R_INF = no limit).  Returns at
 * once with *request_id.  Errors: RP_EINVAL. */
rp_status rp_submit_tune(rp_server *srv, double alpha, int32_t R, int64_t *request_id);

/* rp_submit_search: queue GreedySearch of nq host query rows (packed, d
 * elements of the base's dtype each; copied before the call returns) on the
 * graph tuned to (alpha, R), tuning it first if it is not resident; alpha = 0
 * searches the base itself.  The list size used is max(L, k) (a request with
 * L < k is raised to k and counted as a clamp).  ids (int32[nq * k]) and
 * dists (float[nq * k] or NULL) are host buffers that must stay valid until
 * rp_poll reports the request finished; they receive rp_search's outputs.
 * Errors: RP_EINVAL (nq < 1, k < 1, L or k above RP_MAX_L, bad alpha or R,
 * null pointer). */
rp_status rp_submit_search(rp_server *srv, double alpha, int32_t R, const void *queries,
                           int64_t nq, int32_t L, int32_t k, int32_t *ids, float *dists,
                           int64_t *request_id);

enum { RP_REQ_QUEUED = 0, RP_REQ_RUNNING = 1, RP_REQ_DONE = 2 };

typedef struct {
  int32_t state;      /* RP_REQ_* */
  rp_status status;   /* outcome of a finished request (RP_OK or the failing call's code) */
  rp_graph graph;     /* the tuned graph that served it (0 if it failed) */
  int32_t L_eff;      /* list size used by a search */
  int32_t round;      /* scheduling round that ran it (1-based) */
  int64_t submit_ns;  /* steady-clock times since the server started */
  int64_t start_ns;
  int64_t done_ns;
} rp_request_info;

/* rp_poll: wait up to timeout_ms (0 = do not wait) for a request.  Returns
 * RP_OK with *info filled once it has finished (and forgets it: a second poll
 * of the same id returns RP_ENOTFOUND), RP_ETIMEOUT if it has not finished in
 * time (*info filled with its state), RP_ENOTFOUND for an unknown id,
 * RP_EINVAL for timeout_ms < 0. */
rp_status rp_poll(rp_server *srv, int64_t request_id, int32_t timeout_ms, rp_request_info *info);

typedef struct {
  int64_t requests_done;
  int64_t requests_failed;
  int64_t queries_done;
  int64_t rounds;
  int64_t tune_launches;     /* tune_batch calls */
  int64_t targets_tuned;
  int64_t search_launches;   /* search_multi calls */
  int64_t evictions;
  int64_t l_clamps;          /* searches submitted with L < k */
  int64_t resident_graphs;   /* tuned graphs held now */
  int64_t peak_resident_graphs;
  int64_t busy_ns;           /* time the scheduler spent running rounds */
} rp_server_stats_t;

rp_status rp_server_stats(rp_server *srv, rp_server_stats_t *out);

/* Message of the last failed request or call on the server (owned by it). */
const char *rp_server_last_error(rp_server *srv);

#ifdef __cplusplus
}
#endif

#endif /* RP_H_ */
