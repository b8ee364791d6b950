/*
 * lagr.h -- C ABI of the GB300 masked-semiring graph library.
 *
 * The library computes the data-parallel products under LAGraph's algorithms
 * (Mattson et al., 2021) on one GPU:
 *   - triangle counting, C<s(L)> = L plus.pair U' followed by a reduction
 *     (Alg. 6, Sec. IV-E), fused so that C is never materialised;
 *   - direction-optimizing parents BFS, push q'A / pull A'q over any.secondi
 *     with the visited set as a complemented structural mask (Alg. 1 and 2,
 *     Sec. IV-A);
 *   - PageRank, repeated A' plus.second w (Alg. 4, Sec. IV-C), a weighted
 *     plus.times form and its adjoint;
 *   - batched forms: 64 BFS sources in one bitmap frontier (the ns x n
 *     frontier of Alg. 3, Sec. IV-B) and many graphs in one launch.
 *
 * Conventions (Sec. II-C, II-D):
 *   - arguments are ordered outputs, then input/outputs, then inputs, then
 *     `msg`;
 *   - the return value is 0 on success, < 0 on error, > 0 for a warning;
 *   - `msg` is a caller-owned buffer of LAGR_MSG_LEN chars (or NULL).  It is
 *     set to "" on success and holds a description on an error or warning;
 *   - an output that is not wanted may be passed as NULL.
 *
 * Memory: every array argument documented "device" is a device pointer that
 * the caller allocates and keeps alive for the duration of the call (and, for
 * the graph's primary arrays, for the life of the graph).  Work space and
 * cached graph properties are allocated by the library through the allocator
 * set with lagr_set_allocator (stream-ordered cudaMallocAsync by default).
 *
 * Streams: every call takes a CUDA stream as `void *stream` (a cudaStream_t;
 * NULL means the legacy default stream) and issues all its device work on
 * it.  Calls that return a host scalar (lagr_tc's count, lagr_pagerank's
 * iteration count, lagr_bfs's depth) synchronise that stream before they
 * return; the others return once the work is enqueued, except where noted.
 *
 * Index types: int32 vertex ids and row pointers, so n < 2^31 and
 * nnz < 2^31 (larger inputs are rejected with LAGR_ERR_TOO_LARGE).
 */
#ifndef LAGR_H
#define LAGR_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define LAGR_MSG_LEN 256

/* return codes (Sec. II-D: 0 ok, < 0 error, > 0 warning) */
#define LAGR_OK 0
#define LAGR_ERR_NULL_POINTER (-1)
#define LAGR_ERR_INVALID_VALUE (-2)
#define LAGR_ERR_INVALID_GRAPH (-3)
#define LAGR_ERR_PROPERTY_MISSING (-4)
#define LAGR_ERR_OUT_OF_MEMORY (-5)
#define LAGR_ERR_CUDA (-6)
#define LAGR_ERR_TIMEOUT (-7)
#define LAGR_ERR_DEVICE_CHECK (-8)
#define LAGR_ERR_TOO_LARGE (-9)
#define LAGR_WARN_NOT_CONVERGED 1

/* graph kinds (Sec. II-A) */
#define LAGR_UNDIRECTED 0
#define LAGR_DIRECTED 1

/* lagr_tc methods: the degree-sort decision of Alg. 6 */
#define LAGR_TC_AUTO 0   /* sort when mean degree > 4 x median degree, as Alg. 6 */
#define LAGR_TC_SORT 1   /* always orient by ascending degree */
#define LAGR_TC_NOSORT 2 /* never: L = tril(A,-1), U = triu(A,1) on the given labels */

/* lagr_bfs flags */
#define LAGR_BFS_PUSH_ONLY 1 /* Alg. 1: every level is a push q'A */
#define LAGR_BFS_PULL_ONLY 2 /* every level after the first is a pull A'q */

/* lagr_pagerank / lagr_pagerank_backward flags */
#define LAGR_PR_GAP 0            /* Alg. 4 as written: dangling rows lose their mass */
#define LAGR_PR_DANGLING 1       /* redistribute the dangling mass through the teleport vector */
#define LAGR_PR_WEIGHTED 2       /* plus.times with the graph's values (row-stochastic W) */
#define LAGR_PR_WARM_START 4     /* `rank` holds the starting vector on entry */

/*
 * The graph (Sec. II-A): primary components plus cached properties.  The
 * struct is not opaque; a field that is not known is NULL (or -1 for the
 * scalars).  The primary arrays are BORROWED device pointers: the caller
 * keeps ownership and must keep them alive and unchanged while the graph
 * exists (if they change, call lagr_delete_properties).  Cached properties
 * are owned by the library and freed by lagr_delete_properties /
 * lagr_graph_free.
 */
typedef struct lagr_graph_struct {
  /* primary components */
  int32_t n;             /* number of vertices */
  int64_t nnz;           /* number of stored entries of A */
  int32_t kind;          /* LAGR_UNDIRECTED (A symmetric) or LAGR_DIRECTED */
  const int32_t *rowptr; /* device [n+1], rowptr[0] = 0, nondecreasing, rowptr[n] = nnz */
  const int32_t *colidx; /* device [nnz], each row strictly increasing, 0 <= j < n */
  const float *val;      /* device [nnz] or NULL: edge values (used by LAGR_PR_WEIGHTED) */

  /* cached: A' held by row (the CSC of A).  For an undirected graph these
   * alias the primary arrays. */
  int32_t *at_rowptr, *at_colidx;
  float *at_val;
  int32_t at_owned;

  /* cached: degrees (row degree of A; the column degree is that of A') */
  int32_t *row_degree;

  /* cached: triangle-counting orientation U (strict upper part after the
   * optional degree ordering of Alg. 6), held in the row slots of A: row v
   * (original label) is u_colidx[rowptr[v] .. rowptr[v] + u_dplus[v]), the
   * ranks of v's neighbours that rank above v in the order of A(v,:), a rank
   * being the position in the stable ascending-degree order (or the label
   * itself when Alg. 6 does not sort).  u_dplus: device [n+1] (d+ per vertex);
   * u_colidx: device [nnz] (slots past a row's d+ are unused).  u_order is the
   * LAGR_TC_* method it was built for. */
  int32_t *u_dplus, *u_colidx;
  int32_t u_order;

  /* cached scalars */
  int32_t a_pattern_is_symmetric; /* -1 unknown, 0 no, 1 yes */
  int64_t ndiag;                  /* number of self-loops, -1 unknown */

  /* statistics of the last call on this graph */
  int32_t last_levels;      /* BFS: number of levels (depth) */
  int32_t last_push_levels; /* BFS: levels done as push */
  int32_t last_pull_levels; /* BFS: levels done as pull */
  int32_t last_iters;       /* PageRank: iterations done */
  double last_resid;        /* PageRank: last L1 change */

  void *priv; /* library-private work space; do not touch */
} lagr_graph_struct;

typedef lagr_graph_struct *lagr_graph;

/*
 * Allocator hook (Sec. V, the malloc/free wrappers): every device
 * allocation of the library goes through alloc(bytes, stream, ctx) and
 * free_(ptr, stream, ctx).  alloc returns NULL on failure, which the calling
 * function reports as LAGR_ERR_OUT_OF_MEMORY.  Passing NULLs restores the
 * default: stream-ordered allocation (cudaMallocFromPoolAsync / cudaFreeAsync
 * on the call's stream) from a memory pool the library creates per device,
 * which keeps freed memory for later calls instead of returning it to the
 * driver at the next synchronisation.  Not thread-safe: set it before the
 * first call.
 */
typedef void *(*lagr_alloc_fn)(size_t bytes, void *stream, void *ctx);
typedef void (*lagr_free_fn)(void *ptr, void *stream, void *ctx);
int lagr_set_allocator(lagr_alloc_fn alloc, lagr_free_fn free_, void *ctx);

/*
 * Hand memory the default allocator keeps back to the driver (no paper
 * counterpart; the counterpart of LAGraph's finalize for the memory pools):
 * every per-device pool of the library is trimmed to at most keep_bytes of
 * free memory (cudaMemPoolTrimTo; memory of live graphs, or freed by work
 * still queued on a stream, stays), and the recycled pinned host scalars of
 * freed graphs are released.  Thread-safe.  Returns LAGR_ERR_CUDA (with the
 * device in msg) if a trim fails.
 */
int lagr_release_memory(uint64_t keep_bytes, char *msg);

/*
 * Create a graph from a device CSR (the "move" constructor of Sec. II-A,
 * except that the arrays are borrowed, not moved: PyTorch or the caller owns
 * device memory).  Host-only: no device work, no validation beyond sizes
 * (see lagr_graph_check).  *G receives a new host struct.
 * Errors: NULL_POINTER (G, or rowptr/colidx with n > 0 / nnz > 0),
 * INVALID_VALUE (n < 0, nnz < 0, bad kind), TOO_LARGE (n or nnz >= 2^31).
 */
int lagr_graph_new(lagr_graph *G, int32_t n, int64_t nnz, const int32_t *rowptr,
                   const int32_t *colidx, const float *val, int32_t kind, char *msg);

/* Free the struct and every cached property (LAGraph_Delete, Sec. II-A); *G
 * is set to NULL.  Frees are issued on `stream`.  A NULL *G is a no-op. */
int lagr_graph_free(lagr_graph *G, void *stream, char *msg);

/* Drop every cached property (Sec. V, DeleteProperties). */
int lagr_delete_properties(lagr_graph G, void *stream, char *msg);

/*
 * Validate the graph on the device (Sec. V, CheckGraph): rowptr[0] = 0,
 * rowptr nondecreasing, rowptr[n] = nnz, every column index in [0, n), each
 * row strictly increasing (sorted, no duplicates), and, for
 * LAGR_UNDIRECTED, A equal to A'.  Sets a_pattern_is_symmetric and ndiag.
 * Returns LAGR_ERR_INVALID_GRAPH with a description when a check fails.
 * Synchronises the stream.
 */
int lagr_graph_check(lagr_graph G, void *stream, char *msg);

/* Compute and cache A' by row (Sec. II-A, Property_AT).  Rows of A' are
 * sorted; for an undirected graph A' aliases A.  Deterministic. */
int lagr_property_AT(lagr_graph G, void *stream, char *msg);

/* Compute and cache the row degree (Sec. V, Property_RowDegree). */
int lagr_property_row_degree(lagr_graph G, void *stream, char *msg);

/*
 * Triangle count (Alg. 6, Sec. IV-E): the number of unique 3-cliques of the
 * undirected graph G, i.e. t = sum(C) with C<s(L)> = L plus.pair U', L and U
 * the strictly lower and upper parts of A after the degree ordering that
 * `method` selects (LAGR_TC_*).  Self-loops are ignored (strict parts).
 * The product C is never formed; the count is exact (uint64).
 * ntriangles: host, output.  Caches G->u_* (the orientation).  Synchronises
 * the stream.  Errors: NULL_POINTER, INVALID_VALUE (bad method),
 * INVALID_GRAPH (G directed), OUT_OF_MEMORY, CUDA.
 */
int lagr_tc(uint64_t *ntriangles, lagr_graph G, int32_t method, void *stream, char *msg);

/*
 * Triangle count with C kept: the unfused form of Alg. 6 (Sec. IV-E), C<s(L)> = L plus.pair U'
 * after the degree ordering that `method` selects (LAGR_TC_*).  c[e] for every stored entry
 * e = (i,j) of A (CSR order, the caller's labels) is C at that entry -- the number of vertices k
 * adjacent to both i and j that lie strictly between them in the degree order -- when the entry is
 * in L (i after j in that order), and 0 when it is in U; every triangle is counted at one entry
 * (the one joining its first and last vertex in the order), so the sum of c is the triangle count.
 * c: device [nnz] output (uint32; may be NULL when nnz = 0).  ntriangles: host output (the sum of
 * c) or NULL.  Caches the
 * orientation G->u_* like lagr_tc.  Synchronises the stream.  Errors: NULL_POINTER, INVALID_VALUE
 * (bad method), INVALID_GRAPH (G directed), OUT_OF_MEMORY, CUDA.
 */
int lagr_tc_edges(uint32_t *c, uint64_t *ntriangles, lagr_graph G, int32_t method, void *stream, char *msg);

/*
 * Parents BFS (Alg. 1 / Alg. 2, Sec. IV-A).  level[v] = number of edges on a
 * shortest path from src to v (-1 when unreachable); parent[v] = some u with
 * A(u,v) stored and level[u] = level[v] - 1 (the `any` monoid: which one is
 * unspecified), parent[src] = src, -1 when unreachable.  Direction
 * optimisation switches between push (rows of A) and pull (rows of A') per
 * level; flags may force one direction.  Directed graphs follow out-edges;
 * the pull needs A' (computed and cached when missing).
 * level, parent: device [n] outputs, either may be NULL.  depth: host output
 * (number of levels, >= 1) or NULL.  Synchronises the stream.
 * Errors: NULL_POINTER, INVALID_VALUE (src out of range, bad flags),
 * OUT_OF_MEMORY, TIMEOUT (a capped device wait ran out), CUDA.
 */
int lagr_bfs(int32_t *level, int32_t *parent, int32_t *depth, lagr_graph G, int32_t src,
             int32_t flags, void *stream, char *msg);

/*
 * Independent parents BFS from k sources (k <= LAGR_BFS_MULTI_MAX), each the
 * traversal of lagr_bfs (Alg. 1 / 2, Sec. IV-A) with the same flags: row t of
 * level / parent (device [k][n], row-major; either may be NULL) holds source
 * src[t]'s result, depth (host [k] or NULL) its level count.  The traversals
 * run interleaved on the library's side streams (they start after the work
 * queued on `stream`, which waits for them before the call returns), so one
 * host synchronisation per round serves all of them and their narrow levels
 * run side by side.  Duplicate sources are allowed.  G's last_* statistics are
 * those of src[k-1].  src: host [k].  Synchronises the stream.  Errors:
 * NULL_POINTER, INVALID_VALUE (k, a source out of range, bad flags),
 * OUT_OF_MEMORY, TIMEOUT, CUDA.
 */
#define LAGR_BFS_MULTI_MAX 64
int lagr_bfs_multi(int32_t *level, int32_t *parent, int32_t *depth, lagr_graph G, const int32_t *src, int32_t k,
                   int32_t flags, void *stream, char *msg);

/*
 * lagr_bfs_noalloc: the parents BFS of lagr_bfs for callers that cannot allocate device memory
 * (the paper has no counterpart; it exists for users whose device memory is fixed up front by
 * another owner, or who must not enter the allocator while other work runs).  It takes the
 * undirected graph as raw device CSR arrays (no lagr_graph, whose cached properties allocate) and
 * allocates nothing: all work space lives in one file-scope device array of the library, sized for
 * at most LAGR_BFS_NOALLOC_MAX_N vertices (about 17 MB).  A GPU reserves that array when the
 * library's BFS device code is first loaded on it (with CUDA's lazy module loading, at the first
 * BFS call on that device) and keeps it until the process exits; the first call on each device also
 * looks the array's address up.  Make one warm-up call per device at start-up, before any stream
 * capture and before the device memory is handed out.  Calls share the array: a call resets what
 * it uses, and calls whose GPU work overlaps race, so the caller must not run two at once on one
 * device.  The CSR must be a valid undirected graph (symmetric, every column index in [0, n), as
 * lagr_graph_check verifies): nothing here checks it, and an index out of range writes outside the
 * array.
 * level, parent: device [n] outputs, either may be NULL; depth: host output or NULL; results as
 * lagr_bfs.  Synchronises the stream.  Errors: INVALID_VALUE (n < 1, src out of range),
 * TOO_LARGE (n > LAGR_BFS_NOALLOC_MAX_N or nnz >= 2^31), NULL_POINTER, TIMEOUT, CUDA.
 */
#define LAGR_BFS_NOALLOC_MAX_N (1 << 21)
int lagr_bfs_noalloc(int32_t *level, int32_t *parent, int32_t *depth, int32_t n, int64_t nnz,
                     const int32_t *rowptr, const int32_t *colidx, int32_t src, void *stream,
                     char *msg);

/*
 * k BFS at once (1 <= k <= 64) from the sources src[0..k-1] (host array),
 * as one 64-bit bitmap frontier per vertex: the frontier matrix of Alg. 3
 * (Sec. IV-B) with ns = k and the any/or monoid in place of plus.
 * level: device [k][n] output, row s holds the levels from src[s] with the
 * same meaning as lagr_bfs.  Undirected graphs only.  Synchronises the
 * stream.  Errors: NULL_POINTER, INVALID_VALUE (k out of range or a source
 * out of range), INVALID_GRAPH (directed), OUT_OF_MEMORY, CUDA.
 */
int lagr_bfs_batch64(int32_t *level, lagr_graph G, const int32_t *src, int32_t k, void *stream,
                     char *msg);

/*
 * Batched betweenness centrality (Alg. 3, Sec. IV-B) in float64 from ns <= 64 sources at once:
 * centrality[j] = sum over the sources s_k of sum over targets t != s_k, j of
 * sigma(s_k, t | j) / sigma(s_k, t), sigma counting shortest paths (following out-edges on a
 * directed graph).  This is Alg. 3's -ns + sum_k B(k, j), with the path counts P and the backtrack
 * values B and W in float64; the backtrack runs over every BFS level, from the deepest one to the
 * first.  A source listed twice counts twice.  src: host [ns], 1 <= ns <= 64.  centrality: device
 * [n] output (float64).  levels: host output (the number of BFS levels past the sources) or NULL.
 * Work space: 4 ns n float64 values plus the level lists.  Synchronises the stream once per BFS
 * level.  Errors: NULL_POINTER, INVALID_VALUE (ns or a source out of range), OUT_OF_MEMORY,
 * TIMEOUT, CUDA.
 */
int lagr_betweenness(double *centrality, int32_t *levels, lagr_graph G, const int32_t *src, int32_t ns,
                     void *stream, char *msg);

/*
 * Single-source shortest paths by delta-stepping (Alg. 5, Sec. IV-D) over min.plus in float32.
 * dist[v] = the least fixed point of dist(v) = min over the entries A(u,v) of dist(u) + A(u,v)
 * with dist(src) = 0, every sum rounded to float32: the float32 length of a shortest path from src
 * (+inf when v is unreachable).  The edge values G->val are the weights; as in Alg. 5 the entries
 * with 0 < A <= delta are light and those with A > delta heavy, and entries with A <= 0 take no
 * part.  Directed graphs follow out-edges.  delta > 0 only sets the bucket width (the work, not
 * the result).  dist: device [n] output.  buckets: host output (buckets settled) or NULL.
 * Synchronises the stream once per relaxation step.  Errors: NULL_POINTER, INVALID_VALUE (no
 * values, src out of range, delta not positive and finite), OUT_OF_MEMORY, TIMEOUT, CUDA.
 */
int lagr_sssp(float *dist, int32_t *buckets, lagr_graph G, int32_t src, float delta, void *stream, char *msg);

/*
 * Connected components by FastSV (Alg. 7, Sec. IV-F): component[u] = the smallest vertex id of
 * u's connected component, the root every vertex of the component points to once the forest of
 * Alg. 7 stops changing.  Rounds of stochastic hooking, aggressive hooking, shortcutting and
 * grandparent updates (steps 1-4) run until a round changes neither the parents nor the
 * grandparents.  Undirected graphs only.  component: device [n] output.  rounds: host output or
 * NULL.  Synchronises the stream once per round.  Errors: NULL_POINTER, INVALID_GRAPH (directed),
 * OUT_OF_MEMORY, TIMEOUT (no fixed point within 2 log2(n) + 64 rounds), CUDA.
 */
int lagr_connected_components(int32_t *component, int32_t *rounds, lagr_graph G, void *stream, char *msg);

/*
 * PageRank (Alg. 4, Sec. IV-C) in float32.
 * Unweighted (flags without LAGR_PR_WEIGHTED):
 *   r = 1/n; repeat: t = r; w = damping * t / d_out (rows with d_out > 0);
 *   r = (1 - damping) * v + A' plus.second w [+ damping * (sum of t over
 *   dangling rows) * v when LAGR_PR_DANGLING]; stop when sum|t - r| < tol.
 * Weighted (LAGR_PR_WEIGHTED; G->val holds a row-stochastic W):
 *   r = (1 - damping) v + damping W' r [+ dangling term as above].
 * v is `teleport` (device [n], a distribution) or uniform 1/n when NULL.
 * rank: device [n] output (input too with LAGR_PR_WARM_START).  iters: host
 * output or NULL.  Returns LAGR_WARN_NOT_CONVERGED when itermax iterations
 * did not reach tol (rank holds the last iterate).  Synchronises the stream.
 * Errors: NULL_POINTER, INVALID_VALUE (damping outside (0,1), itermax < 1,
 * tol < 0, WEIGHTED without values), OUT_OF_MEMORY, CUDA.
 */
int lagr_pagerank(float *rank, int32_t *iters, lagr_graph G, float damping, float tol,
                  int32_t itermax, const float *teleport, int32_t flags, void *stream, char *msg);

/*
 * Adjoint of the weighted PageRank fixed point of Alg. 4 (Sec. IV-C, with
 * plus.times of Table II; the paper has no adjoint:
 * this is the implicit-function derivative of the iteration above).  For a
 * loss L with dL/drank = g, solve
 *   lambda = g + damping W lambda [+ damping (v . lambda) 1_dangling]
 * by the same gather machinery on the rows of W, then
 *   dL/dW(i,j) = damping * rank(i) * lambda(j)      (every stored (i,j))
 *   dL/dv(j)   = ((1 - damping) + damping * delta) * lambda(j),
 * delta = sum of rank over dangling rows under LAGR_PR_DANGLING, else 0.
 * rank: device [n], the forward fixed point, or NULL to recompute it here
 * (nothing is stored per iteration either way).  dL_dw: device [nnz] output
 * in CSR order, or NULL.  dL_dteleport: device [n] output or NULL.
 * iters: host output (adjoint iterations) or NULL.  Uses G->val (W);
 * flags must include LAGR_PR_WEIGHTED.  The adjoint iteration stops when its
 * L1 change is below tol times the L1 norm of the new iterate (relative: the
 * scale of lambda is that of dL/drank); `tol` and `itermax` of the forward
 * recompute (rank == NULL) keep the absolute criterion of Alg. 4.  Returns
 * LAGR_WARN_NOT_CONVERGED when itermax adjoint iterations did not reach tol.
 * Synchronises the stream.
 */
int lagr_pagerank_backward(float *dL_dw, float *dL_dteleport, int32_t *iters,
                           const float *dL_drank, const float *rank, lagr_graph G, float damping,
                           float tol, int32_t itermax, const float *teleport, int32_t flags,
                           void *stream, char *msg);

/*
 * Many graphs at once: the triangle count of Alg. 6 and the PageRank of
 * Alg. 4 for each of g graphs in one launch, against the per-call overhead
 * the paper measures on high-diameter inputs (Sec. VI-B).  A batch is g
 * undirected graphs concatenated block-diagonally into one CSR (vertex ids
 * shifted by voff).  A plan holds
 * the orientation, the work partition and a CUDA graph of the whole pass
 * (triangle count of every member, then `iters` PageRank iterations, GAP
 * form, of every member, the teleport of member i being (1-damping)/n_i);
 * lagr_batch_run replays it as one graph launch.
 * lagr_batch_plan: voff is a HOST array [g+1]; rowptr/colidx device arrays of
 * the concatenated CSR, borrowed for the plan's life.  tile: rows per work
 * item of the triangle kernel (0 = autotune; the choice is cached in
 * tune_cache, a JSON file path, when not NULL).
 * lagr_batch_run: ntri device [g] (uint64), rank device [N] (float).
 */
typedef struct lagr_batch_struct *lagr_batch;
int lagr_batch_plan(lagr_batch *B, int32_t g, const int32_t *voff, int32_t N, int64_t nnz,
                    const int32_t *rowptr, const int32_t *colidx, float damping, int32_t iters,
                    int32_t tile, const char *tune_cache, void *stream, char *msg);
int lagr_batch_run(uint64_t *ntri, float *rank, lagr_batch B, void *stream, char *msg);
int lagr_batch_tile(int32_t *tile, lagr_batch B);
int lagr_batch_free(lagr_batch *B, void *stream, char *msg);

/* Diagnostics (no paper counterpart): force the capacities of the triangle count's anchor lists
 * (CTA items, chunked warp items) for later lagr_tc calls on graphs whose orientation is rebuilt;
 * 0 restores the capacities computed from the graph.  A list that overflows its capacity is never
 * written or read past its end: lagr_tc returns LAGR_ERR_INVALID_GRAPH instead.  For tests of that
 * bound.  Returns LAGR_ERR_INVALID_VALUE for a negative capacity.  Not thread-safe with running
 * lagr_tc calls. */
int lagr_debug_tc_capacity(int64_t capc, int64_t capwh);

/* library version string (no paper counterpart; LAGraph's version query) */
const char *lagr_version(void);

/* Diagnostics: the number of CUDA kernels this library has launched since it was loaded (kernels
 * replayed from a captured CUDA graph are counted once, when captured).  No paper counterpart. */
uint64_t lagr_kernel_launches(void);

/* Diagnostics: per-kernel device time of the hot kernels (no paper counterpart).
 * lagr_timing_enable(1) makes every later launch of a timed kernel record a pair of CUDA events
 * on its launching stream around the launch (not inside CUDA-graph capture); 0 stops it.
 * lagr_timing_read(name, &ms, &launches) waits for the recorded events of kernel `name`, adds
 * their durations to the running totals and returns the totals since the last lagr_timing_reset().
 * Timed names: "pr_gather" (one PageRank / adjoint iteration's row-block gather), "tc_count_cta",
 * "tc_count_warp" (the masked-product count kernels), "bfs_push_small", "bfs_push_lb", "bfs_pull".
 * Returns LAGR_ERR_INVALID_VALUE for an unknown name, LAGR_ERR_CUDA if an event failed; the
 * facility is process-wide and thread-safe, and events hold no device memory of the caller. */
int lagr_timing_enable(int on);
int lagr_timing_read(const char *kernel, double *ms, int64_t *launches);
int lagr_timing_reset(void);

#ifdef __cplusplus
}
#endif

#endif /* LAGR_H */
