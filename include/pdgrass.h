/*
 * pdgrass.h -- C ABI of the GB300 off-tree edge-recovery library.
 *
 * The library computes the off-tree edge-recovery step of pdGRASS
 * (parallel density-aware graph spectral sparsification): given a weighted
 * undirected graph G = (V, E, w) and a spanning tree T of G, it returns the
 * first alpha*|V| off-tree edges recovered by the strict-similarity greedy
 * (Sec. 2.1 problem statement; Sec. 2.2 budget; Algorithm 1).
 *
 * Per off-tree edge e = (u, v) the library computes
 *   l      = LCA_T(u, v)                                  (Algorithm 1, step 1)
 *   R_T(e) = sum of 1/w over the tree path u -> l -> v    (Eq. RT), summed
 *            exactly and rounded once to nearest-even FP64
 *   score  = fl(w_e * R_T(e))  (STRETCH, default) or R_T(e) (RESISTANCE)
 *   beta*  = min(hops(u, l), hops(v, l), c)               (Eq. beta-new)
 * orders the edges by (score descending, edge id ascending) (Algorithm 1,
 * step 2), groups them into subtasks by LCA (step 3; Lemma "share LCA"), and
 * inside every subtask recovers an edge unless an earlier recovered edge e'
 * of the subtask has it strictly similar (Def. "Similar edge (Strict)" with
 * the beta*-hop neighbourhoods of e' in T).  The result equals the sequential
 * greedy over the global order stopped after k = floor(alpha*|V|) edges.
 *
 * Everything runs on one CUDA device.  All entry points are synchronous with
 * respect to the host unless stated otherwise; device work is issued on the
 * stream given at init.  Handles are not thread-safe: use one handle per host
 * thread (several handles may share a device and run concurrently).
 */
#ifndef PDGRASS_H_
#define PDGRASS_H_

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ------------------------------------------------------------------ status */
#define PDG_OK 0
#define PDG_UNDER_BUDGET 1      /* fewer than k edges survive one pass; all of them are returned */
#define PDG_E_INVALID_ARG (-1)  /* NULL pointer, bad size, bad alpha/c/mem kind */
#define PDG_E_NOT_SYMMETRIC (-2)/* CSR is not symmetric with equal weights both ways */
#define PDG_E_NOT_A_TREE (-3)   /* parent[] is not a spanning tree made of edges of G */
#define PDG_E_BAD_WEIGHT (-4)   /* weight not finite, not > 0, or outside [2^-900, 2^900] */
#define PDG_E_RANGE (-5)        /* the exact fixed-point root distances would overflow 96 bits */
#define PDG_E_CAPACITY (-6)     /* out_capacity smaller than the number of edges to return */
#define PDG_E_OOM (-7)          /* device allocation failed */
#define PDG_E_CUDA (-8)         /* a CUDA runtime call failed */
#define PDG_E_TIMEOUT (-9)      /* a bounded device wait ran out (status word set by a kernel) */
#define PDG_E_NOT_CSR (-10)     /* row_ptr not monotone, column out of range, self loop,
                                   unsorted or duplicate neighbours */

/* ------------------------------------------------------------ memory kinds */
#define PDG_MEM_HOST 0   /* pointer is host memory (pageable or pinned) */
#define PDG_MEM_DEVICE 1 /* pointer is device memory of the handle's device */

/* ------------------------------------------------------------- score modes */
#define PDG_SCORE_STRETCH 0    /* score = fl(w * R_T): spectral criticality (default) */
#define PDG_SCORE_RESISTANCE 1 /* score = R_T (Algorithm 1 sorts by "resistance") */

#define PDG_MAX_C 3 /* largest supported beta cap c */

typedef struct pdg_options {
  int32_t score_mode;       /* PDG_SCORE_STRETCH or PDG_SCORE_RESISTANCE */
  int32_t warp_tier_max;    /* subtasks with 2..warp_tier_max candidates get one warp each (<= 32) */
  int64_t k_override;       /* >= 0: use this budget instead of floor(alpha*|V|) */
  double candidate_factor;  /* first candidate prefix holds about factor*k edges (>= 1) */
  int32_t max_rounds;       /* rounds of the cooperative (hash) tier before the serial finisher */
  int32_t use_graph;        /* 1: capture the recovery pipeline in a CUDA graph and replay it */
  int64_t spin_limit;       /* iteration bound of every device-side wait */
  int32_t profile;          /* 1: time every step with CUDA events (see pdg_last_timings) */
  int32_t block_tier_max;   /* subtasks with warp_tier_max+1..block_tier_max candidates get one block each
                               (shared-memory marker table); 0 turns the block tier off; at most 896 */
  int32_t sort_tile_keys;   /* keys per tile of the radix-sort scatter: 2048, 3072 or 4096 (0: 3072) */
  int32_t sort_one_launch;  /* 1 (default): the ordering step runs as one cooperative launch whenever every
                               tile of the candidates fits in one resident block; 0: one kernel per pass */
} pdg_options;

typedef struct pdg_sparsifier* pdg_handle; /* opaque, owned by the library */

/* Fill *opt with the defaults (STRETCH, warp tier 32, factor 1.5, ...). */
void pdg_default_options(pdg_options* opt);

/* Human-readable text of a status code (static storage). */
const char* pdg_status_string(int status);

/*
 * sparsify_init -- upload and validate one graph and its spanning tree.
 *
 *   n        number of vertices, 1 <= n < 2^30.
 *   row_ptr  int64[n+1], CSR row offsets; row_ptr[0] = 0, non-decreasing.
 *   col      int32[row_ptr[n]], neighbours of each row, strictly increasing
 *            within a row, no self loops; the CSR must be symmetric.
 *   w        float64[row_ptr[n]], w[(u,v)] == w[(v,u)] bit for bit, finite,
 *            in [2^-900, 2^900].
 *   parent   int32[n], parent[root] = -1 for exactly one root, otherwise the
 *            tree parent; every (v, parent[v]) must be an edge of G and the
 *            parent links must be acyclic (T spans G).
 *   mem_kind PDG_MEM_HOST or PDG_MEM_DEVICE for all four input arrays.
 *   opt      NULL for defaults.
 *   stream   cudaStream_t on which all device work of the handle runs
 *            (NULL = the legacy default stream).
 *
 * The library copies the inputs into device memory it owns; the caller may
 * free its buffers when this returns.  On success *out receives a handle to
 * release with sparsifier_free.  On failure *out is NULL and a negative
 * status is returned (PDG_E_NOT_CSR, PDG_E_NOT_SYMMETRIC, PDG_E_NOT_A_TREE,
 * PDG_E_BAD_WEIGHT, PDG_E_RANGE, PDG_E_OOM, PDG_E_CUDA, PDG_E_INVALID_ARG).
 */
int sparsify_init(pdg_handle* out, int64_t n, const int64_t* row_ptr, const int32_t* col, const double* w,
                  const int32_t* parent, int mem_kind, const pdg_options* opt, void* stream);

/*
 * recover_offtree -- run the off-tree edge-recovery step (Algorithm 1).
 *
 *   alpha         recovery ratio; k = floor(alpha * n) in IEEE double
 *                 (ignored when opt.k_override >= 0).  alpha >= 0, finite.
 *   c             beta cap of Eq. beta-new, 0 <= c <= PDG_MAX_C.
 *   out_edge_ids  int32[out_capacity]: canonical undirected edge ids of the
 *                 recovered edges, in recovery order (score descending, id
 *                 ascending).  Canonical id of edge {u,v}, u < v = rank of
 *                 the CSR entry (u, v) among all entries with row < col, in
 *                 row-major order.
 *   out_capacity  capacity of out_edge_ids / out_scores; must be >= the
 *                 number of edges returned (min(k, survivors)), else
 *                 PDG_E_CAPACITY and nothing is written.
 *   out_count     host int64: number of ids written.
 *   out_scores    nullable float64[out_capacity]: the score of each id.
 *   out_mem_kind  memory kind of out_edge_ids and out_scores.
 *
 * Returns PDG_OK, PDG_UNDER_BUDGET (fewer than k edges survive; all
 * survivors are returned) or a negative error.  The call is deterministic:
 * the same inputs give the same ids on every run and device.
 */
int recover_offtree(pdg_handle h, double alpha, int32_t c, int32_t* out_edge_ids, int64_t out_capacity,
                    int64_t* out_count, double* out_scores, int out_mem_kind);

/* Release a handle and all its device memory.  NULL-safe. */
void sparsifier_free(pdg_handle h);

/*
 * pdg_edge_endpoints -- map canonical edge ids of the handle's graph back to
 * their endpoints (u < v).  ids/u/v share mem_kind; count >= 0.
 */
int pdg_edge_endpoints(pdg_handle h, const int32_t* ids, int64_t count, int32_t* u, int32_t* v, int mem_kind);

/*
 * sparsify_batch_init -- upload a batch of independent graphs packed into one
 * CSR (a disjoint union).  Graph g owns vertices [vtx_ptr[g], vtx_ptr[g+1]),
 * its rows are contiguous, its neighbours and its parent entries are global
 * vertex ids inside its own range, and parent = -1 at each graph's root.
 *
 *   num_graphs  G >= 1.
 *   vtx_ptr     HOST int64[G+1], vtx_ptr[0] = 0, strictly increasing,
 *               vtx_ptr[G] = n < 2^30.
 *   other arrays as in sparsify_init over the packed n vertices.
 *
 * Validation is as in sparsify_init, plus: no edge may cross two graphs and
 * each graph's tree must span it.
 */
int sparsify_batch_init(pdg_handle* out, int32_t num_graphs, const int64_t* vtx_ptr, const int64_t* row_ptr,
                        const int32_t* col, const double* w, const int32_t* parent, int mem_kind,
                        const pdg_options* opt, void* stream);

/*
 * recover_offtree_batch -- recovery for every graph of a batch in one
 * pipeline (one pass of kernels over the packed CSR; replayed from a CUDA
 * graph when opt.use_graph is set).
 *
 *   alpha        HOST float64[G]: per-graph ratio, k_g = floor(alpha[g]*n_g).
 *   c            beta cap shared by the batch (0..PDG_MAX_C).
 *   out_ptr      HOST int64[G+1]: graph g writes its ids to
 *                out_edge_ids[out_ptr[g] .. out_ptr[g] + out_count[g]);
 *                out_ptr[g+1] - out_ptr[g] must be >= k_g.
 *   out_edge_ids int32[out_ptr[G]]: per-graph LOCAL canonical ids (the id
 *                the graph would have on its own), in recovery order.
 *   out_count    HOST int64[G].
 *   out_scores   nullable float64[out_ptr[G]].
 *   graph_status nullable HOST int32[G]: PDG_OK or PDG_UNDER_BUDGET per graph.
 *
 * Returns PDG_OK when every graph met its budget, PDG_UNDER_BUDGET when some
 * did not, or a negative error.  Each graph's result equals what
 * recover_offtree returns for that graph alone.
 */
int recover_offtree_batch(pdg_handle h, const double* alpha, int32_t c, const int64_t* out_ptr,
                          int32_t* out_edge_ids, int64_t* out_count, double* out_scores, int32_t* graph_status,
                          int out_mem_kind);

/*
 * pdg_handle_info -- sizes of the resident graph (any pointer may be NULL):
 * vertices, undirected edges, off-tree edges, number of graphs, maximum hop
 * depth of the tree(s), device bytes held by the handle.
 */
int pdg_handle_info(pdg_handle h, int64_t* n, int64_t* m, int64_t* n_offtree, int32_t* num_graphs,
                    int64_t* max_depth, int64_t* device_bytes);

/*
 * pdg_last_stats -- counters of the last recovery: candidates examined (the
 * prefix of the global order that was scored into subtasks), subtasks,
 * largest subtask, candidates in the warp tier / cooperative tier, rounds of
 * the cooperative tier, prefix retries, attempts, kernels launched by the
 * recovery, cooperative-tier candidates that showed an earlier registrant of
 * one of their pairs ("constrained"), ancestor pairs registered by the
 * cooperative tier, and the site of a failed internal index check (0 if none;
 * such a recovery returns PDG_E_CUDA).  stats must hold 12 int64.
 */
int pdg_last_stats(pdg_handle h, int64_t* stats);

/*
 * pdg_last_timings -- device time in milliseconds of each step of the last
 * recovery, measured with CUDA events on the handle's stream when
 * opt.profile = 1 (zeros otherwise): [0] classify (A1), [1] tree (A2),
 * [2] score (A3), [3] select (A4a), [4] sort (A4b), [5] accept (A5+A6),
 * [6] budget (A7), [7] whole recovery.  Steps 3-6 are summed over prefix
 * retries.  ms must hold 8 floats.
 */
int pdg_last_timings(pdg_handle h, float* ms);

/*
 * pdg_spanning_tree -- generate the spanning tree that recovery starts from
 * (Sec. 2.2: feGRASS's first step builds the tree from the effective weight,
 * Eq. weff; the plain maximum-weight tree is the other common choice).
 *
 *   n, row_ptr, col, w, mem_kind  the graph, as in sparsify_init (symmetric
 *                 CSR, sorted rows, no self loops, weights in [2^-900, 2^900]).
 *   tree_kind     PDG_TREE_MAX_WEIGHT: the maximum spanning forest for the
 *                 order (w descending, canonical edge id ascending);
 *                 PDG_TREE_FEGRASS: the maximum spanning tree for the order
 *                 (W_eff descending, id ascending) with
 *                 W_eff(e) = fl(fl(w * fl(log(max(deg u, deg v)))) / (d(u) + d(v))),
 *                 d = unweighted BFS distance from the maximum-degree vertex
 *                 (the graph must be connected).
 *   parent_out    int32[n]: the tree as a parent array, each component rooted
 *                 at its maximum-degree vertex (ties: smaller id), -1 there.
 *   out_mem_kind  memory kind of parent_out.
 *   stream        cudaStream_t for the device work.
 *
 * Both orders are strict, so the tree is unique and the call deterministic.
 * Device memory is allocated for the call and released before it returns.
 * Returns PDG_OK, PDG_E_INVALID_ARG (bad arguments, or PDG_TREE_FEGRASS on a
 * disconnected graph), PDG_E_NOT_CSR, PDG_E_NOT_SYMMETRIC, PDG_E_BAD_WEIGHT,
 * PDG_E_OOM or PDG_E_CUDA.
 */
#define PDG_TREE_MAX_WEIGHT 0
#define PDG_TREE_FEGRASS 1
int pdg_spanning_tree(int64_t n, const int64_t* row_ptr, const int32_t* col, const double* w, int mem_kind,
                      int tree_kind, int32_t* parent_out, int out_mem_kind, void* stream);

/*
 * pdg_pcg_quality -- measure a sparsifier the way Sec. 5 does: the number of
 * preconditioned conjugate-gradient iterations that solving L_G x = b takes
 * with the sparsifier's Laplacian L_P (the tree plus the given edges) as the
 * preconditioner, to ||r|| <= tol ||b'||.
 *
 *   n, row_ptr, col, w, parent  the graph and its spanning tree, as in
 *                 sparsify_init (one root: the graph is connected).
 *   edge_ids      int32[n_edges]: distinct canonical ids of off-tree edges
 *                 (e.g. a recovery's output), 0 <= n_edges <= 8192.
 *   b             float64[n]: right-hand side; b' = b - mean(b) is solved
 *                 (L_G is singular).
 *   tol, max_iter stopping rule (tol > 0; max_iter >= 1).
 *   mem_kind      memory kind of all array inputs.
 *   out_iters, out_relres  host: iterations run and the final ||r|| / ||b'||.
 *
 * x starts at 0; the preconditioner solves L_P z = r exactly (grounded at
 * the tree root, then centred): tree solves over the Euler tour plus a
 * k x k capacitance matrix for the k extra edges (Woodbury).  Device memory
 * is allocated for the call and released before it returns.  Returns PDG_OK
 * or PDG_E_INVALID_ARG (arguments, an edge id out of range, a tree edge or a
 * repeated id), the errors of sparsify_init, PDG_E_OOM or PDG_E_CUDA.
 */
int pdg_pcg_quality(int64_t n, const int64_t* row_ptr, const int32_t* col, const double* w, const int32_t* parent,
                    const int32_t* edge_ids, int64_t n_edges, const double* b, double tol, int32_t max_iter,
                    int mem_kind, int32_t* out_iters, double* out_relres, void* stream);

/*
 * pdg_pcg_trace -- pdg_pcg_quality with the run's intermediate results, so
 * that the iteration can be checked step by step (Sec. 5 measure).
 *
 *   out_history    host float64[max_iter]: entry i - 1 receives ||r_i|| / ||b'||
 *                  after iteration i, for i = 1 .. *out_iters.
 *   out_precond_b  host float64[n]: the preconditioner applied to b', i.e. the
 *                  solution z of L_P z = b' grounded at the tree root, then
 *                  centred (the first z of the iteration).
 *   every other argument and every status as in pdg_pcg_quality; both
 *   outputs must be non-NULL (else PDG_E_INVALID_ARG).
 */
int pdg_pcg_trace(int64_t n, const int64_t* row_ptr, const int32_t* col, const double* w, const int32_t* parent,
                  const int32_t* edge_ids, int64_t n_edges, const double* b, double tol, int32_t max_iter,
                  int mem_kind, int32_t* out_iters, double* out_relres, double* out_history, double* out_precond_b,
                  void* stream);

/*
 * pdg_edge_endpoints_noalloc -- the mapping of pdg_edge_endpoints for callers
 * that must not allocate device memory (for example code that may only use a
 * caller-owned memory pool, or a serving loop that must not stall on
 * cudaMalloc/cudaFree).  The paper has no counterpart: this is a service of
 * the library, not a step of the method.
 *
 *   n        vertices of the caller's graph, 1 <= n <= PDG_NOALLOC_MAX_N.
 *   row_ptr  DEVICE int64[n+1], col DEVICE int32[row_ptr[n]]: the symmetric
 *            CSR with sorted rows (as for sparsify_init; not re-validated).
 *   ids      DEVICE int32[count], canonical edge ids; u, v DEVICE
 *            int32[count] receive the endpoints (u < v), or -1 for an id out
 *            of range (then PDG_E_INVALID_ARG is returned).
 *   stream   cudaStream_t for the work; the call waits on the host until
 *            the stream has finished it (it synchronises that stream).
 *
 * No device memory is allocated: the only scratch is a fixed array of about
 * 16 MB inside the library (PDG_NOALLOC_MAX_N + 1 row prefixes plus scan
 * block sums), present on every device that loads the library until the
 * process exits.  Calls share that array, so calls that overlap on one
 * device race and must be serialised by the caller.  The first call on each
 * device looks the array's address up (cudaGetSymbolAddress) with that device
 * current; make that first call before any stream capture.
 * Returns PDG_OK, PDG_E_INVALID_ARG (bad size or id) or PDG_E_CUDA.
 */
#define PDG_NOALLOC_MAX_N (1 << 21)
int pdg_edge_endpoints_noalloc(int64_t n, const int64_t* row_ptr, const int32_t* col, const int32_t* ids,
                               int64_t count, int32_t* u, int32_t* v, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* PDGRASS_H_ */
