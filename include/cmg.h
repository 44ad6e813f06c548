/*
 * cmg.h -- C-ABI of the GB300 cascadic multigrid (CMG) Fiedler-vector library.
 *
 * Method: J. C. Urschel, X. Hu, J. Xu, L. T. Zikatanov, "A cascadic multigrid
 * algorithm for computing the Fiedler vector of graph Laplacians",
 * arXiv 1412.0565.  The library computes an approximation of the Fiedler
 * vector phi_2 and of the algebraic connectivity lambda_2 (Sec. 2,
 * Definition 2.2) of a weighted undirected graph by Alg. 1: heavy edge
 * coarsening (Alg. 2) with Galerkin coarse Laplacians L^{i+1} = I L I^T
 * (Sec. 2 Step 1), power iteration on the coarsest graph from a Gaussian
 * vector (Alg. 1 Step 2, Remark 2.3), then prolongation and power iteration
 * (Alg. 3) on every finer level (Alg. 1 Step 3).
 *
 * Conventions shared by every entry point
 *   - Graphs are CSR: row_ptr[n+1], col[nnz] (0-based), w[nnz].  The matrix is
 *     the weighted adjacency matrix W of the graph; the Laplacian is
 *     L = diag(W 1) - W (Definition 2.1).  The diagonal is never stored.
 *   - Input contract (checked when options.validate != 0): n >= 2;
 *     row_ptr[0] = 0, non-decreasing, row_ptr[n] = nnz < 2^31; every column
 *     in [0, n), strictly ascending within a row (no duplicates), no
 *     self-loop (Sec. 2: (i, i) is not an edge); every weight finite and > 0;
 *     W symmetric with bitwise equal mirrored weights; no isolated vertex.
 *     The graph is assumed connected (lambda_2 > 0); a disconnected graph is
 *     processed but its result is a vector of the zero eigenspace.
 *   - `mem` arguments say where a caller buffer lives: CMG_MEM_HOST or
 *     CMG_MEM_DEVICE (a device pointer of the current CUDA device).
 *   - `stream` is a cudaStream_t (NULL = the legacy default stream).  Work is
 *     stream-ordered; calls that return host values synchronise the stream.
 *   - Input buffers are borrowed for the duration of the call and copied;
 *     the library never keeps a caller pointer.  Output buffers are owned by
 *     the caller and must have the stated length.
 *   - Every call returns a cmg_status_t and never aborts the process.
 */
#ifndef CMG_H
#define CMG_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define CMG_MAX_LEVELS 64

typedef enum cmg_status {
    CMG_OK = 0,
    CMG_WARN_MAXITER = 1,          /* a sweep cap stopped some level; result still usable */
    CMG_ERR_INVALID_ARG = -1,      /* NULL pointer, bad enum, bad level index, ...        */
    CMG_ERR_NOT_SYMMETRIC = -2,    /* a (i,j,w) without an identical (j,i,w)              */
    CMG_ERR_SELF_LOOP = -3,
    CMG_ERR_BAD_WEIGHT = -4,       /* weight <= 0, NaN or infinite                        */
    CMG_ERR_ISOLATED_VERTEX = -5,
    CMG_ERR_TOO_SMALL = -6,        /* n < 2                                               */
    CMG_ERR_OOM = -7,              /* a device allocation failed                          */
    CMG_ERR_CUDA = -8,             /* a CUDA runtime call failed                          */
    CMG_ERR_DEVICE_TIMEOUT = -9,   /* a bounded device-side wait gave up                  */
    CMG_ERR_BAD_CSR = -10,         /* row_ptr not monotone, column out of range,
                                      columns not strictly ascending                      */
    CMG_ERR_TOO_LARGE = -11,       /* nnz >= 2^31 or a size beyond a stated limit         */
    CMG_ERR_TIMEOUT = -12          /* a host-side wait with a time limit gave up          */
} cmg_status_t;

enum { CMG_MEM_HOST = 0, CMG_MEM_DEVICE = 1 };
/* Sweep precision.  FP64: every power-iteration sweep in FP64.  FP32_SWEEP:
 * the sweeps of the levels that carry the bytes run in FP32 with FP32
 * accumulation -- in cmg_setup / cmg_fiedler the levels with at least 2^20
 * stored entries, in the batched form union level 0 -- and every other level keeps
 * FP64 sweeps (those levels are latency-bound and run the longest sweep
 * chains, along which FP32 rounding would accumulate); in both forms the
 * stop statistic, mean and norm are float-float sums (about 48 bits), and
 * the last level-0 sweep is recomputed in FP64 from the previous iterate.
 * cmg_level_precision reports each level's choice. */
enum { CMG_PRECISION_FP64 = 0, CMG_PRECISION_FP32_SWEEP = 1 };
enum { CMG_SCHEDULE_TOL = 0, CMG_SCHEDULE_FIXED = 1, CMG_SCHEDULE_REPLAY = 2 };

/* Solver options.  cmg_options_default() fills the paper's settings. */
typedef struct cmg_options {
    double tol;        /* Alg. 3 stopping rule: stop when cos(u^k, u^{k-1}) >= 1 - tol
                          (Sec. 2.2; Sec. 4 uses tol = 1e-8)                           */
    double beta;       /* schedule FIXED: k_j = ceil(k0 * beta^j) sweeps on level j
                          (Sec. 3, Theorem 3.10)                                        */
    uint64_t seed;     /* keys the visit order of Alg. 2 and the Gaussian start of
                          Alg. 1 Step 2                                                */
    int32_t coarse_size;          /* Alg. 1: coarsen while n_i > coarse_size (25)      */
    int32_t max_levels;           /* at most this many levels, 1..64 (64)              */
    int32_t precision;            /* CMG_PRECISION_FP64 or CMG_PRECISION_FP32_SWEEP     */
    int32_t schedule;             /* CMG_SCHEDULE_TOL / FIXED / REPLAY                  */
    int32_t k0;                   /* schedule FIXED: sweeps on level 0                 */
    int32_t max_sweeps;           /* sweep cap per level above the coarsest (20000)    */
    int32_t max_sweeps_coarsest;  /* sweep cap on the coarsest level (100000)          */
    int32_t validate;             /* 1: check the input contract in cmg_setup (1)      */
    int32_t timing;               /* 1: cmg_fiedler times each level's power-iteration
                                     launch with CUDA events (stats level_ms) (0)      */
    int32_t reserved;             /* must be 0                                         */
    int32_t replay_sweeps[CMG_MAX_LEVELS]; /* schedule REPLAY: exact sweeps on level j */
} cmg_options_t;

/* Per-solve report.  Level 0 is the input graph; level levels-1 the coarsest. */
typedef struct cmg_stats {
    double lambda2;    /* r = u^T L u for the returned unit vector u (Sec. 4)          */
    double residual;   /* ||(L - r I) u||_2, the error metric of Sec. 4, Table 2       */
    int32_t levels;    /* J + 1                                                        */
    int32_t status;    /* CMG_OK or CMG_WARN_MAXITER                                   */
    int64_t n[CMG_MAX_LEVELS];
    int64_t nnz[CMG_MAX_LEVELS];
    int32_t sweeps[CMG_MAX_LEVELS];      /* power-iteration sweeps k_j on level j      */
    double cos_final[CMG_MAX_LEVELS];    /* cos(u^k, u^{k-1}) at the last sweep        */
    double level_ms[CMG_MAX_LEVELS];     /* device time of level j's power-iteration
                                            launch (options.timing; else 0)            */
    double finalize_ms;                  /* device time of the final-vector launch     */
} cmg_stats_t;

typedef struct cmg_hierarchy_s *cmg_hierarchy_t;

/* Fills *opts with tol = 1e-8, coarse_size = 25, max_levels = 64, seed = 1412,
 * FP64, schedule TOL, beta = 4, k0 = 1, max_sweeps = 20000,
 * max_sweeps_coarsest = 100000, validate = 1.  Errors: INVALID_ARG if NULL. */
cmg_status_t cmg_options_default(cmg_options_t *opts);

/* Static description of a status code (never NULL). */
const char *cmg_status_string(cmg_status_t status);

/* Library version string, e.g. "cmg-gb300 1.0 sm_103a". */
const char *cmg_version(void);

/*
 * Setup phase, Alg. 1 Step 1 (Sec. 2.1): repeated heavy edge coarsening
 * (Alg. 2) and Galerkin products L^{i+1} = I_i^{i+1} L^i (I_i^{i+1})^T while
 * n_i > coarse_size; a level whose coarsening yields fewer than 2 aggregates
 * becomes the coarsest.  The resulting hierarchy stays resident in device
 * memory of the current device and is owned by the library until cmg_free.
 *   n, row_ptr (int64[n+1]), col (int32[nnz]), w (double[nnz]): the graph,
 *     in host or device memory according to `mem`.
 *   opts: NULL means cmg_options_default().
 *   out: receives the hierarchy handle (NULL on error).
 * Errors: INVALID_ARG, TOO_SMALL, TOO_LARGE, BAD_CSR, SELF_LOOP, BAD_WEIGHT,
 * NOT_SYMMETRIC, ISOLATED_VERTEX, OOM, CUDA, DEVICE_TIMEOUT.
 */
cmg_status_t cmg_setup(int64_t n, const int64_t *row_ptr, const int32_t *col, const double *w,
                       int32_t mem, const cmg_options_t *opts, void *stream,
                       cmg_hierarchy_t *out);

/*
 * Solve phase, Alg. 1 Steps 2-3: power iteration (Alg. 3) on the coarsest
 * level from the Gaussian vector of Remark 2.3, then for j = J-1 .. 0
 * prolongation y^(j) = (I_j^{j+1})^T y^(j+1), Gram-Schmidt against 1 (Sec. 2.2)
 * and power iteration on B_g = g I - L^j with g = max_i sum_j |l_ij|.
 *   u_out: double[n_0] in `u_mem` memory, or NULL; receives the unit vector,
 *     orthogonal to 1, scaled so that its largest-magnitude entry (lowest
 *     index on ties) is positive, in the caller's vertex order.
 *   lambda2_out (host, nullable): r = u^T L u.
 *   stats_out (host, nullable): per-level sizes, sweeps, cosines, residual.
 * Returns OK, WARN_MAXITER (a cap was hit; outputs are valid), or an error
 * (INVALID_ARG, OOM, CUDA, DEVICE_TIMEOUT).  Synchronises `stream`.
 */
cmg_status_t cmg_fiedler(cmg_hierarchy_t h, double *u_out, int32_t u_mem, double *lambda2_out,
                         cmg_stats_t *stats_out, void *stream);

/* Options of one solve on a resident hierarchy (cmg_fiedler_ex). */
typedef struct cmg_solve_options {
    uint64_t seed;        /* keys the Gaussian start of Alg. 1 Step 2 for this solve
                             (the hierarchy, whose visit orders the setup's seed keyed,
                             is reused as it is)                                      */
    const double *x0;     /* NULL: cascade from the coarsest level (Steps 2-3);
                             else the start vector of level x0_level, double[n of that
                             level] in that level's vertex order (level 0: the caller's
                             order); levels above it are not visited                  */
    int32_t x0_mem;       /* CMG_MEM_HOST or CMG_MEM_DEVICE (where x0 lives)           */
    int32_t x0_level;     /* 0 .. levels-1                                             */
    int32_t reserved[4];  /* must be 0                                                 */
} cmg_solve_options_t;

/* Fills *so for an ordinary solve of h: seed = the seed h was set up with
 * (options.seed), no start vector.  h may be NULL (seed 1412).
 * Errors: INVALID_ARG if so is NULL. */
cmg_status_t cmg_solve_options_default(cmg_hierarchy_t h, cmg_solve_options_t *so);

/*
 * cmg_fiedler with per-solve options: a re-solve on a resident hierarchy with
 * a new Gaussian start (another seed) or from a given start vector on any
 * level, reusing the setup phase.  The Remark after Alg. 1 (Sec. 2) names
 * applications that compute the Fiedler vector many times, such as recursive
 * spectral bisection; there the setup is the part worth keeping.  With x0 on
 * level s, Alg. 3 runs on level s from x0 (Gram-Schmidt against 1 first),
 * then Step 3 continues from level s-1 down to 0 as usual; stats report 0
 * sweeps for the levels above s.  A host x0 is copied before the solve
 * starts (borrowed for the call only).  Other arguments, results and errors
 * as cmg_fiedler; INVALID_ARG also for a bad x0_level / x0_mem or a nonzero
 * reserved word.  Synchronises `stream`.
 */
cmg_status_t cmg_fiedler_ex(cmg_hierarchy_t h, const cmg_solve_options_t *so, double *u_out,
                            int32_t u_mem, double *lambda2_out, cmg_stats_t *stats_out,
                            void *stream);

/* Most eigenpairs cmg_eigenpairs computes at once. */
#define CMG_MAX_EIGENPAIRS 16

/*
 * k approximate eigenpairs (lambda_2 .. lambda_{k+1} and their vectors) by
 * the cascade of Alg. 1 with k vectors, the extension the Remark after
 * Alg. 4 (Sec. 3) describes: k Gaussian vectors on the coarsest level
 * (vector i keyed by seed + i), and on every level a block power iteration --
 * each sweep multiplies the k vectors by B_g = g I - L and orthogonalises
 * them (Gram-Schmidt against 1 and against the earlier vectors, in order,
 * then normalisation) -- until every vector's cosine with its previous
 * iterate is at least 1 - tol (or the hierarchy's FIXED / REPLAY schedule);
 * then each vector's Rayleigh quotient.  The hierarchy's setup (and its
 * options: tol, caps, schedule) is reused; sweeps are FP64.
 *   k: 1 .. min(CMG_MAX_EIGENPAIRS, n_J - 1).
 *   so: NULL for the hierarchy's seed; only so->seed is used (x0 must be NULL).
 *   U_out: double[k * n_0] in `u_mem` memory, or NULL: vector i at
 *     U_out + i n_0, unit length, orthogonal to 1 and to the others, scaled so
 *     that its largest-magnitude entry (lowest index on ties) is positive.
 *   lambda_out, residual_out (host double[k], nullable): per vector the
 *     Rayleigh quotient u^T L u and ||(L - lambda I) u|| (Sec. 4).
 *   stats_out (nullable): sizes and per-level sweeps (lambda2/residual: the
 *     first vector's).
 * Returns OK, WARN_MAXITER, or an error: INVALID_ARG, TOO_SMALL (the block
 * lost rank: fewer than k independent directions), OOM, CUDA,
 * DEVICE_TIMEOUT.  Synchronises `stream`.
 */
cmg_status_t cmg_eigenpairs(cmg_hierarchy_t h, int32_t k, const cmg_solve_options_t *so,
                            double *U_out, int32_t u_mem, double *lambda_out, double *residual_out,
                            cmg_stats_t *stats_out, void *stream);

/* Level count and per-level sizes (host arrays of length >= levels, nullable). */
cmg_status_t cmg_hierarchy_info(cmg_hierarchy_t h, int32_t *levels, int64_t *n_per_level,
                                int64_t *nnz_per_level);

/* Sweep kernel that runs Alg. 3 on each level (host arrays of length >= levels,
 * nullable).  kind_out[j]: 0 = one CTA with the level in shared memory,
 * 1 = slice kernel over the level's sweep layout, 2 = the same with the
 * iterate's first staged_out[j] entries (its highest-degree rows) copied to
 * shared memory every sweep, 3 = row-tile kernel, 4 = two-phase kernel (a
 * sweep in passes: the columns' values are first copied, block by block
 * through shared memory, into a buffer in the order the rows consume them,
 * then every row sums a contiguous stream in 64-bit fixed point; taken only
 * when the environment variable CMG_2P=1 is set at cmg_setup, for every
 * level with a sweep layout), 5 = cluster kernel (FP64 sweeps of a level of
 * 512 to a few thousand rows spread over one thread-block cluster of 2 to 8
 * CTAs: every CTA holds the iterate, computes its share of the rows and
 * stores them into the others' shared memory; chosen at setup unless
 * CMG_CLUSTER=0).  Staging is chosen at setup where the gathers
 * it serves are several per staged entry and SM; CMG_STAGE=0 (never) or
 * CMG_STAGE=1 (every slice level), read by cmg_setup, overrides that rule.
 * Results do not depend on the kernel beyond rounding; every kernel sums in
 * a fixed order (or exactly), so repeated solves are bit-identical.
 * Errors: INVALID_ARG if h is NULL. */
cmg_status_t cmg_level_kernels(cmg_hierarchy_t h, int32_t *kind_out, int32_t *staged_out);

/* Sweep precision of each level (host int32 array of length >= levels):
 * CMG_PRECISION_FP32_SWEEP or CMG_PRECISION_FP64 (see the precision enum).
 * Errors: INVALID_ARG if h or prec_out is NULL. */
cmg_status_t cmg_level_precision(cmg_hierarchy_t h, int32_t *prec_out);

/* Device bytes held by the hierarchy (levels and solve workspace). */
cmg_status_t cmg_hierarchy_device_bytes(cmg_hierarchy_t h, size_t *bytes);

/* Upper estimate of the device bytes cmg_setup + cmg_fiedler hold for a graph
 * of n vertices and nnz stored entries (used for admission control). */
cmg_status_t cmg_estimate_device_bytes(int64_t n, int64_t nnz, int32_t precision, size_t *bytes);

/* Aggregate map of level `level` onto level+1 (Alg. 2's q): host int32[n_level].
 * Errors: INVALID_ARG if level is the coarsest or out of range. */
cmg_status_t cmg_get_aggregates(cmg_hierarchy_t h, int32_t level, int32_t *agg_out);

/* CSR of level `level` (off-diagonal weights; the diagonal is the row sum):
 * host int64[n+1], int32[nnz], double[nnz]; any pointer may be NULL.
 * Also returns the level's Gershgorin shift g through g_out (nullable). */
cmg_status_t cmg_get_level_csr(cmg_hierarchy_t h, int32_t level, int64_t *row_ptr, int32_t *col,
                               double *w, double *g_out);

/* Releases the hierarchy (stream-ordered on the stream it was built on). */
cmg_status_t cmg_free(cmg_hierarchy_t h);

/* ------------------------------------------------------------------------
 * Batched form: many independent graphs set up and solved together.  The
 * paper treats one graph; this form runs Alg. 1 on each graph of a batch
 * with results equal to what cmg_setup / cmg_fiedler give for that graph
 * alone (same hierarchy bit for bit, same vector within rounding), but with
 * the whole batch in one block-diagonal union per level: one coarsening
 * pass per level for all graphs, and one persistent kernel launch per level
 * for the power iteration of every graph on that level, the launches
 * replayed from a captured CUDA graph.
 *
 * Layout: graph q occupies rows graph_offsets[q] .. graph_offsets[q+1]-1 of
 * one CSR (row_ptr int64[N+1], col int32[nnz], w double[nnz]) whose column
 * indices are union indices; every entry of a row must stay inside the
 * row's graph.  graph_offsets (host int64[G+1]) starts at 0, ends at N, and
 * every graph has at least 2 vertices.  Result vectors use the same union
 * layout.
 * ---------------------------------------------------------------------- */
typedef struct cmg_batch_s *cmg_batch_t;

/* Batched Alg. 1 Step 1.  Same input contract per graph as cmg_setup (checked
 * when opts->validate != 0; an entry leaving its graph is BAD_CSR).  A graph
 * stops coarsening exactly where cmg_setup would stop it.
 * Errors: as cmg_setup; INVALID_ARG also for num_graphs < 1 or offsets that
 * are not non-decreasing; TOO_SMALL for a graph with fewer than 2 vertices. */
cmg_status_t cmg_setup_batch(int32_t num_graphs, const int64_t *graph_offsets,
                             const int64_t *row_ptr, const int32_t *col, const double *w,
                             int32_t mem, const cmg_options_t *opts, void *stream,
                             cmg_batch_t *out);

/* Batched Alg. 1 Steps 2-3 for every graph of the batch.
 *   u_out: double[N] in `u_mem` memory, or NULL: graph q's unit Fiedler vector
 *     (sign rule of cmg_fiedler) in rows graph_offsets[q] .. graph_offsets[q+1]-1.
 *   lambda2_out, residual_out (host double[G], nullable): per graph.
 *   status_out (host int32[G], nullable): CMG_OK or CMG_WARN_MAXITER per graph.
 * Returns WARN_MAXITER if any graph hit a sweep cap, else OK, or an error
 * (INVALID_ARG, OOM, CUDA).  Synchronises `stream`. */
cmg_status_t cmg_fiedler_batch(cmg_batch_t b, double *u_out, int32_t u_mem, double *lambda2_out,
                               double *residual_out, int32_t *status_out, void *stream);

/* Number of graphs, union levels, and the union size of level `level`
 * (nullable outputs; level < 0 skips the sizes). */
cmg_status_t cmg_batch_info(cmg_batch_t b, int32_t *num_graphs, int32_t *union_levels,
                            int32_t level, int64_t *n_level, int64_t *nnz_level);

/* Per-graph report of the last cmg_fiedler_batch (sizes, sweeps, cosines,
 * lambda2, residual, status; level_ms and finalize_ms are 0).  Before the
 * first solve, only levels / n / nnz are filled. */
cmg_status_t cmg_batch_stats(cmg_batch_t b, int32_t graph, cmg_stats_t *stats_out);

/* Graph `graph`'s aggregate map of level `level` onto level+1 in the graph's
 * own numbering (host int32[n_level of that graph]); as cmg_get_aggregates. */
cmg_status_t cmg_batch_get_aggregates(cmg_batch_t b, int32_t graph, int32_t level,
                                      int32_t *agg_out);

/* Graph `graph`'s CSR of level `level` in its own numbering; as
 * cmg_get_level_csr (row_ptr int64[n+1], col int32[nnz], w double[nnz],
 * g_out the level's Gershgorin shift; all nullable). */
cmg_status_t cmg_batch_get_level_csr(cmg_batch_t b, int32_t graph, int32_t level, int64_t *row_ptr,
                                     int32_t *col, double *w, double *g_out);

/* Schedule REPLAY for a batch: exact sweep counts per graph and level, host
 * int32[G * CMG_MAX_LEVELS] (graph-major); NULL returns to
 * opts.replay_sweeps for every graph.  Used only when opts.schedule is
 * CMG_SCHEDULE_REPLAY. */
cmg_status_t cmg_batch_set_replay(cmg_batch_t b, const int32_t *sweeps);

/* Launch shape of a union level's power-iteration kernel: `threads_per_graph`
 * threads (32..1024, a multiple of 32) work on one graph at a time,
 * `lanes_per_row` (1, 2, 4, 8, 16 or 32) of them on each row with more than
 * 32 entries (shorter rows take one lane each, 32 rows per warp); a CTA
 * holds `graphs_per_cta` such groups (tpg * gpc <= 1024; gpc <= 15 unless
 * tpg = 32); `stage_csr` = 1 lets a group copy its graph's CSR into shared
 * memory when it fits.  cmg_batch_config reads or sets one level's shape
 * (set = 0 reads into the pointers, 1 writes them); cmg_batch_autotune times
 * candidate shapes on the batch itself (a few sweeps per graph on every
 * level, `stream`-ordered, synchronising) and keeps the fastest per level.
 * Results do not depend on the shape beyond rounding. */
typedef struct cmg_batch_shape {
    int32_t threads_per_graph;
    int32_t lanes_per_row;
    int32_t graphs_per_cta;
    int32_t stage_csr;
} cmg_batch_shape_t;
cmg_status_t cmg_batch_config(cmg_batch_t b, int32_t level, int32_t set, cmg_batch_shape_t *shape);
cmg_status_t cmg_batch_autotune(cmg_batch_t b, void *stream);

/* Device time of union level `level`'s power-iteration launch in the last
 * cmg_fiedler_batch, when options.timing = 1 (the launches are then issued
 * one by one with CUDA events instead of replaying the captured graph);
 * else 0. */
cmg_status_t cmg_batch_level_ms(cmg_batch_t b, int32_t level, double *ms);

/* Device bytes held by the batch (levels and solve workspace). */
cmg_status_t cmg_batch_device_bytes(cmg_batch_t b, size_t *bytes);

/* Releases the batch. */
cmg_status_t cmg_batch_free(cmg_batch_t b);

/* ------------------------------------------------------------------------
 * Serving: a request loop for Fiedler solves.  The paper has no
 * counterpart; it runs Alg. 1 for a stream of requests on one GPU.
 *
 * Graphs are registered once (host CSR, borrowed: the arrays must stay valid
 * and unchanged until cmg_server_destroy).  A request names a graph and
 * receives its vector, lambda2 and residual.  `workers` host threads, each
 * with its own CUDA stream, run jobs so that their device work overlaps.  A
 * job starts only when its device memory (cmg_estimate_device_bytes per
 * graph; the exact size for a resident hierarchy) fits in `mem_budget`;
 * idle resident hierarchies are evicted least recently used first to make
 * room, and a request that can never fit fails with CMG_ERR_TOO_LARGE.
 * Jobs: a graph with a resident hierarchy is solved with cmg_fiedler
 * (warm); a graph with n > batch_max_n is set up with cmg_setup, solved and
 * (keep_resident) kept; every pending request for a smaller graph without a
 * hierarchy, up to max_batch, joins one batched job (cmg_setup_batch +
 * cmg_fiedler_batch) when at least min_batch of them are pending (a batched
 * job gives each graph a group of threads, which pays only when many graphs
 * fill the GPU; fewer run alone, with the whole GPU each), so requests
 * arriving while others run are admitted together as soon as a worker and
 * memory free up.  Pending requests are
 * taken first-fit in arrival order.  All requests use the server's options.
 * Admission estimate: cmg_estimate_device_bytes, plus three more copies of
 * level 0's stored levels for a graph whose largest degree exceeds 8 times
 * its mean (the coarse levels of such heavy-tailed graphs stay dense).
 * ---------------------------------------------------------------------- */
typedef struct cmg_server_s *cmg_server_t;

typedef struct cmg_server_config {
    int32_t workers;       /* concurrent jobs, 1..64 (4)                              */
    int32_t max_batch;     /* graphs per batched job; 1 disables batching (256)       */
    int64_t batch_max_n;   /* graphs with n <= batch_max_n are batched (8192): a
                              batched job runs each graph's sweeps on one thread
                              group, so a larger graph is faster alone              */
    uint64_t mem_budget;   /* device bytes for jobs and resident hierarchies;
                              0 = 80% of the free device memory at creation          */
    int32_t keep_resident; /* keep single-form hierarchies after their solve (1)      */
    int32_t min_batch;     /* batch small graphs only when at least this many cold
                              small requests are pending; fewer run alone (32).
                              0 selects the default                                  */
} cmg_server_config_t;

typedef struct cmg_request {
    int32_t status;        /* CMG_OK, CMG_WARN_MAXITER or the error of the job        */
    int32_t batch_size;    /* graphs in the job that solved the request (1 = alone)   */
    int32_t warm;          /* 1: the hierarchy was resident (solve only)              */
    int32_t pad;
    double lambda2;
    double residual;
    uint64_t submit_ns, admit_ns, done_ns;  /* host steady clock                      */
} cmg_request_t;

typedef struct cmg_server_stats {
    int64_t completed, single_jobs, batch_jobs, warm_jobs, evictions, resident;
    uint64_t peak_bytes;   /* most device bytes reserved at once (bookkeeping)       */
    uint64_t used_bytes;   /* reserved now (running jobs + resident hierarchies)     */
    uint64_t budget_bytes;
    uint64_t measured_peak_bytes; /* most bytes of the library's device memory pool
                              in use at once since cmg_server_create, as the CUDA
                              driver counts them (the pool serves every user of the
                              library on this device in this process)            */
} cmg_server_stats_t;

/* workers 4, max_batch 256, batch_max_n 8192, mem_budget 0, keep_resident 1,
 * min_batch 32. */
cmg_status_t cmg_server_config_default(cmg_server_config_t *cfg);
/* Starts the workers on the current device.  opts: NULL = defaults
 * (options.timing must be 0).  Errors: INVALID_ARG, CUDA. */
cmg_status_t cmg_server_create(const cmg_server_config_t *cfg, const cmg_options_t *opts,
                               cmg_server_t *out);
/* Registers a graph (host CSR as for cmg_setup, borrowed); *graph_id
 * receives its id.  The input contract is checked when a job sets it up. */
cmg_status_t cmg_server_add_graph(cmg_server_t s, int64_t n, const int64_t *row_ptr,
                                  const int32_t *col, const double *w, int64_t *graph_id);
/* Queues a solve of graph `graph_id`; u_out (host double[n], nullable) must
 * stay valid until the request completes.  *ticket identifies it. */
cmg_status_t cmg_server_submit(cmg_server_t s, int64_t graph_id, double *u_out, int64_t *ticket);
/* cmg_server_submit with per-solve options (cmg_fiedler_ex): a re-solve of a
 * registered graph with another seed, or from a start vector x0 (host memory,
 * borrowed until the request completes), on the graph's resident hierarchy
 * when it has one.  Such a request never joins a batched job.
 * Errors: INVALID_ARG for a NULL `so`, a device x0 or a nonzero reserved
 * word; a bad x0_level is the request's own status. */
cmg_status_t cmg_server_submit_ex(cmg_server_t s, int64_t graph_id, const cmg_solve_options_t *so,
                                  double *u_out, int64_t *ticket);
/* Blocks until the request completes; fills *out (nullable) and returns the
 * request's status.  A ticket can be waited for once. */
cmg_status_t cmg_server_wait(cmg_server_t s, int64_t ticket, cmg_request_t *out);
/* cmg_server_wait that gives up after timeout_ms milliseconds with
 * CMG_ERR_TIMEOUT (the request stays queued and can be waited for again). */
cmg_status_t cmg_server_wait_for(cmg_server_t s, int64_t ticket, int64_t timeout_ms,
                                 cmg_request_t *out);
cmg_status_t cmg_server_get_stats(cmg_server_t s, cmg_server_stats_t *out);
/* Finishes every queued request, stops the workers, frees the hierarchies. */
cmg_status_t cmg_server_destroy(cmg_server_t s);

/* ------------------------------------------------------------------------
 * Geometric cascadic multigrid, Alg. 4 (Sec. 3), in the structured setting of
 * the paper's Table 4 experiment (Sec. 4): the unit-weight grid graph on
 * N^dim vertices (dim 2: 5-point, dim 3: 7-point; vertex (x, y, z) has id
 * (z N + y) N + x), coarsened geometrically J times by keeping every other
 * vertex (level j has N_j = (N - 1)/2^j + 1 vertices per side; N - 1 must be
 * a multiple of 2^J).  The coarsest level starts from its exact eigenvector
 * for lambda_2 that varies along x, cos(pi (x + 1/2) / N_J) (Alg. 4 line 2:
 * solved exactly); every finer level from the multilinear interpolant of the
 * coarser result, made orthogonal to 1 and normalised, then k_j =
 * ceil(k0 beta^j) smoothing steps u <- (I - A_j / ||A_j||_inf) u (Alg. 4
 * line 4), each followed by Gram-Schmidt against 1 and normalisation.
 *   u_out: double[N^dim] in `u_mem` memory, or NULL: the level-0 result.
 *   r0_out, rk_out (host double[J+1], nullable): per level j the Rayleigh
 *     quotient u^T A_j u / u^T u of the prolonged start and of the result
 *     after the k_j steps (Table 4 prints |lambda_2^(j) - r0| and
 *     |lambda_2^(j) - rk| with lambda_2^(j) = 2 - 2 cos(pi / N_j)); for the
 *     coarsest level both are its exact vector's quotient.
 *   k_out (host int32[J+1], nullable): k_j (0 on the coarsest level).
 * FP64 throughout.  Errors: INVALID_ARG (dim not 2 or 3, N < 3, N - 1 not a
 * multiple of 2^J, J outside 0..30, k0 < 0, beta <= 0, bad u_mem), TOO_LARGE
 * (2 dim N^dim >= 2^31), OOM, CUDA, DEVICE_TIMEOUT.  Synchronises `stream`.
 * ---------------------------------------------------------------------- */
cmg_status_t cmg_gcmg_grid(int32_t dim, int32_t N, int32_t J, double beta, int32_t k0,
                           double *u_out, int32_t u_mem, double *r0_out, double *rk_out,
                           int32_t *k_out, void *stream);

/* ------------------------------------------------------------------------
 * Step entry points.  Each runs one step of the method on DEVICE buffers in
 * the library's internal layout (row_ptr as int32[n+1]) on `stream`; they
 * exist so every step can be checked on its own.  Inputs are assumed to meet
 * the input contract (no validation).  Scratch memory is allocated and freed
 * inside the call.
 * ---------------------------------------------------------------------- */

/* Alg. 2, "m <- argmin(L(:, v))": m_out[v] = the neighbour j of maximum w_vj,
 * ties to the lowest j; -1 for a vertex without neighbours.  int32[n]. */
cmg_status_t cmg_heaviest_neighbour(int32_t n, const int32_t *row_ptr, const int32_t *col,
                                    const double *w, int32_t *m_out, void *stream);

/* Alg. 2, "p <- randperm(n)", as visit ranks r(v) = p^{-1}(v): a 4-round
 * Feistel permutation of [0, 2^k) keyed by splitmix64(seed ^ level*0x9E3779B97F4A7C15 ^ t),
 * restricted to [0, n) by cycle walking.  rank_out: device uint32[n]. */
cmg_status_t cmg_visit_ranks(int32_t n, uint64_t seed, int32_t level, uint32_t *rank_out,
                             void *stream);

/* Alg. 2 (heavy edge coarsening) for the visit ranks `rank` (device uint32[n],
 * a permutation of [0, n)): agg_out (device int32[n]) receives q with labels
 * 0..c-1 numbered in visit order; *c_out (host) receives c.  The result equals
 * the sequential algorithm exactly.  Synchronises `stream`. */
cmg_status_t cmg_hec_aggregate(int32_t n, const int32_t *row_ptr, const int32_t *col,
                               const double *w, const uint32_t *rank, int32_t *agg_out,
                               int64_t *c_out, void *stream);

/* Alg. 3 with a fixed sweep count: Gram-Schmidt of x_in against 1,
 * normalisation, then exactly k sweeps u <- B_g u / ||B_g u|| (each followed
 * by projection against 1), B_g = g I - L.  g <= 0 means "use
 * max_i sum_j |l_ij|".  x_in, u_out: device double[n].  *cos_out (host,
 * nullable): cosine between the last two iterates.  Synchronises `stream`. */
cmg_status_t cmg_power_sweeps(int32_t n, const int32_t *row_ptr, const int32_t *col,
                              const double *w, double g, const double *x_in, int32_t k,
                              double *u_out, double *cos_out, void *stream);

/* Rayleigh quotient r = u^T L u / u^T u and residual ||(L - r I) u|| / ||u||
 * (Sec. 4) of device double[n] u; results to host.  Synchronises `stream`. */
cmg_status_t cmg_rayleigh_residual(int32_t n, const int32_t *row_ptr, const int32_t *col,
                                   const double *w, const double *u, double *lambda_out,
                                   double *residual_out, void *stream);

/* Limits of cmg_power_sweeps_noalloc. */
#define CMG_NOALLOC_MAX_N 262144      /* rows    */
#define CMG_NOALLOC_MAX_NNZ 4194304   /* entries */

/* cmg_power_sweeps without any device memory allocation.  The paper has no
 * counterpart; this entry point exists for callers that must not allocate:
 * an application whose device memory is already fully reserved by its own
 * allocator (a cudaMalloc from this library would fail or fragment that
 * pool), or a latency-critical loop in which cudaMalloc / cudaFree, which may
 * synchronise the device, are not allowed.  Same arguments, results and
 * errors as cmg_power_sweeps, except:
 *   - n <= CMG_NOALLOC_MAX_N and nnz <= CMG_NOALLOC_MAX_NNZ; larger graphs
 *     are rejected with CMG_ERR_TOO_LARGE before any device work;
 *   - its scratch is one fixed array of about 8.4 MB in device memory that
 *     every GPU which loads this library holds until the process exits;
 *   - every call looks up that array's device address (cudaGetSymbolAddress,
 *     which allocates nothing) with the device current; the first lookup on
 *     a device loads the library's device code there, so make the first
 *     call on each device before any stream capture;
 *   - all calls on a device share the array, so calls whose GPU work
 *     overlaps (other streams, other host threads) race and give wrong
 *     results: serialise them.  Each call clears what must start at zero.
 * No cudaMalloc, cudaFree or allocating library routine is called. */
cmg_status_t cmg_power_sweeps_noalloc(int32_t n, const int32_t *row_ptr, const int32_t *col,
                                      const double *w, double g, const double *x_in, int32_t k,
                                      double *u_out, double *cos_out, void *stream);

/* Number of kernel launches this library has issued in this process (all
 * devices, all threads): lets a caller count the device work of a call. */
cmg_status_t cmg_kernel_launches(uint64_t *count);

/* Test hook for the error paths: the k-th next device allocation made by the
 * library fails with CMG_ERR_OOM (k = 0: the next one; k < 0: disarm).  The
 * paper has no counterpart; it exists so out-of-memory handling can be
 * tested without exhausting the device. */
cmg_status_t cmg_debug_fail_alloc_after(int64_t k);

/* Test hook for the device-side timeout path: the `launch`-th next
 * cooperative kernel launch of this library that uses more than one CTA
 * (0: the next one, counted over all threads) never releases its grid
 * barrier number `barrier` (0..254), so every CTA's bounded wait there runs
 * out (after 20 ms instead of the usual 2 s), the kernel returns, and the
 * call that issued it reports CMG_ERR_DEVICE_TIMEOUT; later launches of the
 * same call return at their first barrier.  launch < 0 disarms.  The paper
 * has no counterpart.  Errors: INVALID_ARG for a barrier outside 0..254. */
cmg_status_t cmg_debug_stall_barrier(int64_t launch, int32_t barrier);

#ifdef __cplusplus
}
#endif
#endif /* CMG_H */
