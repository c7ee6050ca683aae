/*
 * gmg.h -- C ABI of the GB300 geometric-multigrid solve library (libgmg.so).
 *
 * Method: the multigrid solver of Wiersma, Nasikun, Eisemann, Hildebrandt,
 * "A Fast Geometric Multigrid Method for Curved Surfaces" (SIGGRAPH 2023):
 *   Alg. 1  setup A_{l+1} = P_l^T A_l P_l, then repeat V-cycles until
 *           ||A x - b|| <= eps ||b||;
 *   Alg. 2  V-cycle: Gauss-Seidel pre-relaxation, residual, restriction by
 *           P_l^T, recursive coarse correction with zero initial guess,
 *           prolongation by P_l, post-relaxation; direct solve on the
 *           coarsest level;
 *   Sec. 4  prolongations with at most three entries per row (an INPUT here).
 *
 * Conventions for every entry point:
 *   - Every call returns a gmg_status; GMG_OK on success.  On failure
 *     gmg_last_error() returns a human-readable message for the calling
 *     thread.  No entry point traps, aborts or waits without bound.
 *   - "host" arrays are ordinary CPU memory, read (or written) only during the
 *     call.  "device" arrays are CUDA global-memory pointers on the handle's
 *     device; results in device arrays are ready once work queued on `stream`
 *     before the call returns has completed.
 *   - `stream` is a cudaStream_t passed as void* (NULL = legacy default stream).
 *   - The library copies and owns everything setup needs; caller buffers are
 *     borrowed only for the duration of a call.  One handle must not be used
 *     from two host threads, or on two streams, at the same time.
 *   - Vectors exchanged through the API are in the caller's row numbering
 *     (the numbering of the A and P_l given to gmg_setup); internal colour
 *     permutations are never visible.
 *   - Indices are 0-based.
 */
#ifndef GMG_H
#define GMG_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct gmg_ctx *gmg_handle;

typedef enum {
  GMG_OK = 0,
  GMG_ERR_INVALID_ARG = 1,    /* bad pointer, size, index or option          */
  GMG_ERR_NOT_SPD = 2,        /* A: a diagonal entry <= 0 or A != A^T        */
  GMG_ERR_EMPTY_P_COLUMN = 3, /* a coarse point no fine row maps to: its
                                 Galerkin diagonal would be 0 (the NaN rows
                                 the paper reports for its experiments)      */
  GMG_ERR_CHOLESKY = 4,       /* coarsest operator not positive definite     */
  GMG_ERR_NOT_CONVERGED = 5,  /* max_iter reached; x holds the last iterate  */
  GMG_ERR_NONFINITE = 6,      /* NaN/Inf in an input or in an iterate        */
  GMG_ERR_OOM = 7,            /* device allocation failed                    */
  GMG_ERR_CUDA = 8,           /* a CUDA runtime call failed                  */
  GMG_ERR_TIMEOUT = 9,        /* a bounded device-side wait gave up          */
  GMG_ERR_TOO_LARGE = 10      /* a size exceeds a documented limit           */
} gmg_status;

/* Arithmetic of the V-cycle inside gmg_solve. */
enum {
  GMG_FP64 = 0,        /* plain Alg. 1: FP64 V-cycles, x <- MGI(x, b, 1)       */
  GMG_FP32_REFINE = 1, /* FP64 iterative refinement: r = b - A x (FP64),
                          e = MGI(0, r, 1) in FP32 (coarsest solve FP64),
                          x += e; identical to GMG_FP64 in exact arithmetic   */
  GMG_FP32_PCG = 2,    /* FP64 conjugate gradients preconditioned by one FP32
                          V-cycle per iteration (flexible Polak-Ribiere beta)  */
  GMG_FP64_PCG = 3     /* the same conjugate gradients preconditioned by one
                          FP64 V-cycle per iteration (separates the gain of CG
                          from the gain of the FP32 cycle)                     */
};

enum { GMG_MEM_DEVICE = 0, GMG_MEM_HOST = 1 };

/* System matrix A (host).  n x n, CSR with 64-bit row pointers, sorted and
 * unique column indices per row, the diagonal present in every row.  A must be
 * symmetric with a positive diagonal (A = M + tL of the paper's Eq.
 * (smoothing) or Eq. (Poisson)). */
typedef struct {
  int64_t n;
  const int64_t *rowptr; /* n + 1 */
  const int32_t *col;    /* rowptr[n] */
  const double *val;     /* rowptr[n] */
} gmg_csr;

/* Prolongation P_l in R^{n_fine x n_coarse} (host), Sec. 4.4: row i holds
 * three (index, weight) slots idx[3i+s], w[3i+s], s = 0..2.  A slot with
 * w == 0 is unused (its index must still be in [0, n_coarse)).  The non-zero
 * slots of a row must name distinct coarse points.  Every coarse point must
 * appear in some row with w != 0. */
typedef struct {
  int64_t n_fine, n_coarse;
  const int32_t *idx; /* 3 * n_fine */
  const double *w;    /* 3 * n_fine */
} gmg_prolong;

typedef struct {
  int precision;  /* GMG_FP64 | GMG_FP32_REFINE | GMG_FP32_PCG | GMG_FP64_PCG
                     (default REFINE)                                          */
  int nu_pre;     /* Gauss-Seidel sweeps before the coarse correction (2)     */
  int nu_post;    /* sweeps after it (2)                                      */
  int max_iter;   /* outer iterations (100)                                   */
  int post_forward; /* 0: post-relaxation visits colours in descending order
                       (symmetric cycle, required by the PCG modes); 1: ascending */
  int use_graphs; /* 1: replay each cycle from a captured CUDA graph (default)  */
} gmg_options;

typedef struct {
  int iters;          /* V-cycles (or PCG iterations) performed              */
  double rel_res;     /* final ||b - A x||_2 / ||b||_2, in FP64              */
  double *history;    /* optional host buffer: history[k] = relative residual
                         after k iterations, history[0] for the initial guess */
  int history_cap;    /* capacity of `history` in doubles                    */
} gmg_solve_info;

/* Fills `opt` with the defaults listed above. */
void gmg_default_options(gmg_options *opt);

/* Static text for a status code. */
const char *gmg_status_string(gmg_status s);

/* Message of the last failure on the calling thread ("" if none). */
const char *gmg_last_error(void);

/* Alg. 1 setup.  Copies A and the `n_prolong` prolongations (finest first;
 * P[l].n_fine must equal the size of level l), computes every Galerkin level
 * A_{l+1} = P_l^T A_l P_l on the GPU (two-pass symbolic + numeric product,
 * mirrored to exact symmetry), colours every level, lays the levels out colour
 * by colour, and forms the explicit FP64 inverse of the coarsest level (the
 * direct solve of Alg. 2; block Gauss-Jordan sweeps, every pivot checked
 * positive, which for a symmetric matrix is the Cholesky criterion).
 *
 * `coloring` selects the Gauss-Seidel colouring of Sec. 3's relaxation: NULL,
 * or an array of n_prolong + 1 host pointers, one per level, each NULL (that
 * level gets the library's deterministic colouring: greedy first fit in
 * increasing row index and in smallest-last order, each improved by eight
 * iterated-greedy passes, the one with fewer colours kept) or n_l colours in
 * [0, n_l) in the caller's numbering of level l.  No
 * two adjacent rows of A_l (a stored off-diagonal entry) may share a colour;
 * pre-relaxation visits the colours in ascending order, post-relaxation in
 * descending order.  The coarse levels are numbered as the columns of P_l, and
 * their patterns are those of the Galerkin products (e.g. as the oracle or a
 * previous gmg_level_export reports them).
 *
 * `opt` may be NULL (defaults).  On success *h owns all device memory of the
 * hierarchy; release it with gmg_destroy.  Errors: INVALID_ARG (also an
 * improper or out-of-range colouring), NOT_SPD, EMPTY_P_COLUMN, CHOLESKY,
 * NONFINITE, TOO_LARGE (coarsest level above 8192 rows, or a Galerkin row with
 * more than 768 entries), OOM, CUDA. */
gmg_status gmg_setup(gmg_handle *h, const gmg_csr *A, int n_prolong, const gmg_prolong *P,
                     const int32_t *const *coloring, const gmg_options *opt, void *stream);

/* The colouring gmg_setup gives a level when the caller passes none (the
 * multicolour ordering of Sec. 3's Gauss-Seidel relaxation): greedy first
 * fit in increasing row index and in smallest-last order, each improved by
 * eight iterated-greedy passes, the one with fewer colours kept (the
 * index-order one on a tie).  Host only: no GPU is used.  rowptr (n + 1) and
 * col (rowptr[n]) are a symmetric sparsity pattern with sorted, unique columns
 * per row (the diagonal may be present); color receives n colours in
 * [0, *ncolor).  All buffers are the caller's host memory.  Errors:
 * INVALID_ARG (null pointer, n < 0, rowptr not monotone or not starting at
 * 0, a column out of range, unsorted or repeated, or a pattern that is not
 * symmetric). */
gmg_status gmg_colour(int64_t n, const int64_t *rowptr, const int32_t *col, int32_t *color, int32_t *ncolor);

/* Numeric refresh: new values for A on the SAME sparsity pattern (`val` has
 * rowptr[n] entries in the pattern's order; host or device per `mem`).
 * Recomputes every Galerkin level on the GPU without touching the host-side
 * structure, checks them before returning, and starts the coarsest inverse
 * on a stream of the handle's own, ordered after the Galerkin values on
 * `stream`.  The next call on the handle that needs the inverse (gmg_solve,
 * gmg_solve_batched, gmg_vcycle, gmg_vcycle_batched, gmg_coarse_solve, or
 * another refresh) makes its own stream wait for it (a CG solve only right
 * before its first coarsest solve, so the first cycle's descent overlaps
 * it) and reports a non-positive pivot of it as CHOLESKY.
 * Errors: NOT_SPD, NONFINITE (this call); CHOLESKY (the next such call). */
gmg_status gmg_set_values(gmg_handle h, const double *val, int mem, void *stream);

/* Alg. 1 iteration: solves A x = b to ||b - A x||_2 <= tol ||b||_2.  `x` holds
 * the initial guess on entry and the solution on exit (n doubles, host or
 * device per `mem`).  b == 0 gives x = 0 after 0 iterations.  `info` may be
 * NULL.  Errors: NOT_CONVERGED (x = last iterate), NONFINITE, INVALID_ARG,
 * CHOLESKY (the coarsest inverse of a preceding refresh). */
gmg_status gmg_solve(gmg_handle h, const double *b, double *x, double tol, int mem, gmg_solve_info *info,
                     void *stream);

/* Batched right-hand sides: Alg. 1 (the iteration x <- x + MGI(0, b - A x, 1),
 * which equals x <- MGI(x, b, 1) in exact arithmetic because the cycle of
 * Alg. 2 is affine in x) for nrhs systems with the same A at once; the paper
 * solves one right-hand side at a time, batching is this library's addition.
 * B and X are n x nrhs, row-major (element (i, c) at i * nrhs + c), host or
 * device per `mem`.  Every column is solved to the same tolerance with FP32
 * V-cycles that read each matrix once for all columns, inside FP64
 * refinement.  1 <= nrhs <= 16.  info->iters counts the outer iterations of
 * the batch (every column takes part in each). */
gmg_status gmg_solve_batched(gmg_handle h, int nrhs, const double *B, double *X, double tol, int mem,
                             gmg_solve_info *info, void *stream);

/* ---- A(t) = M + t L kept split (Eq. (smoothing): M lumped mass, L the
 * Laplacian) and the adjoint gradient of a loss of x = A(t)^-1 M u0 ---- */

/* Like gmg_setup (colouring included) for A = M + t L, remembering M (host,
 * n diagonal entries) and L (host CSR; every row must store its diagonal; A
 * shares L's pattern).
 * Errors: those of gmg_setup, and INVALID_ARG for t < 0 or a missing L
 * diagonal. */
gmg_status gmg_setup_ML(gmg_handle *h, const double *M_diag, const gmg_csr *L, double t, int n_prolong,
                        const gmg_prolong *P, const int32_t *const *coloring, const gmg_options *opt,
                        void *stream);

/* Numeric refresh for a new t: A_1 = M + t L on the GPU, then every
 * Galerkin level and the coarsest inverse (as gmg_set_values, with the same
 * overlap of the inverse and the same errors). */
gmg_status gmg_set_t(gmg_handle h, double t, void *stream);

/* out = M u (device vectors, caller numbering): the right-hand side M u0 of
 * Eq. (smoothing). */
gmg_status gmg_mass(gmg_handle h, const double *u, double *out, void *stream);

/* Gradients of a loss of x = A(t)^-1 M u0, given x and the adjoint
 * lambda = A(t)^-1 (dloss/dx) (solved with the same hierarchy since A is
 * symmetric): grad_u0 = M lambda (n), *dLdt = -lambda^T L x (one device
 * double, summed in a fixed order), and G_vals[k] = -lambda_i x_j for the
 * k-th stored entry (i, j) of L (dloss/dA on A's pattern).  All device
 * pointers; any output may be NULL.  Requires a handle from gmg_setup_ML. */
gmg_status gmg_grad(gmg_handle h, const double *lambda, const double *x, double *grad_u0, double *dLdt,
                    double *G_vals, void *stream);

/* The same pattern gradient as gmg_grad without the u0 gradient:
 * G_vals[k] = -lambda_i x_j for the k-th stored entry (i, j) of L (dloss/dA
 * on A's pattern, since dA/dt = L the chain rule gives dloss/dt from it) and
 * *dLdt = -lambda^T L x; either output may be NULL.  Device pointers;
 * requires a handle from gmg_setup_ML. */
gmg_status gmg_grad_pattern(gmg_handle h, const double *lambda, const double *x, double *G_vals, double *dLdt,
                            void *stream);

/* ---- Sec. 4 hierarchy construction on the GPU ----
 * Builds the prolongations P_l that gmg_setup takes, from the finest level's
 * points and neighbour graph, level after level while a level has more than
 * `stop` points (and at most max_levels levels; a level that does not shrink
 * ends the hierarchy):
 *   Sec. 4.2 sampling: points swept in index order; an eligible point becomes
 *            a sample and makes every point within Dijkstra distance r
 *            (Euclidean edge lengths, inside the sample's 2-ring) ineligible;
 *            r = phi^(-1/3) times the mean edge length (summed per row, per
 *            block of 1024 rows, then over blocks, each in index order);
 *   Sec. 4.3 graph Voronoi cells of the samples (multi-source shortest paths,
 *            ties to the smaller sample index) and the coarse neighbour graph
 *            of cells that share an edge;
 *   Sec. 4.4 coarse points at the cell means; for every point the closest
 *            point on the candidate triangles (3-cliques of the coarse graph
 *            with area above 1e-12 times the squared mean edge length) at its
 *            own cell's sample, with barycentric weights (ties to the
 *            lexicographically smallest triangle), inverse-distance weights
 *            over the three closest of the sample and its coarse neighbours
 *            when there is no candidate triangle, and the sample's own row
 *            made the identity for a coarse column left empty.
 * X: 3n host doubles (point i at X[3i..3i+2]); rowptr (n + 1), col: the
 * symmetric neighbour graph (host CSR, sorted columns, no self loops).
 * 0 < phi < 1 (the paper uses 1/8).  *out receives a host-side record of
 * every level (release with gmg_destroy_hierarchy); device memory is used only
 * during the call.  Errors: INVALID_ARG, NONFINITE, TOO_LARGE (a 2-ring of
 * more than 96 points, a cell bordering more than 512 cells, a sample with
 * more than 63 coarse neighbours), OOM, CUDA. */
typedef struct gmg_hier_ctx *gmg_hierarchy;
gmg_status gmg_build_hierarchy(gmg_hierarchy *out, int64_t n, const double *X, const int64_t *rowptr,
                               const int32_t *col, double phi, int64_t stop, int max_levels, void *stream);
/* Number of prolongations built and the construction's GPU time in ms
 * (either output may be NULL). */
gmg_status gmg_hierarchy_info(gmg_hierarchy h, int *n_prolong, double *build_ms);
/* Level l's record (host outputs, each may be NULL): sizes; P_l as three
 * (index, weight) slots per fine row (idx, w: 3 n_fine, the layout gmg_setup
 * takes); the samples (fine index of every coarse point, n_coarse), the cell
 * of every fine point (n_fine), the coarse points (3 n_coarse), the coarse
 * neighbour graph (graph_rowptr n_coarse + 1, graph_col graph_nnz), and
 * stats = {fallback rows, repaired columns, single-entry rows, samples}. */
gmg_status gmg_hierarchy_level(gmg_hierarchy h, int l, int64_t *n_fine, int64_t *n_coarse, int64_t *graph_nnz,
                               int32_t *idx, double *w, int32_t *samples, int32_t *cell, double *Xc,
                               int64_t *graph_rowptr, int32_t *graph_col, int64_t *stats);
/* Releases the record (NULL accepted). */
gmg_status gmg_destroy_hierarchy(gmg_hierarchy h);

/* ---- many independent systems (meshes of uneven size) in one batch ---- */
typedef struct gmg_many_ctx *gmg_many;

/* Alg. 1 setup for `nmesh` systems: mesh k has system A[k] and the
 * n_prolong[k] prolongations P[k][0..] (host arrays, as for gmg_setup, with
 * the library's colourings).  Errors: those of gmg_setup for the failing mesh
 * (the message names it). */
gmg_status gmg_setup_many(gmg_many *m, int nmesh, const gmg_csr *A, const int *n_prolong,
                          const gmg_prolong *const *P, const gmg_options *opt, void *stream);

/* Alg. 1 for many independent systems at once (the paper solves one system
 * at a time; the batch is this library's addition): solves every mesh's
 * n_k x nrhs system A_k X_k = B_k (row-major, host or device per `mem`; B[k],
 * X[k] per mesh, X holding the initial guesses) to ||B - A X||_2 <= tol ||B||_2
 * per column, with FP32 V-cycles (Alg. 2, multi-right-hand-side kernels)
 * inside FP64 refinement.  The whole solve is one CUDA-graph launch: a
 * conditional WHILE node repeats an iteration in which every mesh that has
 * not converged runs its cycle (one conditional IF node per mesh, all
 * concurrent) and a device-side check updates each mesh's residual and
 * iteration count.  info (NULL or nmesh entries) receives the iteration count
 * and the worst column's relative residual per mesh; each mesh stops at its
 * own convergence.  Where the CUDA driver refuses conditional nodes, one
 * graph per iteration runs every mesh until all have converged.
 * 1 <= nrhs <= 16. */
gmg_status gmg_solve_many(gmg_many m, int nrhs, const double *const *B, double *const *X, double tol, int mem,
                          gmg_solve_info *info, void *stream);

/* gmg_autotune_batched for every mesh of the batch (blocks of nrhs
 * columns); the batch's captured iterations for that width are rebuilt on the
 * next solve. */
gmg_status gmg_autotune_many(gmg_many m, int nrhs, void *stream);

/* Releases the batch (NULL accepted). */
gmg_status gmg_destroy_many(gmg_many m);

/* Releases the handle and its device memory.  NULL is accepted. */
gmg_status gmg_destroy(gmg_handle h);

/* Launch-shape autotuner: for every level with Gauss-Seidel sweeps, times
 * four FP32 sweeps (captured in a CUDA graph, as a solve runs them) with each
 * row split over G = 1, 2, 4 and 8 warps and keeps the fastest G, then does
 * the same for the residual, which gets its own split.  Synchronises `stream`
 * first.  lanes_out (NULL or nlev - 1 ints) receives the Gauss-Seidel choices.  The split changes only the summation order of
 * a row.  Call between solves; it drops captured graphs (they are re-captured
 * on the next solve) and overwrites the FP32 work vectors. */
gmg_status gmg_autotune(gmg_handle h, int *lanes_out, void *stream);

/* Sets the warps-per-row split of every level with Gauss-Seidel sweeps, for
 * the sweeps and the residual alike
 * (lanes: nlev - 1 ints, each 1, 2, 4 or 8; GMG_ERR_INVALID_ARG otherwise,
 * nothing changed).  A fixed choice, e.g. one made earlier by gmg_autotune,
 * makes the launch sequence independent of timing.  Drops captured graphs
 * like gmg_autotune; synchronous. */
gmg_status gmg_set_lanes(gmg_handle h, const int *lanes);

/* Launch-shape autotuner of the multi-right-hand-side kernels (the batched
 * and many-mesh solves) for blocks of nrhs columns (rounded up to 1, 2, 4, 8
 * or 16): for every level with Gauss-Seidel sweeps, times four sweeps and a
 * residual (captured in a CUDA graph) with each row split over G = 1, 2, 4 and
 * 8 warps, and keeps the fastest G for that level and block width.  The
 * split changes only the summation order of a row.  Synchronises `stream`;
 * overwrites the batched work vectors.  lanes_out: NULL or nlev - 1 ints. */
gmg_status gmg_autotune_batched(gmg_handle h, int nrhs, int *lanes_out, void *stream);
/* Sets that split for blocks of nrhs columns (lanes: nlev - 1 ints, each 1,
 * 2, 4 or 8; GMG_ERR_INVALID_ARG otherwise, nothing changed). */
gmg_status gmg_set_lanes_batched(gmg_handle h, int nrhs, const int *lanes);

/* ---- kernel timing (measurement support, not part of the method) ----
 * With profiling enabled, gmg_solve records CUDA events on its stream around
 * the finest level's pre- and post-smoothing blocks and around every finest
 * V-cycle (inside captured graphs as external event nodes).
 * gmg_profile_read returns the sums since the last read and resets them:
 * out[0] = ms spent in finest-level smoothing blocks, out[1] = Gauss-Seidel
 * colour launches in them, out[2] = ms spent in V-cycles, out[3] = V-cycles. */
gmg_status gmg_profile(gmg_handle h, int enable);
/* Number of this library's CUDA kernels launched from the calling thread so
 * far (each replay of a captured graph counts its kernel nodes). */
uint64_t gmg_kernel_launches(void);
gmg_status gmg_profile_read(gmg_handle h, double *out /* 4 */);
/* Per-level sums over the same timed cycles since the last call (then reset):
 * out[4l + 0] = ms in level l's Gauss-Seidel sweeps, out[4l + 1] = its colour
 * launches, out[4l + 2] = ms in its residual, restriction and prolongation,
 * out[4l + 3] = ms of the whole level including the coarser ones.  A level
 * run inside the FP32 cycle's cluster tail, or as the coarsest solve, has
 * only out[4l + 3] (the levels below it report 0).  out: 4 * nlev doubles. */
gmg_status gmg_profile_levels(gmg_handle h, double *out);

/* ---- introspection (host outputs) ---- */
/* Warnings of the set-up (conditions that are not errors: the solve runs as
 * usual).  GMG_WARN_P_UNITY: the weights of some row of some P_l do not sum
 * to 1 within 1e-12 (the barycentric weights of Sec. 4.4, and the fallback's
 * normalised weights, sum to 1, so that a constant on a coarse level
 * prolongs to a constant).  *flags receives the OR of the warning bits;
 * max_dev, if not NULL, receives the largest |sum_k w_ik - 1| over the rows
 * of every P_l.  Errors: INVALID_ARG (null handle or flags). */
#define GMG_WARN_P_UNITY 1u
gmg_status gmg_warnings(gmg_handle h, uint32_t *flags, double *max_dev);
gmg_status gmg_num_levels(gmg_handle h, int *nlev);
/* rows, stored entries (diagonal included) and colours of level l. */
gmg_status gmg_level_info(gmg_handle h, int l, int64_t *n, int64_t *nnz, int *ncolors);

/* How the FP32 V-cycle runs level l (the FP64 cycle always uses one launch per
 * colour): 0 = one kernel launch per Gauss-Seidel colour, residual,
 * restriction and prolongation; 1 = a cluster level: its sweeps, residual and
 * restriction in one thread-block-cluster launch and its prolongation and
 * sweeps in another, rows split over the cluster's CTAs with halo copies in
 * distributed shared memory (the same arithmetic per row as path 0 with
 * one warp per row); 2 = inside the cluster tail (this level and all coarser ones in
 * one launch); 3 = the coarsest level (direct solve).  Errors: INVALID_ARG. */
gmg_status gmg_level_path(gmg_handle h, int l, int *path);
/* Copies level l's Galerkin operator A_l (CSR, caller numbering, rowptr n+1,
 * col/val nnz) and its colouring (n) into host buffers; any may be NULL. */
gmg_status gmg_level_export(gmg_handle h, int l, int64_t *rowptr, int32_t *col, double *val, int32_t *color);

/* ---- single steps of Alg. 2 on device vectors in the caller's numbering of
 * level l (FP64 arrays; with fp32 != 0 the step runs on the FP32 copy of the
 * level: inputs are rounded to FP32 and outputs widened back).  These are the
 * kernels the solve runs, exposed for step-by-step checks. ---- */

/* `nsweep` multicolour Gauss-Seidel sweeps on A_l x = b, colours ascending
 * (descending != 0: descending).  x is updated in place. */
gmg_status gmg_smooth(gmg_handle h, int l, int fp32, const double *b, double *x, int nsweep, int descending,
                      void *stream);
/* r = b - A_l x. */
gmg_status gmg_residual(gmg_handle h, int l, int fp32, const double *x, const double *b, double *r, void *stream);
/* bc = P_l^T r  (bc has n_{l+1} entries). */
gmg_status gmg_restrict(gmg_handle h, int l, int fp32, const double *r, double *bc, void *stream);
/* x += P_l u  (u has n_{l+1} entries). */
gmg_status gmg_prolong_add(gmg_handle h, int l, int fp32, const double *u, double *x, void *stream);
/* x = A_lambda^-1 b on the coarsest level (FP64 factor in both modes). */
gmg_status gmg_coarse_solve(gmg_handle h, int fp32, const double *b, double *x, void *stream);
/* One V-cycle x <- MGI(x, b, 1) of Alg. 2 on the finest level. */
gmg_status gmg_vcycle(gmg_handle h, int fp32, const double *b, double *x, void *stream);
/* One FP32 V-cycle X <- MGI(X, B, 1) of Alg. 2 applied to nrhs columns at
 * once, with the kernels gmg_solve_batched and gmg_solve_many run (each matrix
 * entry read once for all columns): B and X are device n x nrhs blocks,
 * row-major in the caller's numbering; X holds the initial iterates and is
 * overwritten.  Inputs are rounded to FP32; the coarsest solve accumulates in
 * FP64.  1 <= nrhs <= 16. */
gmg_status gmg_vcycle_batched(gmg_handle h, int nrhs, const double *B, double *X, void *stream);

/* The reciprocal 1/d that the coarsest inverse (Alg. 2's direct solve) takes
 * of each pivot, and the set-up of every level of 1/a_ii: from an FP32 seed
 * built from d's bits, one cubic Newton-Raphson step r0 (1 + e + e^2),
 * e = 1 - d r0.  Applied elementwise to n device values d (out: n device
 * values); exposed so that it can be checked against the correctly rounded
 * division (within one unit in the last place).  Values outside
 * [2^-100, 2^101) in magnitude take the FP64 division.
 * Errors: INVALID_ARG (n < 0, or a null pointer with n > 0). */
gmg_status gmg_pivot_reciprocal(int64_t n, const double *d, double *out, void *stream);

/* The precision conversions of the solver's kernels, done on the IEEE 754
 * bit patterns with integer operations: dir 0 narrows n device doubles `in`
 * to floats `out` (round to nearest even), dir 1 widens n device floats to
 * doubles (exact).  Exposed so that they can be checked against the IEEE 754
 * conversions.  Errors: INVALID_ARG (n < 0, dir not 0 or 1, or a null
 * pointer with n > 0). */
gmg_status gmg_convert(int64_t n, int dir, const void *in, void *out, void *stream);

/* Self-test of the bounded device-side wait (no counterpart in the paper).
 * The cluster-level kernels wait for their streamed matrix entries on an
 * mbarrier with a limit of polls, after which they set an error word that
 * gmg_solve reports as GMG_ERR_TIMEOUT, instead of hanging.  This runs that
 * wait, in one warp, on an mbarrier that nothing arrives on: *timed_out
 * receives 1 when the wait gave up (the expected outcome), *ms (may be NULL)
 * its device time.  polls <= 0 uses the limit of the solve kernels.  The
 * kernel returns normally, so the context stays usable.  Errors: INVALID_ARG
 * (null timed_out), OOM, CUDA. */
gmg_status gmg_wait_selftest(int polls, int *timed_out, double *ms, void *stream);

/* ---- allocation-free residual (no counterpart in the paper) ----
 * For callers that cannot allocate device memory (code running inside
 * another framework's memory pool, under an allocator that forbids
 * cudaMalloc, or where an allocation would synchronise the device): the
 * FP64 residual r = b - A x of a caller-owned CSR matrix and the norms
 * norms[0] = ||r||_2, norms[1] = ||b||_2, with no handle and no allocation.
 * All pointers are device pointers owned by the caller (rowptr n + 1,
 * col/val rowptr[n], x/b/r n, norms 2 doubles); results are ready when work
 * queued on `stream` completes.  The block partial sums live in a 1 MiB
 * static device array that every GPU loading the library keeps until the
 * process exits, so n is limited to 16,777,216 rows (GMG_ERR_TOO_LARGE
 * beyond).  The first call on a device looks up that array's device address
 * (with the device current): make it before any stream capture.  The address
 * is cached per device and CUDA context; after cudaDeviceReset (a new
 * context) the next call looks it up again, so that call too belongs before
 * any capture.  All calls
 * share the array, so calls that overlap on the GPU (other streams, or
 * other host threads on the same device) race and must be serialised by the
 * caller.  Sums run in a fixed order: repeated calls give identical bits. */
gmg_status gmg_residual_norm_noalloc(int64_t n, const int64_t *rowptr, const int32_t *col, const double *val,
                                     const double *x, const double *b, double *r, double *norms, void *stream);

#ifdef __cplusplus
}
#endif
#endif /* GMG_H */
