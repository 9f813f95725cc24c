/*
 * amg.h -- C ABI of libamg_gb: matching-aggregation algebraic multigrid as
 * the preconditioner of a right-preconditioned flexible GMRES solver, on one
 * NVIDIA GB300 (sm_103a).
 *
 * The method follows P. Kumar, "Aggregation based on graph matching and
 * inexact coarse grid solve for algebraic multigrid" (arXiv:1105.3468):
 *   - problem: A x = b, A in R^{N x N} sparse, x, b in R^N (Section 1,
 *     eq. (1); Algorithm 1, its title);
 *   - setup: aggregates from graph matching (Section 2), prolongation P with
 *     P_ij = 1 iff i in G_j (Section 2, definition of P and eq. (4)),
 *     Galerkin coarse matrix A_c = P^T A P (eq. (3) of Section 2 and its
 *     entrywise form), ILU(0) smoother S = L0 U0 (Algorithm 1, setup);
 *   - preconditioner B~ = (S^{-1} + M~^{-1} - M~^{-1} A S^{-1})^{-1} without
 *     post-smoothing, M~ = P A~_c P^T (eq. (5), Algorithm 1's preconditioner and coarse-solve
 *     applications);
 *   - Krylov accelerator: GMRES with Givens rotations (Algorithm 1), here
 *     the flexible right-preconditioned variant FGMRES(m).
 * Readings where the paper is silent (matching rule and tie-breaks, the
 * inexact coarse solve as Richardson steps preconditioned by the two-grid
 * construction of the coarse matrix, orderings, tolerances) are fixed by the
 * options below and described with each option.
 *
 * Conventions for every entry point
 *   - Return value: an AMG_* status code; nothing is thrown across the ABI.
 *     amg_last_error() returns a message for the calling thread's last
 *     failure.
 *   - Pointers: "host or device" arguments may be ordinary host memory,
 *     pinned host memory or device memory of the current CUDA device; the
 *     library detects the kind and copies as needed.  "device" arguments
 *     must be device memory.  The caller owns every buffer it passes;
 *     nothing the caller passes is retained after the call returns, except
 *     the stream given to amg_setup.
 *   - Streams: all work of a handle is ordered on the stream given to
 *     amg_setup (NULL = the legacy default stream).  Calls that return host
 *     results synchronise that stream before returning.
 *   - Index types: row pointers int64 at the ABI (internally int32: the
 *     library rejects nnz >= 2^31 with AMG_ERR_INVALID_ARG); column indices
 *     int32, strictly ascending within each row; every row must store its
 *     diagonal entry.
 *   - Determinism: every reduction has a fixed order, so repeated calls on
 *     the same inputs give bit-identical results.
 */
#ifndef AMG_GB_H
#define AMG_GB_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---------------------------------------------------------------- status */
#define AMG_OK 0
#define AMG_ERR_INVALID_ARG 1   /* bad CSR, null pointer, bad option      */
#define AMG_ERR_CUDA 2          /* a CUDA runtime call failed             */
#define AMG_ERR_OOM 3           /* device allocation failed               */
#define AMG_ERR_NOT_SUPPORTED 4 /* valid request outside what is built    */
#define AMG_ERR_BREAKDOWN 5     /* zero or non-finite pivot in a factor   */
#define AMG_ERR_NUMERIC 6       /* NaN/Inf in a residual or a norm        */
#define AMG_ERR_NOT_CONVERGED 7 /* maxit reached; x holds the last iterate */
#define AMG_ERR_LIMIT 8         /* a bounded device loop hit its cap      */

/* V-cycle arithmetic (FGMRES itself always runs in FP64). */
#define AMG_FP64 0              /* all FP64                                */
#define AMG_FP32 1              /* FP32 storage and arithmetic             */
#define AMG_BF16 2              /* as FP32, with the finest level's ILU(0)
                                   factors stored in BF16                 */
#define AMG_BF16_ALL 3          /* as FP32, with the ILU(0) factors of every
                                   smoothed level stored in BF16 (residuals
                                   and coarse matrices stay FP32)         */

/* Elimination order of the ILU(0) factors of one level. */
#define AMG_ORDER_COLOR 0       /* colour-major (rows of a colour are independent) */
#define AMG_ORDER_NATURAL 1     /* row index order, the paper's GMG-NO (Section 3) */

/* Colouring priority used by AMG_ORDER_COLOR. */
#define AMG_COLOR_HASH_JP 0     /* priority (mix64(i ^ (seed + 0x9e3779b97f4a7c15)), i) */
#define AMG_COLOR_FIRST_FIT 1   /* priority -i (first fit in index order)  */

/* Edge weight of the heavy-edge matching (amg_options_t.match_weight). */
#define AMG_MATCH_PLAIN 0       /* w_uv = (|a_uv| + |a_vu|)/2              */
#define AMG_MATCH_SCALED 1      /* the same divided by sqrt(|a_uu| |a_vv|) */

/* Coarse solve of level 1 (amg_options_t.coarse_solver). */
#define AMG_COARSE_RECURSIVE 0  /* coarse_inner Richardson steps, each
                                   preconditioned by the same two-grid
                                   construction on the coarse level        */
#define AMG_COARSE_ILUT 1       /* the paper's two-grid form: level 1 is the
                                   last level, factored once by ILUT(ilut_tau)
                                   (Section 2) and solved with its factors  */

/* Driver of the FGMRES loop (amg_options_t.solve_loop). */
#define AMG_LOOP_HOST 0
#define AMG_LOOP_DEVICE 1

/* Orthogonalisation of the outer FGMRES (Arnoldi process). */
#define AMG_ORTHO_MGS 0         /* modified Gram-Schmidt                   */
#define AMG_ORTHO_CGS2 1        /* classical Gram-Schmidt, two passes      */

typedef struct amg_handle amg_handle_t;

/* A square sparse matrix in CSR form (Section 1: A in R^{N x N}). */
typedef struct {
    int32_t n;                /* rows = columns, n >= 1                    */
    int64_t nnz;              /* stored entries = row_ptr[n]               */
    const int64_t *row_ptr;   /* [n+1], row_ptr[0] = 0, non-decreasing     */
    const int32_t *col;       /* [nnz], ascending within a row, in [0, n)  */
    const double *val;        /* [nnz] FP64                                */
} amg_csr_t;

typedef struct {
    /* coarsening: each level is aggregated by `passes` heavy-edge matching
     * passes (aggregates of at most 2^passes points; Section 2 aggregation
     * by graph matching).  Matching rule: greedy maximal matching in
     * decreasing key order, key = (w_uv, mix64(((u<<32)|v) ^ seed), u, v),
     * u < v, edges with w > 0; w_uv = (|a_uv| + |a_vu|)/2 divided by
     * sqrt(|a_uu| |a_vv|) (match_weight = AMG_MATCH_SCALED), or not divided
     * (AMG_MATCH_PLAIN). */
    int32_t passes;           /* default 2                                 */
    int32_t coarse_inner;     /* Richardson steps solving level 1: 5       */
    int32_t deep_inner;       /* Richardson steps on levels >= 2: 1        */
    int32_t dense_max;        /* a level with <= dense_max rows is the last
                                 one and is solved exactly (its FP64
                                 inverse, one warp per row): 0..4096,
                                 default 4096                               */
    int32_t max_levels;       /* 2..24, default 12                         */
    int32_t order_fine;       /* ILU(0) order of level 0: AMG_ORDER_NATURAL */
    int32_t order_coarse;     /* ILU(0) order of levels >= 1: AMG_ORDER_COLOR */
    int32_t coloring;         /* AMG_COLOR_HASH_JP                         */
    int32_t restart;          /* FGMRES restart length m: 30               */
    int32_t maxit;            /* total inner iterations cap: 600           */
    int32_t vcycle_prec;      /* AMG_FP64 / AMG_FP32 / AMG_BF16 /
                                 AMG_BF16_ALL: AMG_FP64                    */
    int32_t build_adjoint;    /* nonzero: also build transposed structures */
    int32_t use_graphs;       /* nonzero: replay the inner iteration as a CUDA
                                 graph captured once per handle: 1          */
    int32_t persistent;       /* ILU(0) smoother schedule.  0: one launch per
                                 schedule level.  1: an application with
                                 more than 16 schedule levels (forward +
                                 backward) is one kernel: one block or one
                                 cluster with both solve vectors in shared
                                 memory when they fit, else a cooperative
                                 grid with a bounded grid barrier between
                                 levels.  2: every application is one
                                 cooperative kernel in which each row
                                 starts when the rows it reads are written
                                 (no level barriers; bounded waits).  3:
                                 dataflow on the finest level only, as 1
                                 elsewhere.  4: dataflow on every level too
                                 large for the shared-memory kernel.  5:
                                 as 3, but a finest level in natural order
                                 whose matrix is a 5-point (2D) or 7-point
                                 (3D) grid stencil (detected from the
                                 pattern) is solved in grid tiles: one
                                 block per 16^3 (64^2) tile with the tile's
                                 wavefronts in shared memory, only the
                                 faces between tiles through global memory
                                 (amg_get_tile_grid reports the tiling).
                                 All six give bit-identical results.  A
                                 wait that gives up returns AMG_ERR_LIMIT.
                                 Default: 5                                 */
    int32_t deep_block_max;   /* levels >= 2 with at most this many rows (and
                                 all levels below them) run their V-cycle in
                                 one thread block when deep_inner == 1;
                                 0 disables (default: measured slower)      */
    int32_t orthog;           /* Arnoldi orthogonalisation of the outer
                                 FGMRES: AMG_ORTHO_MGS (modified Gram-
                                 Schmidt, one cooperative kernel per
                                 column) or AMG_ORTHO_CGS2 (classical
                                 Gram-Schmidt with one re-orthogonalisation
                                 pass): AMG_ORTHO_MGS                      */
    int32_t spmv_block;       /* threads per block of the outer FP64 SpMV:
                                 64/128/256/512, or 0 = autotuned at setup */
    int32_t spmv_unroll;      /* unroll depth of its column loop: 2/4/8, or
                                 0 = autotuned at setup.  Neither changes
                                 the result (rows are summed in the same
                                 order by every variant): 0                 */
    int32_t dot2;             /* Arnoldi inner products and norms as if in
                                 twice the working precision (Dot2, Ogita-
                                 Rump-Oishi 2005), independent of the
                                 reduction order: 1 on, 0 plain FMA sums,
                                 -1 = on with the FP64 V-cycle only: -1    */
    int32_t match_weight;     /* AMG_MATCH_SCALED: the coupling measured
                                 against its endpoints' diagonals, so a
                                 vertex left unmatched on one level is not
                                 outweighed forever by its growing
                                 neighbours (default); AMG_MATCH_PLAIN:
                                 the coupling alone                        */
    uint64_t seed;            /* tie-break seed, default 0                 */
    int32_t coarse_solver;    /* AMG_COARSE_RECURSIVE (default) or
                                 AMG_COARSE_ILUT                           */
    int32_t solve_loop;       /* AMG_LOOP_DEVICE: the FGMRES loop runs as one
                                 CUDA graph with conditional nodes (all
                                 members of a batch in one graph), the host
                                 reads the state once at the end; used when
                                 use_graphs is on and no kernel class is
                                 timed (default).  AMG_LOOP_HOST: the host
                                 reads the stop flag after every inner
                                 iteration.  Both give the same bits.      */
    double ilut_tau;          /* drop tolerance of AMG_COARSE_ILUT (the
                                 factorisation of amg_ilut_host): >= 0,
                                 default 1e-6                               */
} amg_options_t;

typedef struct {
    int32_t status;           /* same as the call's return value           */
    int32_t iters;            /* inner FGMRES iterations                   */
    int32_t restarts;
    int32_t nlevels;
    double rel_res_true;      /* ||b - A x|| / ||b|| in FP64 at return      */
    double setup_ms;          /* wall time of amg_setup                    */
    double solve_ms;          /* wall time of the solve call               */
    int32_t n_coarse;         /* rows of level 1                           */
    int32_t n_colors;         /* colours (or DAG levels) of level 0 sweeps */
    int64_t nnz_coarse;       /* stored entries of level 1                 */
    int64_t kernel_launches;  /* kernels this call launched (graph replays count their nodes) */
} amg_stats_t;

/* ------------------------------------------------------------ basics */
const char *amg_status_string(int status);
const char *amg_last_error(void);
/* Fills *opt with the defaults listed above.  Returns AMG_OK, or
 * AMG_ERR_INVALID_ARG for a NULL pointer. */
int amg_default_options(amg_options_t *opt);

/* --------------------------------------------------------------- setup */
/* Builds the hierarchy for A (Algorithm 1, setup): per level the
 * matching passes, aggregates, Galerkin products, the ILU(0) factors in the
 * chosen order, and the dense inverse of the last level; then the FP32/BF16
 * copies and, if requested, the transposed structures.  A's arrays are host
 * or device; they are copied.  `stream` is a cudaStream_t (NULL allowed).
 * Errors: AMG_ERR_INVALID_ARG (bad CSR: unsorted or out-of-range columns,
 * missing diagonal, nnz >= 2^31; bad option), AMG_ERR_BREAKDOWN (zero ILU(0),
 * ILUT or dense pivot), AMG_ERR_LIMIT (matching/colouring rounds or a coarse row
 * over its capacity), AMG_ERR_OOM, AMG_ERR_CUDA.  On error *out is NULL. */
int amg_setup(const amg_csr_t *A, const amg_options_t *opt, void *stream,
              amg_handle_t **out);

/* New values for the matrix of an existing handle, with the same sparsity
 * pattern (val: nnz doubles in the pattern's order, host or device).  The
 * aggregation of every level (all matching results) is kept; everything
 * numeric is recomputed from the new values: the Galerkin products (eq. (3)),
 * the ILU(0) factors, the dense last level, the precision copies and the
 * transposes.  Equivalent to amg_setup on the new values with the
 * aggregation frozen, so repeated solves with changing coefficients (an
 * optimisation loop over the adjoint gradient) skip the matching.  If the
 * update fails the handle keeps its previous hierarchy.
 * Errors: AMG_ERR_INVALID_ARG (null, batched handle), AMG_ERR_BREAKDOWN
 * (a zero pivot in the new factors), AMG_ERR_OOM, AMG_ERR_CUDA. */
int amg_update_values(amg_handle_t *h, const double *val);

/* Releases everything the handle owns.  NULL is allowed. */
void amg_destroy(amg_handle_t *h);

/* ILUT(tau) of a HOST CSR matrix, computed on the host: the inexact coarse
 * factorisation A~_c = L~_c U~_c = ILUT(A_c) of Section 2 (Algorithm 1
 * setup), with the dropping rule of Saad's ILUT (tau_i = tau * ||a_i||_2; an
 * entry of L~ is dropped when |a_ik / u_kk| < tau_i, one of U~ when it is
 * below tau_i; the diagonal is always kept; no cap per row), no pivoting,
 * natural order.  tau = 0 keeps every nonzero (the complete LU without
 * pivoting).  row_ptr [n+1] / col / val: sorted columns, diagonal present.
 * Output, in caller-owned host arrays: f_row_ptr [n+1] and f_col / f_val
 * [cap], row i holding its L~ part (unit diagonal implied) then its U~ part,
 * ascending columns; *f_nnz receives the number of stored entries.
 * Errors: AMG_ERR_INVALID_ARG (null pointer, n < 0, tau < 0 or NaN, bad CSR),
 * AMG_ERR_LIMIT (cap < *f_nnz: nothing written but *f_nnz; call again with
 * cap >= *f_nnz), AMG_ERR_BREAKDOWN (a zero or non-finite u_ii; the factors
 * are still written), AMG_ERR_OOM.  Needs no GPU. */
int amg_ilut_host(int32_t n, const int64_t *row_ptr, const int32_t *col, const double *val, double tau,
                  int64_t cap, int64_t *f_row_ptr, int32_t *f_col, double *f_val, int64_t *f_nnz);

/* --------------------------------------------------------------- solve */
/* Solves A x = b by FGMRES(restart) preconditioned with B~ (Algorithm 1,
 * Krylov iteration), stopping when the true relative residual
 * ||b - A x|| / ||b|| <= tol (Section 3 stopping rule).  b: host or device
 * [n]; x: host or device [n], read as the initial guess, written with the
 * result.  stats may be NULL.  The loop runs on the device (solve_loop) unless
 * a kernel class is timed.  Returns AMG_ERR_NOT_CONVERGED when maxit is
 * reached (x holds the last iterate), AMG_ERR_NUMERIC for NaN/Inf,
 * AMG_ERR_LIMIT when a bounded device wait gave up. */
int amg_solve(amg_handle_t *h, const double *b, double *x, double tol, amg_stats_t *stats);

/* Solves the adjoint system A^T lambda = g by FGMRES preconditioned with
 * B~^{-T} = S^{-T}(I - A^T P C^T P^T) + P C^T P^T, the transpose of the
 * preconditioner (coarse correction first, then the transposed smoother).
 * Needs build_adjoint.  g, lambda: host or device [n]; lambda is read as
 * the initial guess.  Errors as amg_solve. */
int amg_adjoint(amg_handle_t *h, const double *g, double *lambda, double tol, amg_stats_t *stats);

/* ------------------------------------------------------------- batches */
/* Sets up `count` independent systems (the batched path): one hierarchy per
 * system, built concurrently from 8 host threads, each system on its own
 * internal stream (setup memory comes from the library's stream-ordered pool,
 * so the setups do not synchronise one another).  The per-system results are those amg_setup gives for
 * that system alone.  systems: host array of `count` CSR descriptors (their
 * arrays host or device).  Errors as amg_setup, the message naming the
 * first failing system; nothing is kept on error. */
int amg_setup_batched(const amg_csr_t *systems, int32_t count, const amg_options_t *opt, void *stream,
                      amg_handle_t **out);
/* Solves every system of a batched handle: b_cat and x_cat (host or device)
 * hold the systems' vectors back to back, at the offsets amg_batch_size
 * reports.  With solve_loop = AMG_LOOP_DEVICE (default) every system's
 * FGMRES loop is one root chain of a single CUDA graph (conditional nodes;
 * each system's done flag lives in device memory), so the whole batch is one
 * graph launch and one synchronisation, built on the first call and replayed
 * afterwards.  With AMG_LOOP_HOST one host loop advances all systems: each
 * active system queues one inner iteration (a graph replay on its stream),
 * then each is collected; a converged or failed system drops out.
 * per_system (host, may be NULL) receives `count` stats.  Returns the first
 * error, else AMG_ERR_NOT_CONVERGED if any system hit maxit, else AMG_OK.
 * Each system's iterates are exactly those of amg_solve on that system
 * alone, with either loop. */
int amg_solve_batched(amg_handle_t *h, const double *b_cat, double *x_cat, double tol,
                      amg_stats_t *per_system);
/* Number of systems and their row offsets (host, count + 1 entries; may be
 * NULL) of a batched handle; count = 0 for a single-system handle. */
int amg_batch_size(amg_handle_t *h, int32_t *count, int64_t *offsets);
/* The handle of system k of a batch (owned by the batch; for introspection
 * calls such as amg_get_history), or NULL. */
amg_handle_t *amg_batch_member(amg_handle_t *h, int32_t k);

/* Residual history of the last solve or adjoint call: entry 0 is
 * ||r0||/||b||, then one FGMRES estimate |s_{j+1}|/||b|| per inner
 * iteration.  out: host [cap]; *len receives the full length. */
int amg_get_history(amg_handle_t *h, double *out, int32_t cap, int32_t *len);

/* q = B~^{-1} z (transpose = 0) or B~^{-T} z (transpose = 1) at level 0, in
 * the handle's V-cycle precision with FP64 input and output (Algorithm 1,
 * preconditioner application).  z, q: device [n]. */
int amg_precond_apply(amg_handle_t *h, const double *z, double *q, int32_t transpose);

/* y = A x in FP64 for a CSR given on the device (row_ptr int64).  x, y:
 * device [n].  Synchronises `stream`.  Errors: AMG_ERR_INVALID_ARG for a
 * null pointer, nnz >= 2^31, row pointers that are not a non-decreasing
 * sequence from 0 to nnz, or columns outside [0, n) (no out-of-range entry
 * is ever used as an index: y is then unspecified); AMG_ERR_CUDA. */
int amg_spmv(const amg_csr_t *A, const double *x, double *y, void *stream);

/* y = A x like amg_spmv, for callers that must not let the library allocate
 * device memory: a process whose own caching allocator has reserved the free
 * device memory up front (a library cudaMalloc would fail or eat into its
 * budget), or a loop that must not stall the device (cudaFree synchronises
 * the whole device).  The int32 row-pointer copy that amg_spmv allocates per
 * call lives instead in a fixed file-scope device array of
 * AMG_NOALLOC_MAX_ROWS + 1 entries plus a status word (16 MiB + 512 B), held
 * by every GPU that loads the library until the process exits.  The paper
 * has no counterpart: this is an interface variant only.  Pointers as in
 * amg_spmv (device).  The first call on a device looks up the array's
 * address with that device current.  Every call shares the array, so calls
 * that overlap on the GPU race: serialise them on one stream.  Synchronises
 * `stream`.  Errors: AMG_ERR_INVALID_ARG for n > AMG_NOALLOC_MAX_ROWS,
 * nnz >= 2^31, null pointers, row pointers that are not a non-decreasing
 * sequence from 0 to nnz, or columns outside [0, n) (no out-of-range entry
 * is ever used as an index); AMG_ERR_CUDA. */
#define AMG_NOALLOC_MAX_ROWS 4194304
int amg_spmv_noalloc(const amg_csr_t *A, const double *x, double *y, void *stream);

/* ------------------------------------------------------- introspection */
/* Level l facts: info[0] rows, [1] stored entries, [2] sweep levels of the
 * forward ILU(0) solve (colours in colour order), [3] 1 if dense final
 * level, [4] rows after the first matching pass (-1 if none), [5] rows of
 * the next level (-1 if last), [6] colours (0 in natural order),
 * [7] sweep levels of the backward solve.  info: host [8]. */
int amg_get_level_info(amg_handle_t *h, int32_t level, int64_t *info);
/* Grid tiling of the finest level's smoother (persistent = 5): info[0] 1 when
 * the finest level is solved in grid tiles, else 0 (and the rest 0);
 * [1..3] the detected grid nx, ny, nz (nz = 1 in 2D); [4..6] the tile
 * extents; [7] the number of tiles.  info: host [8].  AMG_ERR_INVALID_ARG
 * for a null argument or a batched handle. */
int amg_get_tile_grid(amg_handle_t *h, int64_t *info);
/* The smoother variant of level l's last application, kind[0] for S^{-1}
 * and kind[1] for S^{-T} (-1: not applied yet): 0 one launch per schedule
 * level, 1 one block, 2 a grid of up to 8 blocks run as one cluster, 3
 * cooperative grid with grid barriers, 4 one cluster with both solve
 * vectors replicated in every CTA's shared memory, 5 dataflow solve, 6 grid
 * tiles.  kind: host [2].  Which variant runs depends on the persistent
 * option and the level's size; all give the same bits. */
int amg_get_sweep_kind(amg_handle_t *h, int32_t level, int32_t *kind);
int amg_num_levels(amg_handle_t *h, int32_t *nlevels);

/* Launch geometry the outer SpMV of h uses (picked by the autotuner unless
 * fixed by the options).  No counterpart in the paper.  block, unroll: host. */
int amg_get_spmv_config(amg_handle_t *h, int32_t *block, int32_t *unroll);

/* Aggregate map of level l: pass 0 = composite map to level l+1 (rows of
 * level l), pass p >= 1 = map of matching pass p.  out: host. */
int amg_get_aggregates(amg_handle_t *h, int32_t level, int32_t pass, int32_t *out);

/* Matrix of level l (level 0 = A as stored) in CSR: rp [n+1], col [nnz],
 * val [nnz]; all host.  Level l >= 1 is the Galerkin product. */
int amg_get_matrix(amg_handle_t *h, int32_t level, int64_t *rp, int32_t *col, double *val);

/* Intermediate Galerkin product after matching pass p (1 <= p < passes) of
 * level l: sizes via info[0] rows / info[1] nnz when rp == NULL. */
int amg_get_pass_matrix(amg_handle_t *h, int32_t level, int32_t pass, int64_t *info,
                        int64_t *rp, int32_t *col, double *val);

/* Colour (AMG_ORDER_COLOR) or 0 (natural) per row of level l.  host. */
int amg_get_colors(amg_handle_t *h, int32_t level, int32_t *out);

/* FP64 ILU(0) factors of level l on that level's CSR layout: L entries
 * (unit diagonal implied) before the row in the elimination order, U
 * entries (with the diagonal) after.  out: host [nnz].  AMG_ERR_INVALID_ARG
 * on the dense level and on the ILUT level of AMG_COARSE_ILUT (its factors
 * have their own pattern: amg_ilut_host computes the same factors). */
int amg_get_ilu(amg_handle_t *h, int32_t level, double *out);

/* ------------------------------------------------------------ profiling */
/* Times one kernel class with CUDA events on the handle's stream (for a
 * roofline figure measured while solving): 0 off, 1 the outer FP64 SpMV
 * w = A z_j, 2 every ILU(0) smoother application (forward + backward
 * solve) on every level, 3 the orthogonalisation of one column (the MGS
 * kernel, or the first CGS2 pass).  Setting
 * a class clears the totals.  No effect on results.  Errors:
 * AMG_ERR_INVALID_ARG. */
int amg_set_kernel_timing(amg_handle_t *h, int32_t kclass);
/* Totals since the class was set: summed event time (ms), timed launches,
 * and the algorithmic bytes those launches move (each array counted once per
 * launch).  Synchronises the stream. */
int amg_get_kernel_timing(amg_handle_t *h, double *ms_total, int64_t *launches, double *bytes_total);
/* Kernels the library has launched from the calling thread so far. */
int64_t amg_launch_counter(void);

/* ------------------------------------------------------------ FV input */
/* Cell-centred finite-volume matrix of eq. (2) (Section 1) on an
 * nx x ny (x nz) grid of [0,1]^dim, h = 1/nx: two-point diffusive fluxes
 * with the harmonic mean of the face-normal conductivities, first-order
 * upwind convection, u = 0 on y = 0 and y = 1 (Dirichlet, half-cell
 * distance), du/dn = 0 elsewhere (zero-gradient ghost, the outward flux
 * goes to the diagonal).  Faces are visited W, E, S, N, B, T; columns come
 * out ascending.  All pointers device.  kx/ky/kz [N] conductivity
 * components per cell; fx [(nx+1) ny nz], fy [nx (ny+1) nz], fz
 * [nx ny (nz+1)] integrated face fluxes (+axis direction); f [N] source.
 * Outputs row_ptr [N+1] (int64), col/val with room for (2 dim + 1) N
 * entries, b [N] = f h^dim; *nnz_out (host) receives nnz.  Synchronises
 * the stream.  Errors: AMG_ERR_INVALID_ARG for bad sizes. */
int amg_fv_assemble(int32_t dim, int32_t nx, int32_t ny, int32_t nz,
                    const double *kx, const double *ky, const double *kz,
                    const double *fx, const double *fy, const double *fz,
                    const double *f, int64_t *row_ptr, int32_t *col, double *val,
                    double *b, int64_t *nnz_out, void *stream);

/* Gradient of a loss L(x) with respect to log kx, log ky, log kz per cell
 * given lambda = A^{-T} dL/dx and x: dL/dA_ij = -lambda_i x_j restricted to
 * the diffusive transmissibilities (interior T = h^(d-2) 2 kP kN/(kP+kN),
 * dT/dlog kP = T kN/(kP+kN); Dirichlet T = h^(d-2) 2 kP, dT/dlog kP = T).
 * All pointers device; gz unused (may be NULL) in 2D. */
int amg_fv_grad_logk(int32_t dim, int32_t nx, int32_t ny, int32_t nz,
                     const double *kx, const double *ky, const double *kz,
                     const double *lambda, const double *x,
                     double *gx, double *gy, double *gz, void *stream);

/* The same assembly for an isotropic conductivity given by its logarithm:
 * kappa = exp(logk) per cell is computed on the device into `kappa` (device
 * [n], reused by amg_fv_grad_logk_iso), then eq. (2) is assembled with
 * kx = ky = kz = kappa.  Other arguments and errors as amg_fv_assemble. */
int amg_fv_assemble_logk(int32_t dim, int32_t nx, int32_t ny, int32_t nz, const double *logk, double *kappa,
                         const double *fx, const double *fy, const double *fz, const double *f,
                         int64_t *row_ptr, int32_t *col, double *val, double *b, int64_t *nnz_out,
                         void *stream);

/* dL/dlog kappa per cell for an isotropic conductivity (kx = ky = kz =
 * kappa): the derivative of amg_fv_grad_logk summed over the axes in the
 * order (x + y) + z, in one kernel.  All pointers device [n]; g is written. */
int amg_fv_grad_logk_iso(int32_t dim, int32_t nx, int32_t ny, int32_t nz, const double *kappa,
                         const double *lambda, const double *x, double *g, void *stream);

/* Gradient of a loss with respect to the stored values of A for A x = b:
 * grad_val[k] = -lambda[row_k] * x[col_k] with lambda = A^{-T} dL/dx (the
 * implicit-function derivative of the solve; dL/db = lambda).  All device
 * pointers; A's arrays as in amg_csr_t.  Stream-ordered, no synchronisation. */
int amg_csr_value_grad(const amg_csr_t *A, const double *lambda, const double *x, double *grad_val,
                       void *stream);

/* ------------------------------------------------------------- version */
const char *amg_version(void);

#ifdef __cplusplus
}
#endif
#endif /* AMG_GB_H */
