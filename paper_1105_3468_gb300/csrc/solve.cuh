// solve.cuh -- declarations of the solve-phase kernels' host launchers and
// the device-resident FGMRES state.
#pragma once

#include "internal.cuh"

namespace amg {

// Largest restart length supported by the fused multi-dot kernels.
constexpr int KMAX1 = 32;

// FGMRES scalars, resident in device memory and updated by single-thread
// kernels (Givens, back substitution) so that the inner loop needs no host
// round trip except the stop flag.
struct FgState {
    int m, maxit, total, hist_len, hist_cap, jdone, stop, status;
    int j, pad_i;                           // current inner column
    double tol, bnorm, hn, pad;           // hn = h_{j+1,j} of the last column
    double H[(KMAX1 + 1) * KMAX1];
    double cs[KMAX1], sn[KMAX1], s[KMAX1 + 1], y[KMAX1];
    double h1[KMAX1 + 1], h2[KMAX1 + 1], nrm2[2];
    // device-driven solve loop (graph conditional nodes): done ends the
    // loop; relres = true residual of the last cycle end; passes counts loop
    // bodies, capped at loop_cap
    int done, restarts, passes, loop_cap;
    double relres, pad2;
    double *hist;
};

// Matrix view for a level in value type V.
template <typename V>
struct LevelMats {
    int n, nnz;
    const int *rp, *ci;
    const V *v;
};

// Sweep view in vector type T and value type V.
template <typename T, typename V>
struct SweepView {
    int nlev;
    const int *lev_ptr;   // host
    const int *dlev;      // device copy
    const int *rows, *rp, *ci;
    const V *v;
    const T *d;           // diagonal per schedule position (or nullptr)
};

void spmv_f64(int n, int nnz, const int *rp, const int *ci, const double *v, const double *x, double *y, cudaStream_t s);
void spmv_f64_checked(int n, int nnz, const int *rp, const int *ci, const double *v, const double *x, double *y,
                      int *bad, cudaStream_t s);
void spmv_f64_xf32(int n, int nnz, const int *rp, const int *ci, const double *v, const float *x, double *y, cudaStream_t s);
void residual_f64(int n, int nnz, const int *rp, const int *ci, const double *v, const double *x, const double *b,
                  double *r, cudaStream_t s);

// y = A x (mode 0) or y = b - A x (mode 1) on the SELL-32 copy; each row is
// summed sequentially in column order.
template <typename XT>
void sell_spmv(int n, int nslices, const int64_t *ptr, const int *ci, const double *v, const XT *x, const double *b,
               double *y, int mode, cudaStream_t s, int block = 256, int unroll = 4);

template <typename T, typename V>
void level_residual(const LevelMats<V> &M, const T *x, const T *b, T *r, cudaStream_t s);
// The same from a SELL-32 copy (each row summed in stored order).
template <typename T, typename V>
void level_residual_sell(int n, const int64_t *ptr, const int *ci, const V *v, const T *x, const T *b, T *r,
                         cudaStream_t s);
template <typename T, typename V>
void sweep(const SweepView<T, V> &S, const T *in, T *out, int with_diag, cudaStream_t s);
// Both triangular solves of one smoother application in one cooperative
// launch: y = F^{-1} in (schedule levels of F), out = B^{-1} y, with a
// bounded grid barrier between levels.  bar: 2 device words (zeroed), err:
// device word set when a barrier wait gives up.
// Returns the variant that ran (SWEEP_KIND_*).
template <typename T, typename V>
int sweep_pair_coop(const SweepView<T, V> &F, int f_diag, const SweepView<T, V> &B, int b_diag, const T *in,
                    T *y, T *out, unsigned int *bar, int *err, cudaStream_t s);
// Smoother variants, as amg_get_sweep_kind reports them.
constexpr int SWEEP_KIND_LEVELS = 0;            // one launch per schedule level
constexpr int SWEEP_KIND_BLOCK = 1;             // one block, block barrier
constexpr int SWEEP_KIND_CLUSTER_GRID = 2;      // a grid of <= 8 blocks run as one cluster
constexpr int SWEEP_KIND_GRID = 3;              // cooperative grid, grid barrier
constexpr int SWEEP_KIND_DSM_REPLICATED = 4;    // one cluster, vectors replicated in every CTA's shared memory
constexpr int SWEEP_KIND_DATAFLOW = 5;          // cooperative dataflow solve
constexpr int SWEEP_KIND_TILES = 6;             // grid tiles (finest level, natural-order stencil)
template <typename T, typename V>
void sweep_pair_df(const SweepView<T, V> &F, int f_diag, const SweepView<T, V> &B, int b_diag, const T *in, T *y,
                   T *out, unsigned int *bar, int *err, cudaStream_t s);
template <typename T> void fill_sentinel(T *x, size_t n, cudaStream_t s);
// Grid-tiled triangular solves of a natural-order 5-point (2D) or 7-point
// (3D) stencil level (tiles.cu).  Tiles of tx x ty x tz rows (powers of two);
// step coordinates of a row are its local coordinates in its tile, reversed
// for the backward solve.
struct TileGeom {
    int dim, nx, ny, nz;          // grid (nz = 1 in 2D)
    int tx, ty, tz, lx, ly;       // tile extents, log2 tx, log2 ty
    int ntx, nty, ntz, ntiles;    // tiles per axis, total
    int tv, nd, fs, ne, nq;       // rows per tile, steps per tile, mailbox face stride, halo entries, axes
};
// One triangular solve's factor values in tile layout: c [ntiles][nq][tv]
// (slot q: the q-th neighbour the row consumes), d [ntiles][tv] the diagonal
// (empty when the solve has none); position within a tile = local index
// (i + tx (j + ty k)) in step coordinates.
struct TileFactor {
    DBuf<char> c, d;
};
struct TilePlan {
    TileGeom g{};
    size_t tsz = 0, vsz = 0;      // vector and factor value sizes the plan is built for
    DBuf<int> hwoff;              // [nd + 1] first halo entry of each step
    DBuf<unsigned int> hent;      // [ne] halo entries: face | step << 2 | a << 12 | b << 22
    DBuf<int> torder;             // [ntiles] tiles by anti-diagonal
    DBuf<char> mb[2];             // mailboxes [ntiles][3][fs] of the forward and backward phases
    TileFactor fwd, bwd, fwdT, bwdT;
    int blocks = 0;               // cooperative grid of the tile kernel (tile_prepare)
};
// Detects the grid of a natural-order stencil matrix and builds the plan's
// geometry, tables and mailboxes; false (plan untouched) when the matrix's
// lower offsets do not describe a 2D / 3D grid.  The factor build verifies
// every row against the stencil.
bool tile_plan_build(const DCsr &A, TilePlan &P, size_t tsz, size_t vsz, cudaStream_t s);
void tile_mailbox_reset(TilePlan &P, cudaStream_t s);
// S in tile layout (mirror: the backward solve); false when a row's stored
// entries are not its stencil neighbours in ascending column order.
template <typename T, typename V>
bool tile_factor_build(const TilePlan &P, const SweepView<T, V> &S, bool mirror, TileFactor &F, cudaStream_t s);
// Kernel attributes and the co-resident grid for this plan's layout.
template <typename T, typename V> void tile_prepare(TilePlan &P);
// y = F^{-1} in, out = B^{-1} y: one cooperative launch, a grid barrier
// between the two solves; err set when a bounded wait gave up.
template <typename T, typename V>
void sweep_pair_tiles(const TilePlan &P, const TileFactor &F, const TileFactor &B, const T *in, T *y, T *out,
                      unsigned int *bar, int *err, cudaStream_t s);
// True when a level's two solve vectors (elem bytes per row each) and its
// level pointers fit the shared-memory sweep kernel.
bool sweep_fits_dsm(int n, int nlev_f, int nlev_b, size_t elem);
template <typename T>
void restrict_to(int nc, const int *mptr, const int *midx, const T *r, T *h, cudaStream_t s);
template <typename T, typename Q>
void prolong(int n, const int *agg, const T *t, const T *g, Q *q, int mode, cudaStream_t s);
template <typename T>
void vec_acc(size_t n, const T *in, T *out, int mode, cudaStream_t s);
void convert_f64_f32(size_t n, const double *in, float *out, cudaStream_t s);
void convert_f32_f64(size_t n, const float *in, double *out, cudaStream_t s);
// dot2: each row as an inner product as if in twice the working precision
template <typename T>
void dense_solve(int n, const double *inv, const T *h, T *g, int transpose, int mode, bool dot2, cudaStream_t s);
// The same from an FP32 copy of the inverse, accumulated in FP32 (the FP32 /
// BF16 V-cycles).
void dense_solve_f32(int n, const float *inv, const float *h, float *g, int transpose, cudaStream_t s);

// K = st->j + 1 basis vectors (read on the device)
// Smoothers with more schedule levels than this (forward + backward) run as
// one cooperative launch when the persistent option is on.
constexpr int PERSISTENT_MIN_LEVELS = 16;

// One level of the single-block V-cycle (deep levels, one Richardson step
// per level): g_m = S_m^{-1} h_m + P g_{m+1}, h_{m+1} = P^T (h_m - A_m S_m^{-1} h_m);
// the last level is solved by its dense inverse or by S^{-1} alone.
template <typename T, typename V>
struct DeepLevel {
    int n, dense, has_child, pad;
    const int *rp, *ci;
    const V *v;
    SweepView<T, V> fwd, bwd;
    const double *inv;
    const int *agg, *mptr, *midx;
    T *h, *g, *t, *y, *r;
};

template <typename T, typename V>
void deep_vcycle(const DeepLevel<T, V> *levels, int count, cudaStream_t s);

void mdot(size_t n, const FgState *st, const double *w, const double *V, size_t ldv, double *partials,
          unsigned int *ticket, double *h, cudaStream_t s);
// Modified Gram-Schmidt for column j = st->j in one cooperative launch:
// h1[k] = (w, v_k) with w updated after each k, h2[k] = 0, nrm2[0] = ||w||^2.
// partials: >= 2 x grid doubles; bar/err as for the sweeps.
// dot2: inner products as if in twice the working precision (Dot2).
void mgs(size_t n, FgState *st, double *w, const double *V, size_t ldv, double *partials, unsigned int *bar,
         int *err, bool dot2, cudaStream_t s);
void cgs_update(size_t n, const FgState *st, const double *hin, double *w, const double *V, size_t ldv,
                int want_dots, double *partials, unsigned int *ticket, double *hout, cudaStream_t s);
// zin = V_{st->j} (FP64 copy or FP32 conversion)
template <typename T>
void load_vj(size_t n, const FgState *st, const double *V, T *zin, cudaStream_t s);
// Z_{st->j} = zout
template <typename T>
void store_zj(size_t n, const FgState *st, const T *zout, T *Z, cudaStream_t s);
void norm2(size_t n, const double *v, double *partials, unsigned int *ticket, double *out, bool dot2, cudaStream_t s);
void givens(FgState *st, cudaStream_t s);
void scale_next(size_t n, const double *w, double *vout, const FgState *st, cudaStream_t s);
void backsolve(FgState *st, cudaStream_t s);
template <typename ZT>
void update_x(size_t n, const FgState *st, const ZT *Z, size_t ldz, double *x, cudaStream_t s);
void restart_scale(size_t n, const double *r, double *v0, FgState *st, cudaStream_t s);
// Device-driven solve loop.  cycle_flag: the IF condition = st->stop (the
// inner iteration ended the cycle).  end_cycle (after the update, the true
// residual and its squared norm in st->nrm2[0]): relres, convergence, the
// cap on iterations, status; a continuing solve counts a restart.
// loop_init / loop_flag: the WHILE condition = !done (loop_flag also counts
// the pass and ends the loop with AMG_ERR_LIMIT past loop_cap, or when a
// device wait gave up (*err)).
void cycle_flag(FgState *st, cudaGraphConditionalHandle c, cudaStream_t s);
void end_cycle_dev(FgState *st, cudaStream_t s);
void loop_init(FgState *st, cudaGraphConditionalHandle w, cudaStream_t s);
void loop_flag(FgState *st, const int *err, cudaGraphConditionalHandle w, cudaStream_t s);
int reduce_grid();

}  // namespace amg
