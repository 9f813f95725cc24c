// solve.cu -- solve-phase kernels: CSR and SELL-32 SpMV and residuals, the
// ILU(0) sweeps (per-level launches, level-barrier grid kernels, one-block
// or cluster kernels with the vectors in shared memory, dataflow kernels),
// restriction (segmented sum over aggregate members), prolongation with
// correction, the dense solve of the last level, and the FGMRES pieces
// (modified Gram-Schmidt with plain or Dot2 inner products, CGS2, Givens
// rotations, back substitution, solution update).
//
// Reductions are deterministic: each block writes a partial, then either the
// last block to finish (ticket counter) or every block after a grid barrier
// sums the partials in block order.
#include "solve.cuh"
#include "devsync.cuh"

namespace amg {

template <typename V> __device__ __forceinline__ float tof(V x);
template <> __device__ __forceinline__ float tof<float>(float x) { return x; }
template <> __device__ __forceinline__ float tof<__nv_bfloat16>(__nv_bfloat16 x) { return __bfloat162float(x); }

template <typename T, typename U> __device__ __forceinline__ T cvt(U x) { return (T)x; }

// acc -/+ sum_k v[k] x[ci[k]] over k in [k0, k1), in stored order.  The
// column indices, values and x entries of ROW_CHUNK terms are loaded before
// any of them is used, so their memory latencies overlap; the subtraction
// chain itself keeps the stored order.  COHERENT: x is written by other
// blocks of the same launch and is read past L1.
constexpr int ROW_CHUNK = 8;

template <bool COHERENT, bool SUB, typename T, typename V>
__device__ __forceinline__ T row_acc(T acc, int k0, int k1, const int *__restrict__ ci, const V *__restrict__ v,
                                     const T *x) {
    for (int k = k0; k < k1; k += ROW_CHUNK) {
        int c[ROW_CHUNK];
        V w[ROW_CHUNK];
        T xv[ROW_CHUNK];
#pragma unroll
        for (int q = 0; q < ROW_CHUNK; ++q)
            if (k + q < k1) { c[q] = ci[k + q]; w[q] = v[k + q]; }
#pragma unroll
        for (int q = 0; q < ROW_CHUNK; ++q)
            if (k + q < k1) xv[q] = COHERENT ? __ldcg(x + c[q]) : x[c[q]];
#pragma unroll
        for (int q = 0; q < ROW_CHUNK; ++q)
            if (k + q < k1) acc = SUB ? msub(acc, val_as<T, V>(w[q]), xv[q]) : madd(acc, val_as<T, V>(w[q]), xv[q]);
    }
    return acc;
}
template <bool COHERENT, typename T, typename V>
__device__ __forceinline__ T row_sub(T acc, int k0, int k1, const int *__restrict__ ci, const V *__restrict__ v,
                                     const T *x) {
    return row_acc<COHERENT, true, T, V>(acc, k0, k1, ci, v, x);
}

// ------------------------------------------------------------------ CSR SpMV / residual
// G lanes per row; lanes stride the row, then a shuffle tree reduction.
// mode 0: y = A x;  mode 1: y = b - A x.
template <int G, typename VT, typename XT, typename YT, typename AT>
__global__ void __launch_bounds__(256) k_spmv(int n, const int *__restrict__ rp, const int *__restrict__ ci,
                                              const VT *__restrict__ v, const XT *__restrict__ x,
                                              const YT *__restrict__ b, YT *__restrict__ y, int mode) {
    const int lane = threadIdx.x % G;
    const int rows_per_block = blockDim.x / G;
    // r0 is uniform across the block, so every lane reaches the shuffles
    for (int r0 = blockIdx.x * rows_per_block; r0 < n; r0 += gridDim.x * rows_per_block) {
        const int i = r0 + threadIdx.x / G;
        AT acc = 0;
        if (i < n) {
            const int e1 = rp[i + 1];
            for (int e = rp[i] + lane; e < e1; e += G)
                acc += val_as<AT, VT>(v[e]) * (AT)x[ci[e]];
        }
#pragma unroll
        for (int off = G / 2; off; off >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, off, G);
        if (lane == 0 && i < n) y[i] = mode ? (YT)((AT)b[i] - acc) : (YT)acc;
    }
}

template <typename VT, typename XT, typename YT, typename AT>
void spmv_t(int n, int nnz, const int *rp, const int *ci, const VT *v, const XT *x, const YT *b, YT *y, int mode,
            cudaStream_t s) {
    if (n <= 0) return;
    const int avg = nnz / (n > 0 ? n : 1);
    if (avg <= 6) {
        k_spmv<4, VT, XT, YT, AT><<<grid_for((size_t)n * 4, 256), 256, 0, s>>>(n, rp, ci, v, x, b, y, mode);
    } else if (avg <= 12) {
        k_spmv<8, VT, XT, YT, AT><<<grid_for((size_t)n * 8, 256), 256, 0, s>>>(n, rp, ci, v, x, b, y, mode);
    } else {
        k_spmv<16, VT, XT, YT, AT><<<grid_for((size_t)n * 16, 256), 256, 0, s>>>(n, rp, ci, v, x, b, y, mode);
    }
    CU_LAUNCH("k_spmv"); count_launch();
}

void spmv_f64(int n, int nnz, const int *rp, const int *ci, const double *v, const double *x, double *y, cudaStream_t s) {
    spmv_t<double, double, double, double>(n, nnz, rp, ci, v, x, nullptr, y, 0, s);
}
// y = A x for a caller's CSR whose indices have not been validated: a row
// reads only e in [rp[i], rp[i+1]) (the row pointers were clamped to
// [0, nnz] when they were narrowed), and a column outside [0, n) is skipped
// and counted in *bad instead of being used as an index into x.
template <int G>
__global__ void __launch_bounds__(256) k_spmv_checked(int n, const int *__restrict__ rp, const int *__restrict__ ci,
                                                      const double *__restrict__ v, const double *__restrict__ x,
                                                      double *__restrict__ y, int *bad) {
    const int lane = threadIdx.x % G;
    const int rows_per_block = blockDim.x / G;
    for (int r0 = blockIdx.x * rows_per_block; r0 < n; r0 += gridDim.x * rows_per_block) {
        const int i = r0 + threadIdx.x / G;
        double acc = 0.0;
        int nbad = 0;
        if (i < n) {
            const int e1 = rp[i + 1];
            for (int e = rp[i] + lane; e < e1; e += G) {
                const int c = ci[e];
                if ((unsigned)c < (unsigned)n) acc += v[e] * x[c];
                else ++nbad;
            }
        }
        if (nbad) atomicAdd(bad, nbad);
#pragma unroll
        for (int off = G / 2; off; off >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, off, G);
        if (lane == 0 && i < n) y[i] = acc;
    }
}

void spmv_f64_checked(int n, int nnz, const int *rp, const int *ci, const double *v, const double *x, double *y,
                      int *bad, cudaStream_t s) {
    if (n <= 0) return;
    const int avg = nnz / n;
    if (avg <= 6) {
        k_spmv_checked<4><<<grid_for((size_t)n * 4, 256), 256, 0, s>>>(n, rp, ci, v, x, y, bad);
    } else if (avg <= 12) {
        k_spmv_checked<8><<<grid_for((size_t)n * 8, 256), 256, 0, s>>>(n, rp, ci, v, x, y, bad);
    } else {
        k_spmv_checked<16><<<grid_for((size_t)n * 16, 256), 256, 0, s>>>(n, rp, ci, v, x, y, bad);
    }
    CU_LAUNCH("k_spmv_checked"); count_launch();
}
void spmv_f64_xf32(int n, int nnz, const int *rp, const int *ci, const double *v, const float *x, double *y, cudaStream_t s) {
    spmv_t<double, float, double, double>(n, nnz, rp, ci, v, x, nullptr, y, 0, s);
}
void residual_f64(int n, int nnz, const int *rp, const int *ci, const double *v, const double *x, const double *b,
                  double *r, cudaStream_t s) {
    spmv_t<double, double, double, double>(n, nnz, rp, ci, v, x, b, r, 1, s);
}

template <typename XT, int U>
__global__ void __launch_bounds__(512) k_sell_spmv(int n, const int64_t *__restrict__ ptr, const int *__restrict__ ci,
                                                   const double *__restrict__ v, const XT *__restrict__ x,
                                                   const double *__restrict__ b, double *__restrict__ y, int mode) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const int sl = i >> 5, r = i & 31;
        const int64_t base = ptr[sl];
        const int w = (int)((ptr[sl + 1] - base) >> 5);
        const double *vv = v + base + r;
        const int *cc = ci + base + r;
        double acc = 0.0;
#pragma unroll U
        for (int k = 0; k < w; ++k) acc = madd(acc, __ldg(vv + 32 * k), (double)__ldg(x + __ldg(cc + 32 * k)));
        y[i] = mode ? b[i] - acc : acc;
    }
}

// Launch geometry (threads per block, unroll depth of the column loop) does
// not change what a thread sums or in which order, so every choice gives the
// same bits; the autotuner picks by time.
template <typename XT>
void sell_spmv(int n, int nslices, const int64_t *ptr, const int *ci, const double *v, const XT *x, const double *b,
               double *y, int mode, cudaStream_t s, int block, int unroll) {
    (void)nslices;
    if (block != 64 && block != 128 && block != 256 && block != 512) block = 256;
    const int g = grid_for(n, block);
    switch (unroll) {
    case 2: k_sell_spmv<XT, 2><<<g, block, 0, s>>>(n, ptr, ci, v, x, b, y, mode); break;
    case 8: k_sell_spmv<XT, 8><<<g, block, 0, s>>>(n, ptr, ci, v, x, b, y, mode); break;
    default: k_sell_spmv<XT, 4><<<g, block, 0, s>>>(n, ptr, ci, v, x, b, y, mode); break;
    }
    CU_LAUNCH("k_sell_spmv"); count_launch();
}
template void sell_spmv<double>(int, int, const int64_t *, const int *, const double *, const double *, const double *,
                                double *, int, cudaStream_t, int, int);
template void sell_spmv<float>(int, int, const int64_t *, const int *, const double *, const float *, const double *,
                               double *, int, cudaStream_t, int, int);

// r = b - A x, one thread per row, terms summed in stored column order.
template <typename T, typename V>
__global__ void __launch_bounds__(256) k_residual_seq(int n, const int *__restrict__ rp, const int *__restrict__ ci,
                                                      const V *__restrict__ v, const T *__restrict__ x,
                                                      const T *__restrict__ b, T *__restrict__ r) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const T acc = row_acc<false, false, T, V>(T(0), rp[i], rp[i + 1], ci, v, x);
        r[i] = b[i] - acc;
    }
}

template <typename T, typename V>
void level_residual(const LevelMats<V> &M, const T *x, const T *b, T *r, cudaStream_t s) {
    if (M.n <= 0) return;
    k_residual_seq<T, V><<<grid_for(M.n, 256), 256, 0, s>>>(M.n, M.rp, M.ci, M.v, x, b, r);
    CU_LAUNCH("k_residual_seq"); count_launch();
}
template void level_residual<double, double>(const LevelMats<double> &, const double *, const double *, double *, cudaStream_t);
template void level_residual<float, float>(const LevelMats<float> &, const float *, const float *, float *, cudaStream_t);
template void level_residual<float, __nv_bfloat16>(const LevelMats<__nv_bfloat16> &, const float *, const float *, float *, cudaStream_t);

// ------------------------------------------------------------------ ILU(0) sweeps
// Forward (unit lower): y[i] = z[i] - sum_k L_ik y[k].  Backward:
// t[i] = (y[i] - sum_j U_ij t[j]) / u_ii.  One launch per schedule level;
// each row's terms are summed in stored (ascending column) order.
// with_diag selects the division (backward of LU, forward of the transposed
// solve U^T).
template <typename T, typename V>
__global__ void __launch_bounds__(128) k_sweep(int cnt, const int *__restrict__ rows, const int *__restrict__ rp,
                                               const int *__restrict__ ci, const V *__restrict__ v,
                                               const T *__restrict__ dg, const T *__restrict__ in, T *out,
                                               int with_diag) {
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < cnt; t += gridDim.x * blockDim.x) {
        const int i = rows[t];
        T acc = in[i];
        acc = row_sub<false, T, V>(acc, rp[t], rp[t + 1], ci, v, out);
        out[i] = with_diag ? acc / dg[t] : acc;
    }
}

template <typename T, typename V>
void sweep(const SweepView<T, V> &S, const T *in, T *out, int with_diag, cudaStream_t s) {
    for (int l = 0; l < S.nlev; ++l) {
        const int b = S.lev_ptr[l], cnt = S.lev_ptr[l + 1] - b;
        if (cnt <= 0) continue;
        k_sweep<T, V><<<grid_for(cnt, 128), 128, 0, s>>>(cnt, S.rows + b, S.rp + b, S.ci, S.v,
                                                          S.d ? S.d + b : nullptr, in, out, with_diag);
    }
    CU_LAUNCH("k_sweep"); count_launch(S.nlev);
}
template void sweep<double, double>(const SweepView<double, double> &, const double *, double *, int, cudaStream_t);

// ------------------------------------------------------------------ persistent sweeps
// The same barrier split in two, so that work independent of the other
// blocks (loading the next level's read-only data) overlaps the wait.
// Thread 0 carries the generation from arrive to wait.
__device__ __forceinline__ void grid_arrive(unsigned int *bar, unsigned int &gen, bool &released) {
    __syncthreads();
    released = false;
    if (threadIdx.x == 0) {
        unsigned int arrived;
        asm volatile("ld.relaxed.gpu.global.u32 %0, [%1];" : "=r"(gen) : "l"(bar + 1) : "memory");
        asm volatile("atom.acq_rel.gpu.global.add.u32 %0, [%1], 1;" : "=r"(arrived) : "l"(bar) : "memory");
        if (arrived + 1u == gridDim.x) {
            asm volatile("st.relaxed.gpu.global.u32 [%0], %1;" ::"l"(bar), "r"(0u) : "memory");
            asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(bar + 1), "r"(gen + 1u) : "memory");
            released = true;
        }
    }
}
__device__ __forceinline__ void grid_wait(unsigned int *bar, int *err, unsigned int gen, bool released) {
    if (threadIdx.x == 0 && !released) {
        unsigned int spins = 0;
        while (ld_acquire_gpu(bar + 1) == gen) {
            if (*(volatile int *)err) break;
            if (++spins > SPIN_LIMIT) { atomicExch(err, 1); break; }
            if (spins > 64) __nanosleep(20);
        }
    }
    __syncthreads();
}

template <typename T> __device__ __forceinline__ T ld_cg(const T *p) { return __ldcg(p); }

// Barrier between schedule levels, split into arrive and wait.  SYNC 0:
// grid barrier of a cooperative launch; 1: the grid is one thread-block
// cluster (hardware cluster barrier, release/acquire at cluster scope); 2:
// the grid is one block.
struct LevelSync {
    unsigned int gen;
    bool released;
};
template <int SYNC>
__device__ __forceinline__ void level_arrive(unsigned int *bar, LevelSync &ls) {
    if constexpr (SYNC == 0) {
        grid_arrive(bar, ls.gen, ls.released);
    } else if constexpr (SYNC == 1) {
        asm volatile("barrier.cluster.arrive.release.aligned;" ::: "memory");
    }
}
template <int SYNC>
__device__ __forceinline__ void level_wait(unsigned int *bar, int *err, const LevelSync &ls) {
    if constexpr (SYNC == 0) {
        grid_wait(bar, err, ls.gen, ls.released);
    } else if constexpr (SYNC == 1) {
        asm volatile("barrier.cluster.wait.acquire.aligned;" ::: "memory");
    } else {
        __syncthreads();
    }
}

// Software pipeline over schedule levels.  A thread's row in a level is
// read in two dependent stages: A (row id, extent, diagonal) from the
// position, then B (the first SWEEP_PF column indices and values, and the
// input entry) from A.  Before computing level l the thread issues B for
// level l+1 and A for level l+2, so both loads have a whole level (compute
// plus barrier) to arrive; only the values of earlier rows remain on the
// critical path.  Positions beyond the first a thread owns in a level (levels
// wider than the grid) are read directly.
#ifndef AMG_SWEEP_PF
#define AMG_SWEEP_PF 12
#endif
constexpr int SWEEP_PF = AMG_SWEEP_PF;
constexpr int SWEEP_CLUSTER_MAX = 8;   // portable cluster size
constexpr size_t SWEEP_DL_MAX_BYTES = 48 * 1024;   // level pointers staged in shared memory

template <typename T>
struct RowA {
    int t, i, k0, k1;
    T d;
};
template <typename T, typename V, int PF = SWEEP_PF>
struct RowB {
    int c[PF];
    V v[PF];
    T in;
};

template <typename T, typename V>
__device__ __forceinline__ RowA<T> row_a(const SweepView<T, V> &S, const int *dl, int l, int tid, int with_diag) {
    RowA<T> a{-1, 0, 0, 0, T(1)};
    if (l >= S.nlev) return a;
    const int t = dl[l] + tid;
    if (t >= dl[l + 1]) return a;
    a.t = t;
    a.i = S.rows[t];
    a.k0 = S.rp[t];
    a.k1 = S.rp[t + 1];
    if (with_diag) a.d = S.d[t];
    return a;
}

// IN: 0 global input (plain load), 1 global input written earlier in this
// launch (read past L1), 2 shared-memory input.
template <int IN, typename T, typename V, int PF = SWEEP_PF>
__device__ __forceinline__ RowB<T, V, PF> row_b(const SweepView<T, V> &S, const RowA<T> &a, const T *in) {
    RowB<T, V, PF> b;
    b.in = T(0);
    if (a.t < 0) return b;
#pragma unroll
    for (int q = 0; q < PF; ++q)
        if (a.k0 + q < a.k1) { b.c[q] = S.ci[a.k0 + q]; b.v[q] = S.v[a.k0 + q]; }
    b.in = IN == 1 ? __ldcg(in + a.i) : in[a.i];
    return b;
}

// out_i = (in_i - sum_k v_k x_{c_k}) [/ d] for a pipelined row; x read past L1
// (COHERENT) or directly (shared memory).
template <bool COHERENT, typename T, typename V, int PF = SWEEP_PF>
__device__ __forceinline__ T row_value(const SweepView<T, V> &S, const RowA<T> &a, const RowB<T, V, PF> &b, const T *x,
                                       int with_diag) {
    T xv[PF];
#pragma unroll
    for (int q = 0; q < PF; ++q)
        if (a.k0 + q < a.k1) xv[q] = COHERENT ? __ldcg(x + b.c[q]) : x[b.c[q]];
    T acc = b.in;
#pragma unroll
    for (int q = 0; q < PF; ++q)
        if (a.k0 + q < a.k1) acc = msub(acc, val_as<T, V>(b.v[q]), xv[q]);
    acc = row_sub<COHERENT, T, V>(acc, a.k0 + PF, a.k1, S.ci, S.v, x);
    return with_diag ? acc / a.d : acc;
}

// One triangular solve over all schedule levels of S; dl: the level
// pointers in shared memory.
template <int SYNC, int IN, typename T, typename V>
__device__ __forceinline__ void sweep_phase(const SweepView<T, V> &S, const int *dl, int with_diag, const T *in,
                                            T *out, unsigned int *bar, int *err, int tid, int nthr, bool last_barrier) {
    RowA<T> a0 = row_a(S, dl, 0, tid, with_diag), a1 = row_a(S, dl, 1, tid, with_diag);
    RowB<T, V> b0 = row_b<IN>(S, a0, in);
    for (int l = 0; l < S.nlev; ++l) {
        const RowB<T, V> b1 = row_b<IN>(S, a1, in);
        const RowA<T> a2 = row_a(S, dl, l + 2, tid, with_diag);
        if (a0.t >= 0) {
            out[a0.i] = row_value<true, T, V>(S, a0, b0, out, with_diag);
            const int e = dl[l + 1];
            for (int t = a0.t + nthr; t < e; t += nthr) {
                const int i = S.rows[t];
                T acc = IN == 1 ? __ldcg(in + i) : in[i];
                acc = row_sub<true, T, V>(acc, S.rp[t], S.rp[t + 1], S.ci, S.v, out);
                out[i] = with_diag ? acc / S.d[t] : acc;
            }
        }
        if (l + 1 < S.nlev || last_barrier) {
            LevelSync ls{};
            level_arrive<SYNC>(bar, ls);
            level_wait<SYNC>(bar, err, ls);
        }
        a0 = a1;
        b0 = b1;
        a1 = a2;
    }
}

// Dynamic shared memory: the level pointers of F and B.
template <typename T, typename V, int SYNC>
__global__ void __launch_bounds__(256) k_sweep_pair(SweepView<T, V> F, int f_diag, SweepView<T, V> B, int b_diag,
                                                   const T *in, T *y, T *out, unsigned int *bar, int *err) {
    extern __shared__ int sweep_dl[];
    int *dlf = sweep_dl, *dlb = sweep_dl + F.nlev + 1;
    for (int l = threadIdx.x; l <= F.nlev; l += blockDim.x) dlf[l] = F.dlev[l];
    for (int l = threadIdx.x; l <= B.nlev; l += blockDim.x) dlb[l] = B.dlev[l];
    __syncthreads();
    const int tid = blockIdx.x * blockDim.x + threadIdx.x, nthr = gridDim.x * blockDim.x;
    sweep_phase<SYNC, 0, T, V>(F, dlf, f_diag, in, y, bar, err, tid, nthr, true);
    sweep_phase<SYNC, 1, T, V>(B, dlb, b_diag, y, out, bar, err, tid, nthr, false);
}

// ------------------------------------------------------------------ small levels: cluster + DSMEM
// A level whose two solve vectors (y, out) fit in shared memory runs as one
// thread-block cluster of up to 8 CTAs.  Every CTA keeps a full copy of y
// and out in its shared memory; a computed row value is written to all
// copies with st.shared::cluster, and the level barrier is the cluster
// barrier (release/acquire at cluster scope covers those writes).  Reads of
// earlier rows are then local shared-memory loads, so a schedule level costs
// one cluster barrier instead of a grid barrier plus L2 round trips.  Rows
// are summed in stored order as in every other variant.
// threads per block: 512 for FP32 vectors, 256 for FP64 (register budget)
template <typename T> __host__ __device__ constexpr int dsm_threads() { return sizeof(T) == 8 ? 256 : 512; }
constexpr int DSM_MAX_CTAS = 8;
// row entries prefetched a level ahead in the cluster kernel (deeper spills
// registers at 512 threads)
#ifndef AMG_DSM_PF
#define AMG_DSM_PF 8
#endif
constexpr int DSM_PF = AMG_DSM_PF;
constexpr size_t DSM_MAX_BYTES = 200 * 1024;

__device__ __forceinline__ uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }
__device__ __forceinline__ uint32_t map_rank(uint32_t addr, uint32_t rank) {
    uint32_t r;
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(addr), "r"(rank));
    return r;
}
__device__ __forceinline__ void st_dsm(uint32_t addr, float v) {
    asm volatile("st.shared::cluster.f32 [%0], %1;" ::"r"(addr), "f"(v) : "memory");
}
__device__ __forceinline__ void st_dsm(uint32_t addr, double v) {
    asm volatile("st.shared::cluster.f64 [%0], %1;" ::"r"(addr), "d"(v) : "memory");
}
__device__ __forceinline__ uint32_t cluster_ctarank() {
    uint32_t r;
    asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
    return r;
}
__device__ __forceinline__ uint32_t cluster_nctarank() {
    uint32_t r;
    asm volatile("mov.u32 %0, %%cluster_nctarank;" : "=r"(r));
    return r;
}
__device__ __forceinline__ void cluster_barrier() {
    asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}

// One triangular solve of the DSMEM kernel, pipelined like sweep_phase:
// xs is the local copy read by this solve (shared memory), rem the copies
// written (one per CTA; CLUSTER only).  The result goes to global memory
// only at the end of the kernel, so no level barrier waits for global
// stores.
template <int IN, bool CLUSTER, typename T, typename V>
__device__ __forceinline__ void dsm_phase(const SweepView<T, V> &S, const int *dl, int with_diag, const T *in, T *xs,
                                          const uint32_t *rem, int cs, int tid, int nthr) {
    auto finish = [&](int i, T v) {
        if constexpr (CLUSTER) {
#pragma unroll
            for (int r = 0; r < DSM_MAX_CTAS; ++r)
                if (r < cs) st_dsm(rem[r] + (uint32_t)(i * sizeof(T)), v);
        } else {
            xs[i] = v;
        }
    };
    RowA<T> a0 = row_a(S, dl, 0, tid, with_diag), a1 = row_a(S, dl, 1, tid, with_diag);
    RowB<T, V, DSM_PF> b0 = row_b<IN, T, V, DSM_PF>(S, a0, in);
    for (int l = 0; l < S.nlev; ++l) {
        const RowB<T, V, DSM_PF> b1 = row_b<IN, T, V, DSM_PF>(S, a1, in);
        const RowA<T> a2 = row_a(S, dl, l + 2, tid, with_diag);
        if (a0.t >= 0) {
            finish(a0.i, row_value<false, T, V, DSM_PF>(S, a0, b0, xs, with_diag));
            const int e = dl[l + 1];
            for (int t = a0.t + nthr; t < e; t += nthr) {      // levels wider than the grid
                const int i = S.rows[t];
                const T acc = row_sub<false, T, V>(in[i], S.rp[t], S.rp[t + 1], S.ci, S.v, xs);
                finish(i, with_diag ? acc / S.d[t] : acc);
            }
        }
        // after the last level too: in a cluster, keeps every CTA alive while
        // others write to it
        if constexpr (CLUSTER) cluster_barrier();
        else __syncthreads();
        a0 = a1;
        b0 = b1;
        a1 = a2;
    }
}

// Dynamic shared memory: y[n], out[n], the level pointers of F and B.
// CLUSTER false: the grid is one block and the level barrier is the block
// barrier (17-41 ns against ~250 ns for a cluster barrier on this GPU).
template <typename T, typename V, bool CLUSTER>
__global__ void __launch_bounds__(dsm_threads<T>()) k_sweep_pair_dsm(SweepView<T, V> F, int f_diag, SweepView<T, V> B,
                                                                int b_diag, const T *in, T *out, int n) {
    extern __shared__ __align__(16) unsigned char dsm_raw[];
    T *ys = reinterpret_cast<T *>(dsm_raw);
    T *os = ys + n;
    int *dlf = reinterpret_cast<int *>(os + n);
    int *dlb = dlf + F.nlev + 1;
    for (int l = threadIdx.x; l <= F.nlev; l += dsm_threads<T>()) dlf[l] = F.dlev[l];
    for (int l = threadIdx.x; l <= B.nlev; l += dsm_threads<T>()) dlb[l] = B.dlev[l];
    __syncthreads();
    uint32_t cr = 0, cs = 1;
    uint32_t yr[DSM_MAX_CTAS], orr[DSM_MAX_CTAS];
    if constexpr (CLUSTER) {
        cr = cluster_ctarank();
        cs = cluster_nctarank();
#pragma unroll
        for (int r = 0; r < DSM_MAX_CTAS; ++r)
            if (r < (int)cs) { yr[r] = map_rank(smem_u32(ys), r); orr[r] = map_rank(smem_u32(os), r); }
    }
    const int tid = (int)cr * dsm_threads<T>() + threadIdx.x, nthr = (int)cs * dsm_threads<T>();
    dsm_phase<0, CLUSTER, T, V>(F, dlf, f_diag, in, ys, yr, (int)cs, tid, nthr);
    dsm_phase<2, CLUSTER, T, V>(B, dlb, b_diag, ys, os, orr, (int)cs, tid, nthr);
    for (int i = tid; i < n; i += nthr) out[i] = os[i];     // every CTA holds all of out
}

bool sweep_fits_dsm(int n, int nlev_f, int nlev_b, size_t elem) {
    return n > 0 && 2 * (size_t)n * elem + sizeof(int) * (size_t)(nlev_f + nlev_b + 2) <= DSM_MAX_BYTES;
}

// Launches the DSMEM variant when the level fits; returns false otherwise.
template <typename T, typename V>
static bool sweep_pair_dsm(const SweepView<T, V> &F, int f_diag, const SweepView<T, V> &B, int b_diag, const T *in,
                           T *out, int maxw, cudaStream_t s) {
    const int n = F.lev_ptr[F.nlev];
    const size_t bytes = 2 * (size_t)n * sizeof(T) + sizeof(int) * (size_t)(F.nlev + B.nlev + 2);
    if (n <= 0 || bytes > DSM_MAX_BYTES) return false;
    static const bool ok = [] {               // once: opt in to large shared memory, check a full cluster fits
        if (cudaFuncSetAttribute(k_sweep_pair_dsm<T, V, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)DSM_MAX_BYTES) != cudaSuccess ||
            cudaFuncSetAttribute(k_sweep_pair_dsm<T, V, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)DSM_MAX_BYTES) != cudaSuccess)
            return false;
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3(DSM_MAX_CTAS);
        cfg.blockDim = dim3(dsm_threads<T>());
        cfg.dynamicSmemBytes = DSM_MAX_BYTES;
        cudaLaunchAttribute attr[1];
        attr[0].id = cudaLaunchAttributeClusterDimension;
        attr[0].val.clusterDim.x = DSM_MAX_CTAS;
        attr[0].val.clusterDim.y = 1;
        attr[0].val.clusterDim.z = 1;
        cfg.attrs = attr;
        cfg.numAttrs = 1;
        int clusters = 0;
        if (cudaOccupancyMaxActiveClusters(&clusters, k_sweep_pair_dsm<T, V, true>, &cfg) != cudaSuccess)
            return false;
        return clusters >= 1;
    }();
    if (!ok) { cudaGetLastError(); return false; }
    // One block (block barrier, ~20-40 ns) unless its threads would need many
    // more row rounds than there are levels: in one block a level of w rows
    // takes ceil(w / threads) dependent rounds, in a cluster about one round
    // plus a cluster barrier (~0.5 us more per level).
    int rounds = 0;
    for (int l = 0; l < F.nlev; ++l) rounds += (F.lev_ptr[l + 1] - F.lev_ptr[l] + dsm_threads<T>() - 1) / dsm_threads<T>();
    for (int l = 0; l < B.nlev; ++l) rounds += (B.lev_ptr[l + 1] - B.lev_ptr[l] + dsm_threads<T>() - 1) / dsm_threads<T>();
    int cs = 1;
    if (2 * rounds > 3 * (F.nlev + B.nlev))
        cs = std::min((maxw + 2 * dsm_threads<T>() - 1) / (2 * dsm_threads<T>()), DSM_MAX_CTAS);
    SweepView<T, V> f = F, b = B;
    if (cs == 1) {
        k_sweep_pair_dsm<T, V, false><<<1, dsm_threads<T>(), bytes, s>>>(f, f_diag, b, b_diag, in, out, n);
        CU_LAUNCH("k_sweep_pair_dsm (one block)");
    } else {
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3(cs);
        cfg.blockDim = dim3(dsm_threads<T>());
        cfg.dynamicSmemBytes = bytes;
        cfg.stream = s;
        cudaLaunchAttribute attr[1];
        attr[0].id = cudaLaunchAttributeClusterDimension;
        attr[0].val.clusterDim.x = cs;
        attr[0].val.clusterDim.y = 1;
        attr[0].val.clusterDim.z = 1;
        cfg.attrs = attr;
        cfg.numAttrs = 1;
        CU(cudaLaunchKernelEx(&cfg, k_sweep_pair_dsm<T, V, true>, f, f_diag, b, b_diag, in, out, n));
    }
    count_launch();
    return true;
}

template <typename T, typename V>
int sweep_pair_coop(const SweepView<T, V> &F, int f_diag, const SweepView<T, V> &B, int b_diag, const T *in,
                     T *y, T *out, unsigned int *bar, int *err, cudaStream_t s) {
    static const int grid = [] {               // initialised once, thread-safe
        int per_sm = 0;
        CU(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_sweep_pair<T, V, 0>, 256, SWEEP_DL_MAX_BYTES));
        return sm_count() * (per_sm < 2 ? (per_sm < 1 ? 1 : per_sm) : 2);
    }();
    int maxw = 0;
    for (int l = 0; l < F.nlev; ++l) maxw = max(maxw, F.lev_ptr[l + 1] - F.lev_ptr[l]);
    for (int l = 0; l < B.nlev; ++l) maxw = max(maxw, B.lev_ptr[l + 1] - B.lev_ptr[l]);
    if (sweep_pair_dsm<T, V>(F, f_diag, B, b_diag, in, out, maxw, s)) return SWEEP_KIND_DSM_REPLICATED;
    int g = (maxw + 255) / 256;
    if (g > grid) g = grid;
    if (g < 1) g = 1;
    SweepView<T, V> f = F, b = B;
    const size_t dl_bytes = sizeof(int) * (size_t)(F.nlev + B.nlev + 2);
    if (dl_bytes > SWEEP_DL_MAX_BYTES) {          // too many schedule levels to stage: one launch per level
        sweep<T, V>(F, in, y, f_diag, s);
        sweep<T, V>(B, y, out, b_diag, s);
        return SWEEP_KIND_LEVELS;
    }
    if (g == 1) {
        k_sweep_pair<T, V, 2><<<1, 256, dl_bytes, s>>>(f, f_diag, b, b_diag, in, y, out, bar, err);
        CU_LAUNCH("k_sweep_pair (one block)");
    } else if (g <= SWEEP_CLUSTER_MAX) {
        // a grid this small runs as one cluster: hardware barrier, all blocks co-scheduled
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3(g);
        cfg.blockDim = dim3(256);
        cfg.dynamicSmemBytes = dl_bytes;
        cfg.stream = s;
        cudaLaunchAttribute attr[1];
        attr[0].id = cudaLaunchAttributeClusterDimension;
        attr[0].val.clusterDim.x = g;
        attr[0].val.clusterDim.y = 1;
        attr[0].val.clusterDim.z = 1;
        cfg.attrs = attr;
        cfg.numAttrs = 1;
        CU(cudaLaunchKernelEx(&cfg, k_sweep_pair<T, V, 1>, f, f_diag, b, b_diag, in, y, out, bar, err));
    } else {
        void *args[] = {&f, (void *)&f_diag, &b, (void *)&b_diag, (void *)&in, (void *)&y, (void *)&out, (void *)&bar,
                        (void *)&err};
        CU(cudaLaunchCooperativeKernel((const void *)k_sweep_pair<T, V, 0>, dim3(g), dim3(256), args, dl_bytes, s));
    }
    count_launch();
    return g == 1 ? SWEEP_KIND_BLOCK : g <= SWEEP_CLUSTER_MAX ? SWEEP_KIND_CLUSTER_GRID : SWEEP_KIND_GRID;
}
template int sweep_pair_coop<double, double>(const SweepView<double, double> &, int, const SweepView<double, double> &,
                                              int, const double *, double *, double *, unsigned int *, int *, cudaStream_t);
template int sweep_pair_coop<float, float>(const SweepView<float, float> &, int, const SweepView<float, float> &, int,
                                            const float *, float *, float *, unsigned int *, int *, cudaStream_t);
template int sweep_pair_coop<float, __nv_bfloat16>(const SweepView<float, __nv_bfloat16> &, int,
                                                    const SweepView<float, __nv_bfloat16> &, int, const float *, float *,
                                                    float *, unsigned int *, int *, cudaStream_t);
template void sweep<float, float>(const SweepView<float, float> &, const float *, float *, int, cudaStream_t);
template void sweep<float, __nv_bfloat16>(const SweepView<float, __nv_bfloat16> &, const float *, float *, int, cudaStream_t);

// ------------------------------------------------------------------ dataflow sweeps
// The same triangular solves without level barriers.  Rows are taken in the
// schedule order (a topological order of the solve's dependencies); each
// thread owns positions tid, tid + nthr, ... and a row starts as soon as the
// values it reads are there.  Readiness is carried by the value itself: the
// output vector holds a signalling-NaN sentinel until the row is written, and
// arithmetic never yields that bit pattern (a computed NaN is the quiet
// canonical one; a stored value equal to the sentinel is replaced by it).
// Each aligned 32/64-bit store and load is single-copy atomic, so a reader
// sees either the sentinel or the final value.  The terms of a row are
// consumed in stored order, so the result is the one of the level-by-level
// sweep bit for bit.
//
// Progress: all blocks are resident (cooperative launch) and a warp polls
// with every lane in one loop, so the lowest unfinished position always has
// its inputs and an owner that is not blocked: the solve cannot deadlock.
// Every wait is still bounded (DF_SPIN_LIMIT polls per row); on expiry the
// kernel sets *err and all threads leave.
//
// Sentinel upkeep: y (the forward result) is sentinel on entry and is put back
// to sentinel row by row as the backward solve consumes it; out is reset to
// sentinel during the forward solve and a grid barrier separates that reset
// from the backward solve.
constexpr unsigned int DF_SPIN_LIMIT = 1u << 20;
// Threads for about this many schedule levels of rows in flight, and the
// sleep between polls of a row that is not ready (compile-time tunables).
#ifndef AMG_DF_LEVELS_IN_FLIGHT
#define AMG_DF_LEVELS_IN_FLIGHT 4
#endif
#ifndef AMG_DF_BACKOFF_NS
#define AMG_DF_BACKOFF_NS 0
#endif
constexpr int DF_LEVELS_IN_FLIGHT = AMG_DF_LEVELS_IN_FLIGHT;
constexpr unsigned int DF_BACKOFF_NS = AMG_DF_BACKOFF_NS;

template <typename T>
__global__ void k_fill_sentinel(size_t n, T *x) {
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
        x[i] = Sentinel<T>::value();
}

// One triangular solve in dataflow order.  A lane reads the values of its
// row DF_BATCH at a time (independent loads in flight together), consumes
// them in stored order up to the first one not yet written, and polls again
// after a short sleep.  Returns false when a wait ran out or another thread
// reported one.
constexpr int DF_BATCH = 4;

template <typename T, typename V>
__device__ __forceinline__ bool df_phase(const SweepView<T, V> &S, int with_diag, const T *in, bool in_coherent,
                                         T *out, T *consumed, int *err, int tid, int nthr) {
    const int total = S.dlev[S.nlev];
    const int lane = threadIdx.x & 31;
    for (int base = tid - lane; base < total; base += nthr) {
        const int p = base + lane;
        bool done = p >= total;
        int i = 0, k = 0, k1 = 0;
        T acc = T(0), d = T(1);
        if (!done) {
            i = S.rows[p];
            k = S.rp[p];
            k1 = S.rp[p + 1];
            acc = in_coherent ? ld_cg(in + i) : in[i];
            if (with_diag) d = S.d[p];
        }
        unsigned int spins = 0;
        bool fail = false;
        while (__any_sync(0xffffffffu, !done)) {
            if (!done) {
                bool blocked = false;
                while (k < k1 && !blocked) {
                    T xv[DF_BATCH];
#pragma unroll
                    for (int q = 0; q < DF_BATCH; ++q)
                        if (k + q < k1) xv[q] = Sentinel<T>::ld(out + S.ci[k + q]);
#pragma unroll
                    for (int q = 0; q < DF_BATCH; ++q) {
                        if (blocked || k >= k1) continue;
                        if (Sentinel<T>::is(xv[q])) { blocked = true; continue; }
                        acc = msub(acc, val_as<T, V>(S.v[k]), xv[q]);
                        ++k;
                    }
                }
                if (!blocked) {
                    Sentinel<T>::st(out + i, with_diag ? acc / d : acc);
                    if (consumed) consumed[i] = Sentinel<T>::value();
                    done = true;
                } else if (++spins > DF_SPIN_LIMIT) {
                    atomicExch(err, 1);
                    fail = true;
                    done = true;
                } else if ((spins & 255u) == 0 && *(volatile int *)err) {
                    fail = true;
                    done = true;
                } else if (DF_BACKOFF_NS > 0) {
                    __nanosleep(DF_BACKOFF_NS);
                }
            }
        }
        if (__any_sync(0xffffffffu, fail)) return false;
    }
    return true;
}

template <typename T, typename V>
__global__ void __launch_bounds__(256) k_sweep_df(SweepView<T, V> F, int f_diag, SweepView<T, V> B, int b_diag,
                                                  const T *in, T *y, T *out, unsigned int *bar, int *err) {
    const int tid = blockIdx.x * blockDim.x + threadIdx.x, nthr = gridDim.x * blockDim.x;
    const int nb = B.dlev[B.nlev];
    for (int p = tid; p < nb; p += nthr) out[B.rows[p]] = Sentinel<T>::value();
    df_phase<T, V>(F, f_diag, in, false, y, nullptr, err, tid, nthr);
    grid_barrier(bar, err);
    if (*(volatile int *)err) return;
    df_phase<T, V>(B, b_diag, y, true, out, y, err, tid, nthr);
}

template <typename T>
void fill_sentinel(T *x, size_t n, cudaStream_t s) {
    if (!n) return;
    k_fill_sentinel<T><<<grid_for(n, 256), 256, 0, s>>>(n, x);
    CU_LAUNCH("k_fill_sentinel"); count_launch();
}
template void fill_sentinel<float>(float *, size_t, cudaStream_t);
template void fill_sentinel<double>(double *, size_t, cudaStream_t);

template <typename T, typename V>
void sweep_pair_df(const SweepView<T, V> &F, int f_diag, const SweepView<T, V> &B, int b_diag, const T *in, T *y,
                   T *out, unsigned int *bar, int *err, cudaStream_t s) {
    static const int grid = [] {               // initialised once, thread-safe
        int per_sm = 0;
        CU(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_sweep_df<T, V>, 256, 0));
        return sm_count() * (per_sm < 1 ? 1 : per_sm);
    }();
    // enough threads for a few schedule levels in flight; more only add
    // polling traffic
    int maxw = 0;
    for (int l = 0; l < F.nlev; ++l) maxw = max(maxw, F.lev_ptr[l + 1] - F.lev_ptr[l]);
    for (int l = 0; l < B.nlev; ++l) maxw = max(maxw, B.lev_ptr[l + 1] - B.lev_ptr[l]);
    int g = (int)(((int64_t)DF_LEVELS_IN_FLIGHT * maxw + 255) / 256);
    if (g > grid) g = grid;
    if (g < 1) g = 1;
    SweepView<T, V> f = F, b = B;
    void *args[] = {&f, (void *)&f_diag, &b, (void *)&b_diag, (void *)&in, (void *)&y, (void *)&out, (void *)&bar,
                    (void *)&err};
    CU(cudaLaunchCooperativeKernel((const void *)k_sweep_df<T, V>, dim3(g), dim3(256), args, 0, s));
    count_launch();
}
template void sweep_pair_df<double, double>(const SweepView<double, double> &, int, const SweepView<double, double> &,
                                            int, const double *, double *, double *, unsigned int *, int *, cudaStream_t);
template void sweep_pair_df<float, float>(const SweepView<float, float> &, int, const SweepView<float, float> &, int,
                                          const float *, float *, float *, unsigned int *, int *, cudaStream_t);
template void sweep_pair_df<float, __nv_bfloat16>(const SweepView<float, __nv_bfloat16> &, int,
                                                  const SweepView<float, __nv_bfloat16> &, int, const float *, float *,
                                                  float *, unsigned int *, int *, cudaStream_t);

// Accurate inner products (DOT2): the Dot2 scheme of Ogita, Rump and Oishi
// (2005).  Each product is split exactly into h + r (TwoProduct via fma), the
// h are added with the exact error of each addition kept (TwoSum), errors are
// collected in c; partial (p, c) pairs merge by TwoSum of the p and the sum of
// the c.  The result p + c is the exact inner product correctly rounded in all
// but near-tie cases, so it does not depend on how the sum is split across
// threads and blocks.
__device__ __forceinline__ void two_sum_d(double a, double b, double &s, double &e) {
    const double t = __dadd_rn(a, b);
    const double z = __dsub_rn(t, a);
    e = __dadd_rn(__dsub_rn(a, __dsub_rn(t, z)), __dsub_rn(b, z));
    s = t;
}
__device__ __forceinline__ void dot2_add(double &p, double &c, double x, double y) {
    const double h = __dmul_rn(x, y);
    const double r = __fma_rn(x, y, -h);
    double q;
    two_sum_d(p, h, p, q);
    c = __dadd_rn(c, __dadd_rn(q, r));
}
__device__ __forceinline__ void dot2_merge(double &p, double &c, double p2, double c2) {
    double q;
    two_sum_d(p, p2, p, q);
    c = __dadd_rn(c, __dadd_rn(c2, q));
}

// ------------------------------------------------------------------ dense rows
// Row i of a dense n x n inverse (column i for the transpose) times h, for
// one warp: lane r sums j = r, r + 32, ... in ascending j (fused
// multiply-add); the partial sums are added by halving (lane r + lane r + 16,
// then 8, 4, 2, 1).  Lane 0 returns the result.
template <typename H>
__device__ __forceinline__ double warp_dense_dot(const double *inv, int n, int i, int transpose, int lane, H h) {
    double s = 0.0;
    if (transpose) {
        for (int j = lane; j < n; j += 32) s = __fma_rn(inv[(size_t)j * n + i], h(j), s);
    } else {
        const double *row = inv + (size_t)i * n;
        for (int j = lane; j < n; j += 32) s = __fma_rn(row[j], h(j), s);
    }
#pragma unroll
    for (int off = 16; off; off >>= 1) s = __dadd_rn(s, __shfl_down_sync(0xffffffffu, s, off));
    return s;
}
// The same row as an inner product evaluated as if in twice the working
// precision (Dot2): each lane keeps a (p, c) pair over its terms, the pairs
// merge across the warp, lane 0 returns p + c.  The value does not depend on
// how the terms are split (except in near-tie cases).
template <typename H>
__device__ __forceinline__ double warp_dense_dot2(const double *inv, int n, int i, int transpose, int lane, H h) {
    double p = 0.0, c = 0.0;
    if (transpose) {
        for (int j = lane; j < n; j += 32) dot2_add(p, c, inv[(size_t)j * n + i], h(j));
    } else {
        const double *row = inv + (size_t)i * n;
        for (int j = lane; j < n; j += 32) dot2_add(p, c, row[j], h(j));
    }
#pragma unroll
    for (int off = 16; off; off >>= 1) {
        const double p2 = __shfl_down_sync(0xffffffffu, p, off), c2 = __shfl_down_sync(0xffffffffu, c, off);
        dot2_merge(p, c, p2, c2);
    }
    return __dadd_rn(p, c);
}

// ------------------------------------------------------------------ single-block deep V-cycle
// The levels below a size threshold run their whole V-cycle (deep_inner = 1:
// smoother, residual, restriction, the next level, prolongation) in one
// block: a phase ends with a block barrier instead of a kernel boundary, and
// the small vectors stay in the SM's L1 (reads after the barrier see the
// block's own writes).  Sweeps use the same two-stage row pipeline as the
// grid kernels.
constexpr int DEEP_THREADS = 256;
constexpr int DEEP_PF = 8;   // row entries prefetched a level ahead (register budget of the deep kernel)

template <typename T, typename V>
__device__ __forceinline__ void deep_sweep(const SweepView<T, V> &S, const T *in, T *out, int with_diag) {
    const int tid = threadIdx.x, nthr = DEEP_THREADS;
    RowA<T> a0 = row_a(S, S.dlev, 0, tid, with_diag), a1 = row_a(S, S.dlev, 1, tid, with_diag);
    RowB<T, V, DEEP_PF> b0 = row_b<0, T, V, DEEP_PF>(S, a0, in);
    for (int l = 0; l < S.nlev; ++l) {
        const RowB<T, V, DEEP_PF> b1 = row_b<0, T, V, DEEP_PF>(S, a1, in);
        const RowA<T> a2 = row_a(S, S.dlev, l + 2, tid, with_diag);
        if (a0.t >= 0) {
            out[a0.i] = row_value<false, T, V, DEEP_PF>(S, a0, b0, out, with_diag);
            const int e = S.dlev[l + 1];
            for (int t = a0.t + nthr; t < e; t += nthr) {
                const int i = S.rows[t];
                const T acc = row_sub<false, T, V>(in[i], S.rp[t], S.rp[t + 1], S.ci, S.v, out);
                out[i] = with_diag ? acc / S.d[t] : acc;
            }
        }
        __syncthreads();
        a0 = a1;
        b0 = b1;
        a1 = a2;
    }
}

template <typename T, typename V>
__global__ void __launch_bounds__(DEEP_THREADS) k_deep_vcycle(const DeepLevel<T, V> *L, int count) {
    int m = 0;
    for (; m < count; ++m) {
        const DeepLevel<T, V> &D = L[m];
        if (D.dense) {                       // exact solve of the last level, one warp per row
            const int lane = threadIdx.x & 31;
            for (int i = threadIdx.x >> 5; i < D.n; i += DEEP_THREADS / 32) {
                const double s = warp_dense_dot(D.inv, D.n, i, 0, lane, [&](int j) { return (double)D.h[j]; });
                if (lane == 0) D.g[i] = (T)s;
            }
            __syncthreads();
            break;
        }
        deep_sweep<T, V>(D.fwd, D.h, D.y, 0);
        deep_sweep<T, V>(D.bwd, D.y, D.has_child ? D.t : D.g, 1);
        if (!D.has_child) break;
        for (int i = threadIdx.x; i < D.n; i += DEEP_THREADS)
            D.r[i] = D.h[i] - row_acc<false, false, T, V>(T(0), D.rp[i], D.rp[i + 1], D.ci, D.v, D.t);
        __syncthreads();
        const DeepLevel<T, V> &C = L[m + 1];
        for (int I = threadIdx.x; I < C.n; I += DEEP_THREADS) {
            T acc = 0;
            for (int q = D.mptr[I]; q < D.mptr[I + 1]; ++q) acc += D.r[D.midx[q]];
            C.h[I] = acc;
        }
        __syncthreads();
    }
    for (int k = (m < count ? m : count - 1) - 1; k >= 0; --k) {
        const DeepLevel<T, V> &D = L[k];
        const DeepLevel<T, V> &C = L[k + 1];
        for (int i = threadIdx.x; i < D.n; i += DEEP_THREADS) D.g[i] = D.t[i] + C.g[D.agg[i]];
        __syncthreads();
    }
}

template <typename T, typename V>
void deep_vcycle(const DeepLevel<T, V> *levels, int count, cudaStream_t s) {
    k_deep_vcycle<T, V><<<1, DEEP_THREADS, 0, s>>>(levels, count);
    CU_LAUNCH("k_deep_vcycle");
    count_launch();
}
template void deep_vcycle<double, double>(const DeepLevel<double, double> *, int, cudaStream_t);
template void deep_vcycle<float, float>(const DeepLevel<float, float> *, int, cudaStream_t);
template void deep_vcycle<float, __nv_bfloat16>(const DeepLevel<float, __nv_bfloat16> *, int, cudaStream_t);

// ------------------------------------------------------------------ transfers
// h[I] = sum over members m of I (ascending) of r[m]  (restriction P^T)
template <typename T>
__global__ void k_restrict(int nc, const int *__restrict__ mptr, const int *__restrict__ midx,
                           const T *__restrict__ r, T *__restrict__ h) {
    for (int I = blockIdx.x * blockDim.x + threadIdx.x; I < nc; I += gridDim.x * blockDim.x) {
        T acc = 0;
        for (int t = mptr[I]; t < mptr[I + 1]; ++t) acc += r[midx[t]];
        h[I] = acc;
    }
}
template <typename T>
void restrict_to(int nc, const int *mptr, const int *midx, const T *r, T *h, cudaStream_t s) {
    k_restrict<T><<<grid_for(nc, 256), 256, 0, s>>>(nc, mptr, midx, r, h);
    CU_LAUNCH("k_restrict"); count_launch();
}
template void restrict_to<double>(int, const int *, const int *, const double *, double *, cudaStream_t);
template void restrict_to<float>(int, const int *, const int *, const float *, float *, cudaStream_t);

// With c = g[agg[i]] (agg given) or g[i] (agg null):
// mode 0/3: q = t + c;  mode 1/4: q += t + c;  mode 2: q = c.
template <typename T, typename Q>
__global__ void k_prolong(int n, const int *__restrict__ agg, const T *__restrict__ t, const T *__restrict__ g,
                          Q *__restrict__ q, int mode) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        T c = agg ? g[agg[i]] : g[i];
        if (mode == 2) { q[i] = (Q)c; continue; }
        T val = t[i] + c;
        q[i] = (mode == 1 || mode == 4) ? (Q)((T)q[i] + val) : (Q)val;
    }
}
template <typename T, typename Q>
void prolong(int n, const int *agg, const T *t, const T *g, Q *q, int mode, cudaStream_t s) {
    k_prolong<T, Q><<<grid_for(n, 256), 256, 0, s>>>(n, agg, t, g, q, mode);
    CU_LAUNCH("k_prolong"); count_launch();
}
template void prolong<double, double>(int, const int *, const double *, const double *, double *, int, cudaStream_t);
template void prolong<float, float>(int, const int *, const float *, const float *, float *, int, cudaStream_t);

// out (+)= in  (mode 0 copy, mode 1 add)
template <typename T>
__global__ void k_axpy1(size_t n, const T *__restrict__ in, T *__restrict__ out, int mode) {
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
        out[i] = mode ? out[i] + in[i] : in[i];
}
template <typename T>
void vec_acc(size_t n, const T *in, T *out, int mode, cudaStream_t s) {
    k_axpy1<T><<<grid_for(n, 256), 256, 0, s>>>(n, in, out, mode);
    CU_LAUNCH("k_axpy1"); count_launch();
}
template void vec_acc<double>(size_t, const double *, double *, int, cudaStream_t);
template void vec_acc<float>(size_t, const float *, float *, int, cudaStream_t);

template <typename A, typename B>
__global__ void k_convert(size_t n, const A *__restrict__ in, B *__restrict__ out) {
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
        out[i] = (B)in[i];
}
void convert_f64_f32(size_t n, const double *in, float *out, cudaStream_t s) {
    k_convert<double, float><<<grid_for(n, 256), 256, 0, s>>>(n, in, out);
    CU_LAUNCH("k_convert"); count_launch();
}
void convert_f32_f64(size_t n, const float *in, double *out, cudaStream_t s) {
    k_convert<float, double><<<grid_for(n, 256), 256, 0, s>>>(n, in, out);
    CU_LAUNCH("k_convert"); count_launch();
}

// Dense last level: g = Ainv h (transpose: g = Ainv^T h), one warp per row
// (h staged in shared memory as FP64).  Plain: lane r sums the terms j = r,
// r + 32, ... in ascending j with fused multiply-adds and the 32 partial
// sums are added by halving; DOT2: each row as an inner product evaluated as
// if in twice the working precision (warp_dense_dot2).
constexpr int DENSE_WARPS = 8;
template <typename T, bool DOT2>
__global__ void __launch_bounds__(32 * DENSE_WARPS) k_dense_gemv(int n, const double *__restrict__ inv,
                                                                 const T *__restrict__ h, T *__restrict__ g,
                                                                 int transpose, int mode) {
    extern __shared__ double dense_h[];
    for (int j = threadIdx.x; j < n; j += blockDim.x) dense_h[j] = (double)h[j];
    __syncthreads();
    const int lane = threadIdx.x & 31;
    for (int i = blockIdx.x * DENSE_WARPS + (threadIdx.x >> 5); i < n; i += gridDim.x * DENSE_WARPS) {
        const double s = DOT2 ? warp_dense_dot2(inv, n, i, transpose, lane, [&](int j) { return dense_h[j]; })
                              : warp_dense_dot(inv, n, i, transpose, lane, [&](int j) { return dense_h[j]; });
        if (lane == 0) g[i] = mode ? (T)((double)g[i] + s) : (T)s;
    }
}
template <typename T>
void dense_solve(int n, const double *inv, const T *h, T *g, int transpose, int mode, bool dot2, cudaStream_t s) {
    const int blocks = (n + DENSE_WARPS - 1) / DENSE_WARPS;
    if (dot2)
        k_dense_gemv<T, true><<<blocks, 32 * DENSE_WARPS, sizeof(double) * (size_t)n, s>>>(n, inv, h, g, transpose,
                                                                                            mode);
    else
        k_dense_gemv<T, false><<<blocks, 32 * DENSE_WARPS, sizeof(double) * (size_t)n, s>>>(n, inv, h, g, transpose,
                                                                                             mode);
    CU_LAUNCH("k_dense_gemv"); count_launch();
}
// FP32 inverse, FP32 accumulation: lane r sums the terms j = r, r + 32, ...
// with fused multiply-adds, the 32 partial sums are added by halving.
__global__ void __launch_bounds__(32 * DENSE_WARPS) k_dense_gemv_f32(int n, const float *__restrict__ inv,
                                                                     const float *__restrict__ h,
                                                                     float *__restrict__ g, int transpose) {
    extern __shared__ float dense_hf[];
    for (int j = threadIdx.x; j < n; j += blockDim.x) dense_hf[j] = h[j];
    __syncthreads();
    const int lane = threadIdx.x & 31;
    for (int i = blockIdx.x * DENSE_WARPS + (threadIdx.x >> 5); i < n; i += gridDim.x * DENSE_WARPS) {
        float acc = 0.f;
        if (transpose) {
            for (int j = lane; j < n; j += 32) acc = __fmaf_rn(inv[(size_t)j * n + i], dense_hf[j], acc);
        } else {
            const float *row = inv + (size_t)i * n;
            for (int j = lane; j < n; j += 32) acc = __fmaf_rn(row[j], dense_hf[j], acc);
        }
#pragma unroll
        for (int off = 16; off; off >>= 1) acc = __fadd_rn(acc, __shfl_down_sync(0xffffffffu, acc, off));
        if (lane == 0) g[i] = acc;
    }
}
void dense_solve_f32(int n, const float *inv, const float *h, float *g, int transpose, cudaStream_t s) {
    const int blocks = (n + DENSE_WARPS - 1) / DENSE_WARPS;
    k_dense_gemv_f32<<<blocks, 32 * DENSE_WARPS, sizeof(float) * (size_t)n, s>>>(n, inv, h, g, transpose);
    CU_LAUNCH("k_dense_gemv_f32"); count_launch();
}
template void dense_solve<double>(int, const double *, const double *, double *, int, int, bool, cudaStream_t);
template void dense_solve<float>(int, const double *, const float *, float *, int, int, bool, cudaStream_t);

// ------------------------------------------------------------------ FGMRES pieces
// Block-level reduction of K accumulators into partials[block*KMAX + k].
template <int NT>
__device__ __forceinline__ void block_reduce_store(double *acc, int K, double *partials, int kmax) {
    __shared__ double red[NT / 32][KMAX1];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int k = 0; k < KMAX1; ++k) {
        if (k >= K) break;
        double a = acc[k];
        for (int off = 16; off; off >>= 1) a += __shfl_down_sync(0xffffffffu, a, off);
        if (lane == 0) red[warp][k] = a;
    }
    __syncthreads();
    for (int k = threadIdx.x; k < K; k += NT) {
        double a = 0.0;
        for (int w = 0; w < NT / 32; ++w) a += red[w][k];
        partials[(size_t)blockIdx.x * kmax + k] = a;
    }
}

// Last block to arrive (ticket) returns true; partials are then visible.
__device__ __forceinline__ bool last_block(unsigned int *ticket) {
    __shared__ bool am_last;
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned int t = atomicAdd(ticket, 1u);
        am_last = (t == gridDim.x - 1);
    }
    __syncthreads();
    if (am_last) __threadfence();
    return am_last;
}

// Fixed-order sum of the partials of K accumulators -> out[k].
template <int NT>
__device__ void final_reduce(const double *partials, int K, int kmax, double *out) {
    for (int k = threadIdx.x; k < K; k += NT) {
        double a = 0.0;
        for (int b = 0; b < (int)gridDim.x; ++b) a += ((volatile const double *)partials)[(size_t)b * kmax + k];
        out[k] = a;
    }
    __syncthreads();
}

constexpr int RT = 256;   // threads per reduction block

// h[k] = (w, V_k) for k < K   (first CGS pass)
__global__ void __launch_bounds__(RT) k_mdot(size_t n, const FgState *st, const double *__restrict__ w,
                                             const double *__restrict__ V, size_t ldv, double *partials,
                                             unsigned int *ticket, double *h) {
    const int K = st->j + 1;
    double acc[KMAX1];
#pragma unroll
    for (int k = 0; k < KMAX1; ++k) acc[k] = 0.0;
    for (size_t i = blockIdx.x * (size_t)RT + threadIdx.x; i < n; i += (size_t)gridDim.x * RT) {
        const double wi = w[i];
#pragma unroll
        for (int k = 0; k < KMAX1; ++k)
            if (k < K) acc[k] += wi * V[k * ldv + i];
    }
    block_reduce_store<RT>(acc, K, partials, KMAX1);
    if (last_block(ticket)) {
        final_reduce<RT>(partials, K, KMAX1, h);
        if (threadIdx.x == 0) *ticket = 0;
    }
}

// w -= sum_k hin[k] V_k; then hout[k] = (w, V_k) (second CGS pass) or, with
// K2 == 0, hout[0] = (w, w).
__global__ void __launch_bounds__(RT) k_cgs_update(size_t n, const FgState *st, const double *__restrict__ hin,
                                                   double *w, const double *__restrict__ V, size_t ldv,
                                                   int want_dots, double *partials, unsigned int *ticket,
                                                   double *hout) {
    const int K = st->j + 1;
    __shared__ double hs[KMAX1];
    for (int k = threadIdx.x; k < KMAX1; k += RT) hs[k] = k < K ? hin[k] : 0.0;
    __syncthreads();
    double acc[KMAX1];
#pragma unroll
    for (int k = 0; k < KMAX1; ++k) acc[k] = 0.0;
    for (size_t i = blockIdx.x * (size_t)RT + threadIdx.x; i < n; i += (size_t)gridDim.x * RT) {
        double vk[KMAX1];
        double wi = w[i];
#pragma unroll
        for (int k = 0; k < KMAX1; ++k)
            if (k < K) { vk[k] = V[k * ldv + i]; wi -= hs[k] * vk[k]; }
        w[i] = wi;
        if (want_dots) {
#pragma unroll
            for (int k = 0; k < KMAX1; ++k)
                if (k < K) acc[k] += wi * vk[k];
        } else {
            acc[0] += wi * wi;
        }
    }
    const int Kout = want_dots ? K : 1;
    block_reduce_store<RT>(acc, Kout, partials, KMAX1);
    if (last_block(ticket)) {
        final_reduce<RT>(partials, Kout, KMAX1, hout);
        if (threadIdx.x == 0) *ticket = 0;
    }
}

// Givens step for column j (single thread): H column from h1 + h2 and ||w||,
// apply previous rotations, new rotation, residual estimate.  Each rotated
// entry c1 a + c2 b is fma(c1, a, c2 b): the second product rounded, then one
// fused multiply-add.
__device__ __forceinline__ double mul(double a, double b) { return __dmul_rn(a, b); }
__device__ __forceinline__ double add(double a, double b) { return __dadd_rn(a, b); }
__device__ __forceinline__ double fma2(double c1, double a, double c2, double b) { return __fma_rn(c1, a, mul(c2, b)); }

__global__ void k_givens(FgState *st) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    if (st->stop) return;
    const int m = st->m;
    const int j = st->j;
    double *H = st->H;                       // H[k*m + j]
    for (int k = 0; k <= j; ++k) H[k * m + j] = add(st->h1[k], st->h2[k]);
    const double hn = sqrt(st->nrm2[0]);
    H[(j + 1) * m + j] = hn;
    st->hn = hn;
    for (int k = 0; k < j; ++k) {
        double a = H[k * m + j], c = H[(k + 1) * m + j];
        H[k * m + j] = fma2(st->cs[k], a, st->sn[k], c);
        H[(k + 1) * m + j] = fma2(-st->sn[k], a, st->cs[k], c);
    }
    double a = H[j * m + j], c = H[(j + 1) * m + j];
    double rho = sqrt(fma2(a, a, c, c));
    if (!(rho > 0.0) || !isfinite(rho)) {
        st->status = 6;
        st->stop = 1;
        return;
    }
    st->cs[j] = a / rho;
    st->sn[j] = c / rho;
    H[j * m + j] = rho;
    H[(j + 1) * m + j] = 0.0;
    st->s[j + 1] = mul(-st->sn[j], st->s[j]);
    st->s[j] = mul(st->cs[j], st->s[j]);
    st->total += 1;
    const double est = fabs(st->s[j + 1]) / st->bnorm;
    if (st->hist_len < st->hist_cap) st->hist[st->hist_len++] = est;
    st->jdone = j + 1;
    st->j = j + 1;
    if (!isfinite(est)) { st->status = 6; st->stop = 1; return; }
    if (est <= st->tol || hn == 0.0 || st->total >= st->maxit || j + 1 >= m) st->stop = 1;
}

// V_{j} = w / h_{j,j-1} after the Givens step advanced j (skipped at the last
// column and when w vanished)
__global__ void k_scale_next(size_t n, const double *__restrict__ w, double *__restrict__ V, const FgState *st) {
    const int j = st->j;
    const double hn = st->hn;
    if (j > st->m || hn == 0.0) return;
    double *vout = V + (size_t)j * n;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
        vout[i] = w[i] / hn;
}

template <typename T>
__global__ void k_load_vj(size_t n, const FgState *st, const double *__restrict__ V, T *__restrict__ zin) {
    const double *vj = V + (size_t)st->j * n;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
        zin[i] = (T)vj[i];
}
template <typename T>
void load_vj(size_t n, const FgState *st, const double *V, T *zin, cudaStream_t s) {
    k_load_vj<T><<<grid_for(n, 256), 256, 0, s>>>(n, st, V, zin);
    CU_LAUNCH("k_load_vj"); count_launch();
}
template void load_vj<double>(size_t, const FgState *, const double *, double *, cudaStream_t);
template void load_vj<float>(size_t, const FgState *, const double *, float *, cudaStream_t);

template <typename T>
__global__ void k_store_zj(size_t n, const FgState *st, const T *__restrict__ zout, T *__restrict__ Z) {
    T *zj = Z + (size_t)st->j * n;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
        zj[i] = zout[i];
}
template <typename T>
void store_zj(size_t n, const FgState *st, const T *zout, T *Z, cudaStream_t s) {
    k_store_zj<T><<<grid_for(n, 256), 256, 0, s>>>(n, st, zout, Z);
    CU_LAUNCH("k_store_zj"); count_launch();
}
template void store_zj<double>(size_t, const FgState *, const double *, double *, cudaStream_t);
template void store_zj<float>(size_t, const FgState *, const float *, float *, cudaStream_t);

// y = H(1:j,1:j)^{-1} s(1:j) (single thread)
__global__ void k_backsolve(FgState *st) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    if (st->status) return;                  // a breakdown ends the solve without an update
    const int m = st->m, j = st->jdone;
    for (int k = j - 1; k >= 0; --k) {
        double t = st->s[k];
        for (int l = k + 1; l < j; ++l) t = __fma_rn(-st->H[k * m + l], st->y[l], t);
        st->y[k] = t / st->H[k * m + k];
    }
}

// x += sum_{k<j} y_k Z_k
template <typename ZT>
__global__ void k_update_x(size_t n, const FgState *st, const ZT *__restrict__ Z, size_t ldz, double *x) {
    __shared__ double ys[KMAX1];
    const int j = st->status ? 0 : st->jdone;
    for (int k = threadIdx.x; k < KMAX1; k += blockDim.x) ys[k] = k < j ? st->y[k] : 0.0;
    __syncthreads();
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        double acc = x[i];
        for (int k = 0; k < j; ++k) acc = __fma_rn(ys[k], (double)Z[k * ldz + i], acc);
        x[i] = acc;
    }
}
template <typename ZT>
void update_x(size_t n, const FgState *st, const ZT *Z, size_t ldz, double *x, cudaStream_t s) {
    k_update_x<ZT><<<grid_for(n, 256), 256, 0, s>>>(n, st, Z, ldz, x);
    CU_LAUNCH("k_update_x"); count_launch();
}
template void update_x<double>(size_t, const FgState *, const double *, size_t, double *, cudaStream_t);
template void update_x<float>(size_t, const FgState *, const float *, size_t, double *, cudaStream_t);

// ||v||^2 -> out (deterministic)
// Block reduction of (p, c) pairs: returns the block's pair in thread 0.
__device__ __forceinline__ void block_merge2(double &p, double &c) {
    __shared__ double sp[RT / 32], sc[RT / 32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int off = 16; off; off >>= 1) {
        const double p2 = __shfl_down_sync(0xffffffffu, p, off), c2 = __shfl_down_sync(0xffffffffu, c, off);
        dot2_merge(p, c, p2, c2);
    }
    if (lane == 0) { sp[warp] = p; sc[warp] = c; }
    __syncthreads();
    if (threadIdx.x == 0) {
        p = sp[0];
        c = sc[0];
        for (int w = 1; w < RT / 32; ++w) dot2_merge(p, c, sp[w], sc[w]);
    }
    __syncthreads();
}

template <bool DOT2>
__global__ void __launch_bounds__(RT) k_norm2(size_t n, const double *__restrict__ v, double *partials,
                                              unsigned int *ticket, double *out) {
    if constexpr (DOT2) {
        double p = 0.0, c = 0.0, p2 = 0.0, c2 = 0.0;
        const size_t stride = (size_t)gridDim.x * RT;
        size_t i = blockIdx.x * (size_t)RT + threadIdx.x;
        for (; i + stride < n; i += 2 * stride) {
            dot2_add(p, c, v[i], v[i]);
            dot2_add(p2, c2, v[i + stride], v[i + stride]);
        }
        if (i < n) dot2_add(p, c, v[i], v[i]);
        dot2_merge(p, c, p2, c2);
        block_merge2(p, c);
        if (threadIdx.x == 0) {
            partials[(size_t)blockIdx.x * KMAX1] = p;
            partials[(size_t)blockIdx.x * KMAX1 + 1] = c;
        }
        if (last_block(ticket)) {
            if (threadIdx.x == 0) {
                double P = 0.0, Cc = 0.0;
                for (int b = 0; b < (int)gridDim.x; ++b)
                    dot2_merge(P, Cc, ((volatile const double *)partials)[(size_t)b * KMAX1],
                               ((volatile const double *)partials)[(size_t)b * KMAX1 + 1]);
                out[0] = __dadd_rn(P, Cc);
                *ticket = 0;
            }
        }
    } else {
        double acc[1] = {0.0};
        for (size_t i = blockIdx.x * (size_t)RT + threadIdx.x; i < n; i += (size_t)gridDim.x * RT)
            acc[0] = __fma_rn(v[i], v[i], acc[0]);
        block_reduce_store<RT>(acc, 1, partials, KMAX1);
        if (last_block(ticket)) {
            final_reduce<RT>(partials, 1, KMAX1, out);
            if (threadIdx.x == 0) *ticket = 0;
        }
    }
}

// Modified Gram-Schmidt step of the Arnoldi process, the form of the plain
// sequential definition: for k = 0..j, h_k = (w, v_k) then w <- w - h_k v_k;
// finally ||w||^2.  One cooperative launch; the update of step k is fused
// with the dot product of step k + 1 (or the norm after the last step).  Each
// block reduces its part, a grid barrier follows, and every block then adds
// the block partials in block order, so all blocks hold the same h_k.  Step
// partials alternate between two halves of the buffer: a block still reading
// step k's partials cannot be overtaken by writes of step k + 2, which lie
// behind the barrier of step k + 1.  Products accumulate by fused
// multiply-add, and the update is w - h v as one fused multiply-add.  Each
// element of w is touched by one thread only, so w needs no cross-block
// visibility.
__device__ __forceinline__ double mgs_grid_sum(double acc, double *partials, unsigned int *bar, int *err) {
    __shared__ double red[RT / 32];
    __shared__ double total;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int off = 16; off; off >>= 1) acc = __dadd_rn(acc, __shfl_down_sync(0xffffffffu, acc, off));
    if (lane == 0) red[warp] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double a = 0.0;
        for (int w = 0; w < RT / 32; ++w) a = __dadd_rn(a, red[w]);
        __stcg(partials + blockIdx.x, a);
    }
    grid_barrier(bar, err);
    if (warp == 0) {
        double a = 0.0;
        for (int b = lane; b < (int)gridDim.x; b += 32) a = __dadd_rn(a, __ldcg(partials + b));
        for (int off = 16; off; off >>= 1) a = __dadd_rn(a, __shfl_down_sync(0xffffffffu, a, off));
        if (lane == 0) total = a;
    }
    __syncthreads();
    return total;
}

// Grid sum of (p, c) pairs, same pattern as mgs_grid_sum; partials holds two
// doubles per block.
__device__ __forceinline__ double mgs_grid_sum2(double p, double c, double *partials, unsigned int *bar, int *err) {
    __shared__ double total;
    block_merge2(p, c);
    if (threadIdx.x == 0) {
        __stcg(partials + 2 * blockIdx.x, p);
        __stcg(partials + 2 * blockIdx.x + 1, c);
    }
    grid_barrier(bar, err);
    if (threadIdx.x == 0) {
        double P = 0.0, Cc = 0.0;
        for (int b = 0; b < (int)gridDim.x; ++b) dot2_merge(P, Cc, __ldcg(partials + 2 * b), __ldcg(partials + 2 * b + 1));
        total = __dadd_rn(P, Cc);
    }
    __syncthreads();
    return total;
}

template <bool DOT2>
__global__ void __launch_bounds__(RT) k_mgs(size_t n, FgState *st, double *w, const double *__restrict__ V,
                                            size_t ldv, double *partials, unsigned int *bar, int *err) {
    if (st->stop) return;                    // same value in every block
    const int j = st->j;
    const size_t tid = blockIdx.x * (size_t)RT + threadIdx.x, nthr = (size_t)gridDim.x * RT;
    const size_t half = (size_t)(DOT2 ? 2 : 1) * gridDim.x;
    auto gsum = [&](double p, double c, int k) {
        double *buf = partials + (size_t)(k & 1) * half;
        return DOT2 ? mgs_grid_sum2(p, c, buf, bar, err) : mgs_grid_sum(p, buf, bar, err);
    };
    // Dot2 keeps two independent (p, c) chains per thread (even and odd
    // elements of its stride), merged at the end, for instruction-level
    // parallelism in the FP64 pipe.
    double p = 0.0, c = 0.0, p2 = 0.0, c2 = 0.0;
    if (DOT2) {
        size_t i = tid;
        for (; i + nthr < n; i += 2 * nthr) {
            dot2_add(p, c, w[i], V[i]);
            dot2_add(p2, c2, w[i + nthr], V[i + nthr]);
        }
        if (i < n) dot2_add(p, c, w[i], V[i]);
        dot2_merge(p, c, p2, c2);
    } else {
        for (size_t i = tid; i < n; i += nthr) p = __fma_rn(w[i], V[i], p);
    }
    double h = gsum(p, c, 0);
    for (int k = 0; k <= j; ++k) {
        if (blockIdx.x == 0 && threadIdx.x == 0) { st->h1[k] = h; st->h2[k] = 0.0; }
        const double *vk = V + (size_t)k * ldv;
        const double *vn = k < j ? V + (size_t)(k + 1) * ldv : nullptr;
        p = 0.0;
        c = 0.0;
        if (DOT2) {
            p2 = 0.0;
            c2 = 0.0;
            size_t i = tid;
            for (; i + nthr < n; i += 2 * nthr) {
                const double wa = __fma_rn(-h, vk[i], w[i]), wb = __fma_rn(-h, vk[i + nthr], w[i + nthr]);
                w[i] = wa;
                w[i + nthr] = wb;
                dot2_add(p, c, wa, vn ? vn[i] : wa);
                dot2_add(p2, c2, wb, vn ? vn[i + nthr] : wb);
            }
            if (i < n) {
                const double wa = __fma_rn(-h, vk[i], w[i]);
                w[i] = wa;
                dot2_add(p, c, wa, vn ? vn[i] : wa);
            }
            dot2_merge(p, c, p2, c2);
        } else {
            for (size_t i = tid; i < n; i += nthr) {
                const double wi = __fma_rn(-h, vk[i], w[i]);
                w[i] = wi;
                p = __fma_rn(wi, vn ? vn[i] : wi, p);
            }
        }
        h = gsum(p, c, k + 1);
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) st->nrm2[0] = h;
}

void mgs(size_t n, FgState *st, double *w, const double *V, size_t ldv, double *partials, unsigned int *bar,
         int *err, bool dot2, cudaStream_t s) {
    static const int grid = [] {               // initialised once, thread-safe
        int a = 0, b = 0;
        CU(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&a, k_mgs<false>, RT, 0));
        CU(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_mgs<true>, RT, 0));
        const int per_sm = std::min(a, b);
        const int g = sm_count() * (per_sm < 2 ? (per_sm < 1 ? 1 : per_sm) : 2);
        return std::min(g, reduce_grid() * KMAX1 / 4);   // two halves of (p, c) pairs in the partials
    }();
    size_t g = (n + RT - 1) / RT;
    if (g > (size_t)grid) g = grid;
    if (g < 1) g = 1;
    void *args[] = {(void *)&n, (void *)&st, (void *)&w, (void *)&V, (void *)&ldv, (void *)&partials, (void *)&bar,
                    (void *)&err};
    const void *fn = dot2 ? (const void *)k_mgs<true> : (const void *)k_mgs<false>;
    CU(cudaLaunchCooperativeKernel(fn, dim3((unsigned)g), dim3(RT), args, 0, s));
    count_launch();
}

int reduce_grid() { return sm_count() * 4; }

void mdot(size_t n, const FgState *st, const double *w, const double *V, size_t ldv, double *partials,
          unsigned int *ticket, double *h, cudaStream_t s) {
    k_mdot<<<reduce_grid(), RT, 0, s>>>(n, st, w, V, ldv, partials, ticket, h);
    CU_LAUNCH("k_mdot"); count_launch();
}
void cgs_update(size_t n, const FgState *st, const double *hin, double *w, const double *V, size_t ldv,
                int want_dots, double *partials, unsigned int *ticket, double *hout, cudaStream_t s) {
    k_cgs_update<<<reduce_grid(), RT, 0, s>>>(n, st, hin, w, V, ldv, want_dots, partials, ticket, hout);
    CU_LAUNCH("k_cgs_update"); count_launch();
}
void norm2(size_t n, const double *v, double *partials, unsigned int *ticket, double *out, bool dot2, cudaStream_t s) {
    if (dot2) k_norm2<true><<<reduce_grid(), RT, 0, s>>>(n, v, partials, ticket, out);
    else k_norm2<false><<<reduce_grid(), RT, 0, s>>>(n, v, partials, ticket, out);
    CU_LAUNCH("k_norm2"); count_launch();
}
void givens(FgState *st, cudaStream_t s) {
    k_givens<<<1, 32, 0, s>>>(st);
    CU_LAUNCH("k_givens"); count_launch();
}
void scale_next(size_t n, const double *w, double *V, const FgState *st, cudaStream_t s) {
    k_scale_next<<<grid_for(n, 256), 256, 0, s>>>(n, w, V, st);
    CU_LAUNCH("k_scale_next"); count_launch();
}
void backsolve(FgState *st, cudaStream_t s) {
    k_backsolve<<<1, 32, 0, s>>>(st);
    CU_LAUNCH("k_backsolve"); count_launch();
}

// restart: V_0 = r / beta with beta = sqrt(nrm2); s = beta e1
__global__ void k_restart_scale(size_t n, const double *__restrict__ r, double *__restrict__ v0, FgState *st) {
    if (st->done) return;                    // device loop: the solve ended at this cycle
    const double beta = sqrt(st->nrm2[0]);
    if (beta > 0.0)
        for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
            v0[i] = r[i] / beta;
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        for (int k = 0; k <= st->m; ++k) st->s[k] = 0.0;
        st->s[0] = beta;
        st->jdone = 0;
        st->j = 0;
        st->stop = 0;
    }
}
void restart_scale(size_t n, const double *r, double *v0, FgState *st, cudaStream_t s) {
    k_restart_scale<<<grid_for(n, 256), 256, 0, s>>>(n, r, v0, st);
    CU_LAUNCH("k_restart_scale"); count_launch();
}

__global__ void k_cycle_flag(FgState *st, cudaGraphConditionalHandle c) {
    if (threadIdx.x == 0 && blockIdx.x == 0) cudaGraphSetConditional(c, st->stop ? 1u : 0u);
}
void cycle_flag(FgState *st, cudaGraphConditionalHandle c, cudaStream_t s) {
    k_cycle_flag<<<1, 32, 0, s>>>(st, c);
    CU_LAUNCH("k_cycle_flag"); count_launch();
}

// The host driver's end-of-cycle decision, on the device (status codes as in
// the public header: 6 numeric, 7 not converged).
__global__ void k_end_cycle(FgState *st) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    if (st->status) { st->done = 1; return; }
    const double relres = sqrt(st->nrm2[0]) / st->bnorm;
    st->relres = relres;
    if (!isfinite(relres)) { st->status = 6; st->done = 1; return; }
    if (relres <= st->tol) { st->done = 1; return; }
    if (st->total >= st->maxit) { st->status = 7; st->done = 1; return; }
    st->restarts += 1;
}
void end_cycle_dev(FgState *st, cudaStream_t s) {
    k_end_cycle<<<1, 32, 0, s>>>(st);
    CU_LAUNCH("k_end_cycle"); count_launch();
}

__global__ void k_loop_init(FgState *st, cudaGraphConditionalHandle w) {
    if (threadIdx.x == 0 && blockIdx.x == 0) cudaGraphSetConditional(w, st->done ? 0u : 1u);
}
void loop_init(FgState *st, cudaGraphConditionalHandle w, cudaStream_t s) {
    k_loop_init<<<1, 32, 0, s>>>(st, w);
    CU_LAUNCH("k_loop_init"); count_launch();
}

__global__ void k_loop_flag(FgState *st, const int *err, cudaGraphConditionalHandle w) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    st->passes += 1;
    if (*err && !st->done) st->done = 1;                       // reported by the host as AMG_ERR_LIMIT
    if (!st->done && st->passes >= st->loop_cap) { st->status = 8; st->done = 1; }
    cudaGraphSetConditional(w, st->done ? 0u : 1u);
}
void loop_flag(FgState *st, const int *err, cudaGraphConditionalHandle w, cudaStream_t s) {
    k_loop_flag<<<1, 32, 0, s>>>(st, err, w);
    CU_LAUNCH("k_loop_flag"); count_launch();
}

}  // namespace amg
