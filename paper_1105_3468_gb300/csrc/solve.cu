// solve.cu -- solve-phase kernels: CSR SpMV and residuals, ILU(0) sweeps
// by schedule level, restriction (segmented sum over aggregate members),
// prolongation with correction, the dense solve of the last level, and the
// FGMRES pieces (multi-vector dot products, CGS2 updates, Givens rotations,
// back substitution, solution update).
//
// Reductions are deterministic: each block writes a partial, the last block
// to finish (ticket counter) sums the partials in block order.
#include "solve.cuh"

namespace amg {

template <typename V> __device__ __forceinline__ float tof(V x);
template <> __device__ __forceinline__ float tof<float>(float x) { return x; }
template <> __device__ __forceinline__ float tof<__nv_bfloat16>(__nv_bfloat16 x) { return __bfloat162float(x); }

template <typename T, typename V> __device__ __forceinline__ T val_as(V x);
template <> __device__ __forceinline__ double val_as<double, double>(double x) { return x; }
template <> __device__ __forceinline__ float val_as<float, float>(float x) { return x; }
template <> __device__ __forceinline__ float val_as<float, __nv_bfloat16>(__nv_bfloat16 x) { return __bfloat162float(x); }
template <> __device__ __forceinline__ double val_as<double, float>(float x) { return (double)x; }

template <typename T, typename U> __device__ __forceinline__ T cvt(U x) { return (T)x; }

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
void spmv_f64_xf32(int n, int nnz, const int *rp, const int *ci, const double *v, const float *x, double *y, cudaStream_t s) {
    spmv_t<double, float, double, double>(n, nnz, rp, ci, v, x, nullptr, y, 0, s);
}
void residual_f64(int n, int nnz, const int *rp, const int *ci, const double *v, const double *x, const double *b,
                  double *r, cudaStream_t s) {
    spmv_t<double, double, double, double>(n, nnz, rp, ci, v, x, b, r, 1, s);
}

template <typename T, typename V>
void level_residual(const LevelMats<V> &M, const T *x, const T *b, T *r, cudaStream_t s) {
    spmv_t<V, T, T, T>(M.n, M.nnz, M.rp, M.ci, M.v, x, b, r, 1, s);
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
        for (int e = rp[t]; e < rp[t + 1]; ++e) acc -= val_as<T, V>(v[e]) * out[ci[e]];
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
template void sweep<float, float>(const SweepView<float, float> &, const float *, float *, int, cudaStream_t);
template void sweep<float, __nv_bfloat16>(const SweepView<float, __nv_bfloat16> &, const float *, float *, int, cudaStream_t);

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

// Dense last level: g = Ainv h (transpose: g = Ainv^T h); one warp per row.
template <typename T>
__global__ void k_dense_gemv(int n, const double *__restrict__ inv, const T *__restrict__ h, T *__restrict__ g,
                             int transpose, int mode) {
    const int lane = threadIdx.x & 31;
    const int warps = gridDim.x * blockDim.x / 32;
    for (int i = (blockIdx.x * blockDim.x + threadIdx.x) / 32; i < n; i += warps) {
        double acc = 0.0;
        for (int j = lane; j < n; j += 32)
            acc += (transpose ? inv[(size_t)j * n + i] : inv[(size_t)i * n + j]) * (double)h[j];
        for (int off = 16; off; off >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, off);
        if (lane == 0) g[i] = mode ? (T)((double)g[i] + acc) : (T)acc;
    }
}
template <typename T>
void dense_solve(int n, const double *inv, const T *h, T *g, int transpose, int mode, cudaStream_t s) {
    k_dense_gemv<T><<<grid_for((size_t)n * 32, 256), 256, 0, s>>>(n, inv, h, g, transpose, mode);
    CU_LAUNCH("k_dense_gemv"); count_launch();
}
template void dense_solve<double>(int, const double *, const double *, double *, int, int, cudaStream_t);
template void dense_solve<float>(int, const double *, const float *, float *, int, int, cudaStream_t);

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
__global__ void __launch_bounds__(RT) k_mdot(size_t n, int K, const double *__restrict__ w,
                                             const double *__restrict__ V, size_t ldv, double *partials,
                                             unsigned int *ticket, double *h) {
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
__global__ void __launch_bounds__(RT) k_cgs_update(size_t n, int K, const double *__restrict__ hin, double *w,
                                                   const double *__restrict__ V, size_t ldv, int want_dots,
                                                   double *partials, unsigned int *ticket, double *hout) {
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
// apply previous rotations, new rotation, residual estimate.
__global__ void k_givens(FgState *st, int j) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    const int m = st->m;
    double *H = st->H;                       // H[k*m + j]
    for (int k = 0; k <= j; ++k) H[k * m + j] = st->h1[k] + st->h2[k];
    const double hn = sqrt(st->nrm2[0]);
    H[(j + 1) * m + j] = hn;
    st->inv_hn = hn != 0.0 ? 1.0 / hn : 0.0;
    for (int k = 0; k < j; ++k) {
        double a = H[k * m + j], c = H[(k + 1) * m + j];
        H[k * m + j] = st->cs[k] * a + st->sn[k] * c;
        H[(k + 1) * m + j] = -st->sn[k] * a + st->cs[k] * c;
    }
    double a = H[j * m + j], c = H[(j + 1) * m + j];
    double rho = sqrt(a * a + c * c);
    if (!(rho > 0.0) || !isfinite(rho)) {
        st->status = 6;
        st->stop = 1;
        return;
    }
    st->cs[j] = a / rho;
    st->sn[j] = c / rho;
    H[j * m + j] = rho;
    H[(j + 1) * m + j] = 0.0;
    st->s[j + 1] = -st->sn[j] * st->s[j];
    st->s[j] = st->cs[j] * st->s[j];
    st->total += 1;
    const double est = fabs(st->s[j + 1]) / st->bnorm;
    if (st->hist_len < st->hist_cap) st->hist[st->hist_len++] = est;
    st->jdone = j + 1;
    if (!isfinite(est)) { st->status = 6; st->stop = 1; return; }
    if (est <= st->tol || hn == 0.0 || st->total >= st->maxit) st->stop = 1;
}

// V_{j+1} = w * inv_hn
__global__ void k_scale_next(size_t n, const double *__restrict__ w, double *__restrict__ vout, const FgState *st) {
    const double a = st->inv_hn;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
        vout[i] = w[i] * a;
}

// y = H(1:j,1:j)^{-1} s(1:j) (single thread)
__global__ void k_backsolve(FgState *st) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    const int m = st->m, j = st->jdone;
    for (int k = j - 1; k >= 0; --k) {
        double t = st->s[k];
        for (int l = k + 1; l < j; ++l) t -= st->H[k * m + l] * st->y[l];
        st->y[k] = t / st->H[k * m + k];
    }
}

// x += sum_{k<j} y_k Z_k
template <typename ZT>
__global__ void k_update_x(size_t n, const FgState *st, const ZT *__restrict__ Z, size_t ldz, double *x) {
    __shared__ double ys[KMAX1];
    const int j = st->jdone;
    for (int k = threadIdx.x; k < KMAX1; k += blockDim.x) ys[k] = k < j ? st->y[k] : 0.0;
    __syncthreads();
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        double acc = x[i];
        for (int k = 0; k < j; ++k) acc += ys[k] * (double)Z[k * ldz + i];
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
__global__ void __launch_bounds__(RT) k_norm2(size_t n, const double *__restrict__ v, double *partials,
                                              unsigned int *ticket, double *out) {
    double acc[1] = {0.0};
    for (size_t i = blockIdx.x * (size_t)RT + threadIdx.x; i < n; i += (size_t)gridDim.x * RT) acc[0] += v[i] * v[i];
    block_reduce_store<RT>(acc, 1, partials, KMAX1);
    if (last_block(ticket)) {
        final_reduce<RT>(partials, 1, KMAX1, out);
        if (threadIdx.x == 0) *ticket = 0;
    }
}

int reduce_grid() { return sm_count() * 2; }

void mdot(size_t n, int K, const double *w, const double *V, size_t ldv, double *partials, unsigned int *ticket,
          double *h, cudaStream_t s) {
    k_mdot<<<reduce_grid(), RT, 0, s>>>(n, K, w, V, ldv, partials, ticket, h);
    CU_LAUNCH("k_mdot"); count_launch();
}
void cgs_update(size_t n, int K, const double *hin, double *w, const double *V, size_t ldv, int want_dots,
                double *partials, unsigned int *ticket, double *hout, cudaStream_t s) {
    k_cgs_update<<<reduce_grid(), RT, 0, s>>>(n, K, hin, w, V, ldv, want_dots, partials, ticket, hout);
    CU_LAUNCH("k_cgs_update"); count_launch();
}
void norm2(size_t n, const double *v, double *partials, unsigned int *ticket, double *out, cudaStream_t s) {
    k_norm2<<<reduce_grid(), RT, 0, s>>>(n, v, partials, ticket, out);
    CU_LAUNCH("k_norm2"); count_launch();
}
void givens(FgState *st, int j, cudaStream_t s) {
    k_givens<<<1, 32, 0, s>>>(st, j);
    CU_LAUNCH("k_givens"); count_launch();
}
void scale_next(size_t n, const double *w, double *vout, const FgState *st, cudaStream_t s) {
    k_scale_next<<<grid_for(n, 256), 256, 0, s>>>(n, w, vout, st);
    CU_LAUNCH("k_scale_next"); count_launch();
}
void backsolve(FgState *st, cudaStream_t s) {
    k_backsolve<<<1, 32, 0, s>>>(st);
    CU_LAUNCH("k_backsolve"); count_launch();
}

// restart: V_0 = r / beta with beta = sqrt(nrm2); s = beta e1
__global__ void k_restart_scale(size_t n, const double *__restrict__ r, double *__restrict__ v0, FgState *st) {
    const double beta = sqrt(st->nrm2[0]);
    const double a = beta > 0.0 ? 1.0 / beta : 0.0;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
        v0[i] = r[i] * a;
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        for (int k = 0; k <= st->m; ++k) st->s[k] = 0.0;
        st->s[0] = beta;
        st->jdone = 0;
        st->stop = 0;
    }
}
void restart_scale(size_t n, const double *r, double *v0, FgState *st, cudaStream_t s) {
    k_restart_scale<<<grid_for(n, 256), 256, 0, s>>>(n, r, v0, st);
    CU_LAUNCH("k_restart_scale"); count_launch();
}

}  // namespace amg
