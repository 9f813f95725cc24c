// sell_residual.cu -- the V-cycle's forward residual r = b - A x of a larger
// level from a SELL-32 copy of its matrix (slices of 32 rows, column-major
// inside a slice): each thread sums its row's terms in stored order, one
// fused multiply-add each, as the CSR residual does, but a warp's loads of
// values and columns are contiguous.  The padding terms (value 0) add 0 x:
// they leave every nonzero partial sum unchanged.
#include "solve.cuh"
#include "devsync.cuh"

namespace amg {

template <typename T, typename V>
__global__ void __launch_bounds__(256) k_residual_sell(int n, const int64_t *__restrict__ ptr,
                                                       const int *__restrict__ ci, const V *__restrict__ v,
                                                       const T *__restrict__ x, const T *__restrict__ b,
                                                       T *__restrict__ r) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const int sl = i >> 5, lane = i & 31;
        const int64_t base = ptr[sl];
        const int w = (int)((ptr[sl + 1] - base) >> 5);
        const V *vv = v + base + lane;
        const int *cc = ci + base + lane;
        T acc = T(0);
#pragma unroll 4
        for (int k = 0; k < w; ++k) acc = madd(acc, val_as<T, V>(__ldg(vv + 32 * k)), x[__ldg(cc + 32 * k)]);
        r[i] = b[i] - acc;
    }
}

template <typename T, typename V>
void level_residual_sell(int n, const int64_t *ptr, const int *ci, const V *v, const T *x, const T *b, T *r,
                         cudaStream_t s) {
    if (n <= 0) return;
    k_residual_sell<T, V><<<grid_for(n, 256), 256, 0, s>>>(n, ptr, ci, v, x, b, r);
    CU_LAUNCH("k_residual_sell"); count_launch();
}
template void level_residual_sell<double, double>(int, const int64_t *, const int *, const double *, const double *,
                                                  const double *, double *, cudaStream_t);
template void level_residual_sell<float, float>(int, const int64_t *, const int *, const float *, const float *,
                                                const float *, float *, cudaStream_t);

}  // namespace amg
