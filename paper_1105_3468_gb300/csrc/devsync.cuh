// devsync.cuh -- device helpers shared by the solve-phase kernels: value
// conversion, the fused multiply-subtract every row sum uses, the bounded
// grid barrier of cooperative launches and the sentinel loads and stores of
// the dataflow and tiled sweeps.
#pragma once

#include <cuda_bf16.h>

namespace amg {

template <typename T, typename V> __device__ __forceinline__ T val_as(V x);
template <> __device__ __forceinline__ double val_as<double, double>(double x) { return x; }
template <> __device__ __forceinline__ float val_as<float, float>(float x) { return x; }
template <> __device__ __forceinline__ float val_as<float, __nv_bfloat16>(__nv_bfloat16 x) { return __bfloat162float(x); }
template <> __device__ __forceinline__ double val_as<double, float>(float x) { return (double)x; }

// acc - a*b and acc + a*b as one fused multiply-add (a single rounding):
// every multiply-accumulate of the solve phase rounds this way, in FP64 as
// in FP32, so a row summed in stored order reproduces the sequential
// definition bit for bit.
__device__ __forceinline__ double msub(double acc, double a, double b) { return __fma_rn(-a, b, acc); }
__device__ __forceinline__ float msub(float acc, float a, float b) { return __fmaf_rn(-a, b, acc); }
__device__ __forceinline__ double madd(double acc, double a, double b) { return __fma_rn(a, b, acc); }
__device__ __forceinline__ float madd(float acc, float a, float b) { return __fmaf_rn(a, b, acc); }

// Grid barrier for a cooperative launch (all blocks resident).  bar[0]
// counts arrivals, bar[1] is the generation.  A wait gives up after
// SPIN_LIMIT polls and sets *err; once *err is set every later barrier
// returns at once, so the kernel always terminates.
constexpr unsigned int SPIN_LIMIT = 1u << 22;

__device__ __forceinline__ unsigned int ld_acquire_gpu(const unsigned int *p) {
    unsigned int v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ void grid_barrier(unsigned int *bar, int *err) {
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned int gen, arrived;
        asm volatile("ld.relaxed.gpu.global.u32 %0, [%1];" : "=r"(gen) : "l"(bar + 1) : "memory");
        // arrival releases this block's writes (ordered before by bar.sync) and
        // acquires those of the blocks that arrived earlier
        asm volatile("atom.acq_rel.gpu.global.add.u32 %0, [%1], 1;" : "=r"(arrived) : "l"(bar) : "memory");
        if (arrived + 1u == gridDim.x) {
            asm volatile("st.relaxed.gpu.global.u32 [%0], %1;" ::"l"(bar), "r"(0u) : "memory");
            asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(bar + 1), "r"(gen + 1u) : "memory");
        } else {
            unsigned int spins = 0;
            while (ld_acquire_gpu(bar + 1) == gen) {
                if (*(volatile int *)err) break;
                if (++spins > SPIN_LIMIT) { atomicExch(err, 1); break; }
                if (spins > 64) __nanosleep(20);
            }
        }
    }
    __syncthreads();
}

template <typename T> struct Sentinel;
template <> struct Sentinel<float> {
    static __device__ __forceinline__ unsigned int bits() { return 0x7fa5a5a5u; }
    static __device__ __forceinline__ bool is(float x) { return __float_as_uint(x) == bits(); }
    static __device__ __forceinline__ float value() { return __uint_as_float(bits()); }
    static __device__ __forceinline__ float ld(const float *p) {
        unsigned int u;
        asm volatile("ld.relaxed.gpu.global.u32 %0, [%1];" : "=r"(u) : "l"(p) : "memory");
        return __uint_as_float(u);
    }
    static __device__ __forceinline__ void st(float *p, float x) {
        unsigned int u = __float_as_uint(x);
        if (u == bits()) u = 0x7fffffffu;
        asm volatile("st.relaxed.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(u) : "memory");
    }
};
template <> struct Sentinel<double> {
    static __device__ __forceinline__ unsigned long long bits() { return 0x7ff4a5a5a5a5a5a5ull; }
    static __device__ __forceinline__ bool is(double x) { return (unsigned long long)__double_as_longlong(x) == bits(); }
    static __device__ __forceinline__ double value() { return __longlong_as_double((long long)bits()); }
    static __device__ __forceinline__ double ld(const double *p) {
        unsigned long long u;
        asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(u) : "l"(p) : "memory");
        return __longlong_as_double((long long)u);
    }
    static __device__ __forceinline__ void st(double *p, double x) {
        unsigned long long u = (unsigned long long)__double_as_longlong(x);
        if (u == bits()) u = 0x7fffffffffffffffull;
        asm volatile("st.relaxed.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(u) : "memory");
    }
};

}  // namespace amg
