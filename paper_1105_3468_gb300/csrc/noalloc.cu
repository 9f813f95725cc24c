// noalloc.cu -- amg_spmv_noalloc: y = A x for callers that cannot allocate
// device memory.
//
// amg_spmv converts the caller's int64 row pointers to an int32 copy in a
// temporary device buffer it allocates per call.  Some callers cannot let a
// library call cudaMalloc/cudaFree:
//   * a serving or training process whose own caching allocator has already
//     reserved the free device memory at start-up: a cudaMalloc from a
//     library then fails, or takes memory the process's budget counts on;
//   * a latency-bound loop that must not stall the whole device: cudaFree
//     synchronises the device, not just the caller's stream.
// For them this entry point keeps that buffer in a file-scope device array
// of fixed size instead, so a call allocates nothing.
//
// Limits and sharing:
//   * At most AMG_NOALLOC_MAX_ROWS rows (the array holds n + 1 int32 row
//     pointers plus one status word: 16 MiB + 512 B, resident on every GPU
//     that loads this library, until the process exits).  Larger matrices
//     are rejected with AMG_ERR_INVALID_ARG.
//   * Every call uses the same array: calls that overlap on the GPU (other
//     streams, other host threads) race on it.  Order such calls on one
//     stream, or serialise them.
//   * The status word is cleared at the start of each call; the row-pointer
//     copy is fully rewritten by each call.
//   * Invalid input cannot make the kernels read outside the caller's
//     buffers: row pointers are clamped to [0, nnz] when they are narrowed,
//     and a column outside [0, n) is skipped and counted in the status word,
//     which the call reads back after synchronising `stream`.
//   * The array's device address is looked up once per device, the first
//     time the entry point runs with that device current.
#include "../../include/amg.h"
#include "solve.cuh"

#include <mutex>

namespace amg {

constexpr int NOALLOC_MAX_ROWS = AMG_NOALLOC_MAX_ROWS;
constexpr int NOALLOC_WORDS = NOALLOC_MAX_ROWS + 1 + 128;   // row pointers, padding, status word
constexpr int NOALLOC_STATUS = NOALLOC_WORDS - 64;

static __device__ __align__(256) int g_noalloc_scratch[NOALLOC_WORDS];

static std::mutex g_noalloc_mu;
static int *g_noalloc_ptr[64];        // per device ordinal; host copies of device addresses

static int *noalloc_scratch_for_current_device() {
    int dev = 0;
    CU(cudaGetDevice(&dev));
    if (dev < 0 || dev >= 64) fail(AMG_ERR_NOT_SUPPORTED, "amg_spmv_noalloc: device ordinal >= 64");
    std::lock_guard<std::mutex> lock(g_noalloc_mu);
    if (!g_noalloc_ptr[dev]) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || !p) {
            cudaGetLastError();
            fail(AMG_ERR_CUDA, std::string("amg_spmv_noalloc: cudaGetSymbolAddress failed: ") +
                                   cudaGetErrorString(e));
        }
        g_noalloc_ptr[dev] = static_cast<int *>(p);
    }
    return g_noalloc_ptr[dev];
}

__global__ void k_noalloc_rp32(int n, int64_t nnz, const int64_t *rp64, int *scratch) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i <= n; i += gridDim.x * blockDim.x) {
        const int64_t v = rp64[i];
        bool ok = v >= 0 && v <= nnz;
        if (i == 0 && v != 0) ok = false;
        if (i == n && v != nnz) ok = false;
        if (i < n && rp64[i + 1] < v) ok = false;
        if (!ok) atomicAdd(scratch + NOALLOC_STATUS, 1);
        scratch[i] = (int)(v < 0 ? 0 : (v > nnz ? nnz : v));   // a bad entry never becomes an index
    }
}

}  // namespace amg

extern const char *amg_noalloc_set_error(const char *msg);

extern "C" int amg_spmv_noalloc(const amg_csr_t *A, const double *x, double *y, void *stream) {
    using namespace amg;
    try {
        if (!A || !x || !y || !A->row_ptr || A->n <= 0 || A->nnz < 0 || (A->nnz > 0 && (!A->col || !A->val)))
            fail(AMG_ERR_INVALID_ARG, "amg_spmv_noalloc: bad argument");
        if (A->n > NOALLOC_MAX_ROWS)
            fail(AMG_ERR_INVALID_ARG, "amg_spmv_noalloc: n exceeds AMG_NOALLOC_MAX_ROWS (4194304); use amg_spmv");
        if (A->nnz >= (int64_t)0x7fffffff) fail(AMG_ERR_INVALID_ARG, "amg_spmv_noalloc: nnz >= 2^31");
        cudaStream_t s = (cudaStream_t)stream;
        int *scratch = noalloc_scratch_for_current_device();
        CU(cudaMemsetAsync(scratch + NOALLOC_STATUS, 0, sizeof(int), s));
        k_noalloc_rp32<<<grid_for((size_t)A->n + 1, 256), 256, 0, s>>>(A->n, A->nnz, A->row_ptr, scratch);
        CU_LAUNCH("k_noalloc_rp32");
        count_launch();
        spmv_f64_checked(A->n, (int)A->nnz, scratch, A->col, A->val, x, y, scratch + NOALLOC_STATUS, s);
        int bad = 0;
        CU(cudaMemcpyAsync(&bad, scratch + NOALLOC_STATUS, sizeof(int), cudaMemcpyDeviceToHost, s));
        CU(cudaStreamSynchronize(s));
        if (bad)
            fail(AMG_ERR_INVALID_ARG,
                 "amg_spmv_noalloc: row pointers not a valid sequence from 0 to nnz, or columns out of range");
        return AMG_OK;
    } catch (const Error &e) {
        amg_noalloc_set_error(e.msg.c_str());
        return e.status;
    } catch (...) {
        amg_noalloc_set_error("amg_spmv_noalloc: unexpected exception");
        return AMG_ERR_CUDA;
    }
}
