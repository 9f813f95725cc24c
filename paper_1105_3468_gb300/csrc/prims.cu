// prims.cu -- deterministic device primitives used by the setup phase:
// exclusive scan, a stable LSD radix sort of (key, value) pairs, fills, and
// the CSR transpose built on the sort.  None of them uses floating-point
// atomics, so every result is independent of scheduling.
#include "internal.cuh"

#include <cstdio>
#include <cstring>
#include <mutex>

namespace amg {

// ------------------------------------------------------------------ errors / memory
static thread_local int64_t t_launches = 0;

void count_launch(int64_t n) { t_launches += n; }
int64_t launch_count() { return t_launches; }

void fail(int status, const std::string &msg) { throw Error{status, msg}; }

void cuda_check(cudaError_t e, const char *what, const char *file, int line) {
    if (e == cudaSuccess) return;
    char buf[512];
    snprintf(buf, sizeof buf, "%s failed: %s (%s:%d)", what, cudaGetErrorString(e), file, line);
    if (e == cudaErrorMemoryAllocation) fail(3, buf);
    fail(2, buf);
}

// The stream of the enclosing AllocScope on this thread (nullptr: none).
static thread_local cudaStream_t t_alloc_stream = nullptr;
static thread_local bool t_alloc_scoped = false;

AllocScope::AllocScope(cudaStream_t s) : prev(t_alloc_stream) {
    t_alloc_stream = s;
    t_alloc_scoped = true;
}
AllocScope::~AllocScope() {
    t_alloc_stream = prev;
    t_alloc_scoped = prev != nullptr;
}

// One pool per device, created on first use.  Up to 1 GiB of freed memory
// stays in the pool between synchronisations; memory freed on one stream is
// reused by another only when its free has already completed (no
// dependencies inserted between the streams).
static cudaMemPool_t pool_for_current_device() {
    static std::mutex mu;
    static cudaMemPool_t pools[64] = {};
    int dev = 0;
    CU(cudaGetDevice(&dev));
    if (dev < 0 || dev >= 64) fail(4, "memory pool: device ordinal >= 64");
    std::lock_guard<std::mutex> lock(mu);
    if (!pools[dev]) {
        cudaMemPoolProps props = {};
        props.allocType = cudaMemAllocationTypePinned;
        props.location.type = cudaMemLocationTypeDevice;
        props.location.id = dev;
        CU(cudaMemPoolCreate(&pools[dev], &props));
        uint64_t keep = 1ull << 30;
        CU(cudaMemPoolSetAttribute(pools[dev], cudaMemPoolAttrReleaseThreshold, &keep));
        int off = 0;
        CU(cudaMemPoolSetAttribute(pools[dev], cudaMemPoolReuseAllowInternalDependencies, &off));
    }
    return pools[dev];
}

void *dmalloc(size_t bytes, bool *pooled) {
    void *p = nullptr;
    cudaError_t e;
    if (t_alloc_scoped && t_alloc_stream) {
        e = cudaMallocFromPoolAsync(&p, bytes, pool_for_current_device(), t_alloc_stream);
        *pooled = true;
    } else {
        e = cudaMalloc(&p, bytes);
        *pooled = false;
    }
    if (e != cudaSuccess) {
        cudaGetLastError();
        char buf[160];
        snprintf(buf, sizeof buf, "device allocation (%zu bytes): %s", bytes, cudaGetErrorString(e));
        fail(e == cudaErrorMemoryAllocation ? 3 : 2, buf);
    }
    return p;
}

void dfree(void *p, bool pooled) {
    if (pooled && t_alloc_scoped && t_alloc_stream) cudaFreeAsync(p, t_alloc_stream);
    else cudaFree(p);
}

int sm_count() {
    static const int sms = [] {               // initialised once, thread-safe
        int dev = 0, v = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev);
        return v > 0 ? v : 1;
    }();
    return sms;
}

int grid_for(size_t n, int tpb) {
    size_t b = (n + tpb - 1) / tpb;
    if (b < 1) b = 1;
    const size_t cap = (size_t)sm_count() * 32;
    return (int)(b < cap ? b : cap);
}

// ------------------------------------------------------------------ fills
__global__ void k_iota(int *p, int n) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) p[i] = i;
}
__global__ void k_fill_int(int *p, int v, int n) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) p[i] = v;
}
__global__ void k_fill_double(double *p, double v, size_t n) {
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) p[i] = v;
}

void iota_int(int *p, int n, cudaStream_t s) {
    if (n <= 0) return;
    k_iota<<<grid_for(n, 256), 256, 0, s>>>(p, n);
    CU_LAUNCH("k_iota"); count_launch();
}
void fill_int(int *p, int v, int n, cudaStream_t s) {
    if (n <= 0) return;
    k_fill_int<<<grid_for(n, 256), 256, 0, s>>>(p, v, n);
    CU_LAUNCH("k_fill_int"); count_launch();
}
void fill_double(double *p, double v, size_t n, cudaStream_t s) {
    if (n == 0) return;
    k_fill_double<<<grid_for(n, 256), 256, 0, s>>>(p, v, n);
    CU_LAUNCH("k_fill_double"); count_launch();
}

// ------------------------------------------------------------------ exclusive scan (int32)
// One tile = 1024 threads x 4 items.  Block totals are scanned recursively.
constexpr int SCAN_T = 1024, SCAN_I = 4, SCAN_TILE = SCAN_T * SCAN_I;

__global__ void __launch_bounds__(SCAN_T) k_scan_tile(const int *in, int *out, int *bsum, int n) {
    __shared__ int wsum[32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const long base = (long)blockIdx.x * SCAN_TILE + (long)threadIdx.x * SCAN_I;
    int v[SCAN_I], s = 0;
#pragma unroll
    for (int k = 0; k < SCAN_I; ++k) {
        long idx = base + k;
        v[k] = idx < n ? in[idx] : 0;
        s += v[k];
    }
    int x = s;
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
        int y = __shfl_up_sync(0xffffffffu, x, off);
        if (lane >= off) x += y;
    }
    if (lane == 31) wsum[warp] = x;
    __syncthreads();
    if (warp == 0) {
        int w = lane < (SCAN_T / 32) ? wsum[lane] : 0;
#pragma unroll
        for (int off = 1; off < 32; off <<= 1) {
            int y = __shfl_up_sync(0xffffffffu, w, off);
            if (lane >= off) w += y;
        }
        wsum[lane] = w;
    }
    __syncthreads();
    int run = x - s + (warp > 0 ? wsum[warp - 1] : 0);
#pragma unroll
    for (int k = 0; k < SCAN_I; ++k) {
        long idx = base + k;
        if (idx < n) out[idx] = run;
        run += v[k];
    }
    if (threadIdx.x == SCAN_T - 1) bsum[blockIdx.x] = run;
}

__global__ void __launch_bounds__(SCAN_T) k_scan_add(int *out, const int *boff, int n) {
    const long base = (long)blockIdx.x * SCAN_TILE + (long)threadIdx.x * SCAN_I;
    const int add = boff[blockIdx.x];
#pragma unroll
    for (int k = 0; k < SCAN_I; ++k)
        if (base + k < n) out[base + k] += add;
}

// out = exclusive scan of in; *dtotal (device) = sum.
static void scan_rec(const int *in, int *out, int n, int *dtotal, cudaStream_t s) {
    const int nb = (n + SCAN_TILE - 1) / SCAN_TILE;
    if (nb <= 1) {
        k_scan_tile<<<1, SCAN_T, 0, s>>>(in, out, dtotal, n);
        CU_LAUNCH("k_scan_tile"); count_launch();
        return;
    }
    DBuf<int> bsum(nb), boff(nb);
    k_scan_tile<<<nb, SCAN_T, 0, s>>>(in, out, bsum.get(), n);
    CU_LAUNCH("k_scan_tile"); count_launch();
    scan_rec(bsum.get(), boff.get(), nb, dtotal, s);
    k_scan_add<<<nb, SCAN_T, 0, s>>>(out, boff.get(), n);
    CU_LAUNCH("k_scan_add"); count_launch();
}

void exclusive_scan_int(const int *in, int *out, int n, int *total_host, cudaStream_t s) {
    DBuf<int> dtot(1);
    if (n <= 0) {
        if (total_host) *total_host = 0;
        return;
    }
    scan_rec(in, out, n, dtot.get(), s);
    if (total_host) {
        CU(cudaMemcpyAsync(total_host, dtot.get(), sizeof(int), cudaMemcpyDeviceToHost, s));
        CU(cudaStreamSynchronize(s));
    }
}

// ------------------------------------------------------------------ stable radix sort
// LSD, 8-bit digits.  A block owns a tile of RS_ROUNDS x 256 consecutive
// elements and walks it round by round; inside a round, lanes of a warp are
// ranked with __match_any_sync and warps in order, so equal digits keep
// their input order (stability), independent of scheduling.
constexpr int RS_T = 256, RS_ROUNDS = 8, RS_TILE = RS_T * RS_ROUNDS, RS_W = RS_T / 32;

__global__ void __launch_bounds__(RS_T) k_rs_hist(const uint32_t *keys, int n, int shift, int *hist,
                                                  int nblocks) {
    __shared__ int h[256];
    h[threadIdx.x] = 0;
    __syncthreads();
    const long base = (long)blockIdx.x * RS_TILE;
    for (int r = 0; r < RS_ROUNDS; ++r) {
        long idx = base + (long)r * RS_T + threadIdx.x;
        if (idx < n) atomicAdd(&h[(keys[idx] >> shift) & 255u], 1);
    }
    __syncthreads();
    hist[(long)threadIdx.x * nblocks + blockIdx.x] = h[threadIdx.x];
}

__global__ void __launch_bounds__(RS_T) k_rs_scatter(const uint32_t *kin, const int *vin, uint32_t *kout,
                                                     int *vout, int n, int shift, const int *offs,
                                                     int nblocks) {
    __shared__ int run[256];             // elements of each digit placed so far in this tile
    __shared__ int wcnt[RS_W][256];      // per-warp digit counts of the current round
    __shared__ int goff[256];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    run[threadIdx.x] = 0;
    goff[threadIdx.x] = offs[(long)threadIdx.x * nblocks + blockIdx.x];
    for (int w = 0; w < RS_W; ++w) wcnt[w][threadIdx.x] = 0;
    __syncthreads();
    const long base = (long)blockIdx.x * RS_TILE;
    for (int r = 0; r < RS_ROUNDS; ++r) {
        long idx = base + (long)r * RS_T + threadIdx.x;
        bool valid = idx < n;
        uint32_t key = valid ? kin[idx] : 0u;
        int val = valid ? vin[idx] : 0;
        int d = valid ? (int)((key >> shift) & 255u) : 256 + lane;   // invalid lanes never match
        unsigned peers = __match_any_sync(0xffffffffu, d);
        int rank_in_warp = __popc(peers & ((1u << lane) - 1u));
        if (valid && rank_in_warp == 0) wcnt[warp][d] = __popc(peers);
        __syncthreads();
        // per digit: exclusive prefix over warps, then advance the running count
        {
            int dd = threadIdx.x;
            int acc = run[dd];
            for (int w = 0; w < RS_W; ++w) {
                int c = wcnt[w][dd];
                wcnt[w][dd] = acc;
                acc += c;
            }
            run[dd] = acc;
        }
        __syncthreads();
        if (valid) {
            long dst = (long)goff[d] + wcnt[warp][d] + rank_in_warp;
            kout[dst] = key;
            vout[dst] = val;
        }
        __syncthreads();
        for (int w = 0; w < RS_W; ++w) wcnt[w][threadIdx.x] = 0;
        __syncthreads();
    }
}

// Sorts (keys, vals) by keys (stable); key_bits = significant low bits.
void radix_sort_pairs(uint32_t *keys, int *vals, int n, int key_bits, cudaStream_t s) {
    if (n <= 1) return;
    const int nblocks = (n + RS_TILE - 1) / RS_TILE;
    DBuf<uint32_t> k2(n);
    DBuf<int> v2(n), hist((size_t)256 * nblocks), offs((size_t)256 * nblocks);
    uint32_t *ka = keys, *kb = k2.get();
    int *va = vals, *vb = v2.get();
    int passes = (key_bits + 7) / 8;
    if (passes < 1) passes = 1;
    for (int p = 0; p < passes; ++p) {
        const int shift = 8 * p;
        k_rs_hist<<<nblocks, RS_T, 0, s>>>(ka, n, shift, hist.get(), nblocks);
        CU_LAUNCH("k_rs_hist"); count_launch();
        exclusive_scan_int(hist.get(), offs.get(), 256 * nblocks, nullptr, s);
        k_rs_scatter<<<nblocks, RS_T, 0, s>>>(ka, va, kb, vb, n, shift, offs.get(), nblocks);
        CU_LAUNCH("k_rs_scatter"); count_launch();
        std::swap(ka, kb);
        std::swap(va, vb);
    }
    if (ka != keys) {
        CU(cudaMemcpyAsync(keys, ka, sizeof(uint32_t) * n, cudaMemcpyDeviceToDevice, s));
        CU(cudaMemcpyAsync(vals, va, sizeof(int) * n, cudaMemcpyDeviceToDevice, s));
    }
    CU(cudaStreamSynchronize(s));   // temporaries are freed on return
}

int bits_for(uint32_t maxval) {
    int b = 0;
    while (b < 32 && (maxval >> b) != 0) ++b;
    return b < 1 ? 1 : b;
}

// ------------------------------------------------------------------ transpose
__global__ void k_row_ids(const int *rp, int n, int *rid) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
        for (int e = rp[i]; e < rp[i + 1]; ++e) rid[e] = i;
}
__global__ void k_keys_from_int(const int *a, uint32_t *k, int n) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) k[i] = (uint32_t)a[i];
}
__global__ void k_count_keys(const uint32_t *k, int n, int *cnt) {
    // integer histogram: the counts do not depend on the order of the atomics
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) atomicAdd(cnt + k[i], 1);
}
__global__ void k_gather_int(const int *src, const int *idx, int *dst, int n) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) dst[i] = src[idx[i]];
}

void gather_int(const int *src, const int *idx, int *dst, int n, cudaStream_t s) {
    if (n <= 0) return;
    k_gather_int<<<grid_for(n, 256), 256, 0, s>>>(src, idx, dst, n);
    CU_LAUNCH("k_gather_int"); count_launch();
}

// Segment pointers of a sorted key array over [0, nseg): ptr[s]..ptr[s+1].
void segment_ptr(const uint32_t *sorted_keys, int n, int nseg, DBuf<int> &ptr, cudaStream_t s) {
    DBuf<int> cnt(nseg + 1);
    fill_int(cnt.get(), 0, nseg + 1, s);
    if (n > 0) {
        k_count_keys<<<grid_for(n, 256), 256, 0, s>>>(sorted_keys, n, cnt.get());
        CU_LAUNCH("k_count_keys"); count_launch();
    }
    ptr.alloc(nseg + 1);
    exclusive_scan_int(cnt.get(), ptr.get(), nseg + 1, nullptr, s);
}

void csr_transpose(int n, int nnz, const int *rp, const int *ci, DBuf<int> &trp, DBuf<int> &tci,
                   DBuf<int> &tsrc, cudaStream_t s) {
    DBuf<uint32_t> keys(nnz > 0 ? nnz : 1);
    DBuf<int> rid(nnz > 0 ? nnz : 1);
    tsrc.alloc(nnz > 0 ? nnz : 1);
    tci.alloc(nnz > 0 ? nnz : 1);
    if (nnz > 0) {
        k_keys_from_int<<<grid_for(nnz, 256), 256, 0, s>>>(ci, keys.get(), nnz);
        CU_LAUNCH("k_keys_from_int"); count_launch();
        iota_int(tsrc.get(), nnz, s);
        radix_sort_pairs(keys.get(), tsrc.get(), nnz, bits_for((uint32_t)n), s);
        k_row_ids<<<grid_for(n, 256), 256, 0, s>>>(rp, n, rid.get());
        CU_LAUNCH("k_row_ids"); count_launch();
        k_gather_int<<<grid_for(nnz, 256), 256, 0, s>>>(rid.get(), tsrc.get(), tci.get(), nnz);
        CU_LAUNCH("k_gather_int"); count_launch();
    }
    segment_ptr(keys.get(), nnz, n, trp, s);
    CU(cudaStreamSynchronize(s));
}

}  // namespace amg
