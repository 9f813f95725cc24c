// internal.cuh -- shared declarations of libamg_gb's CUDA translation units.
//
// Layout conventions (all device memory):
//   * Matrices are CSR with int32 row pointers (nnz < 2^31 is enforced at
//     the ABI), int32 columns ascending within a row, and values in FP64
//     (setup and the FP64 paths) plus optional FP32/BF16 copies.
//   * Vectors of level l are in natural row order.
//   * ILU(0) factors are stored twice for the sweeps: the L part of each row
//     (strictly before the row in the elimination order) in forward-schedule
//     row order, and the U part (strictly after) plus the diagonal in
//     backward-schedule row order.  A schedule level holds rows whose
//     dependencies all lie in earlier levels; rows of a level are ascending.
#pragma once

#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <stdint.h>

#include <string>
#include <vector>

namespace amg {

// ------------------------------------------------------------------ errors
struct Error {
    int status;
    std::string msg;
};

[[noreturn]] void fail(int status, const std::string &msg);
void cuda_check(cudaError_t e, const char *what, const char *file, int line);
#define CU(call) ::amg::cuda_check((call), #call, __FILE__, __LINE__)
#define CU_LAUNCH(what) ::amg::cuda_check(cudaGetLastError(), what, __FILE__, __LINE__)

// Count of kernels launched by the library (for the launch statistics).
void count_launch(int64_t n = 1);
int64_t launch_count();

// ------------------------------------------------------------------ memory
// Device allocation with an OOM status instead of an exception type.
// Inside an AllocScope (a setup on one stream), allocations come from the
// library's stream-ordered memory pool on the scope's stream and frees are
// stream-ordered on it: no device-wide synchronisation, so setups of many
// systems on their own streams (a batch) overlap.  Outside a scope, plain
// cudaMalloc / cudaFree.  A pooled buffer freed outside a scope is freed by
// cudaFree, which does not wait: its owner synchronises first (handles do
// before they release their buffers).
void *dmalloc(size_t bytes, bool *pooled);
void dfree(void *p, bool pooled);
struct AllocScope {
    cudaStream_t prev;
    explicit AllocScope(cudaStream_t s);
    ~AllocScope();
};

template <typename T>
struct DBuf {
    T *p = nullptr;
    size_t n = 0;
    bool pooled = false;
    DBuf() = default;
    explicit DBuf(size_t count) { alloc(count); }
    DBuf(const DBuf &) = delete;
    DBuf &operator=(const DBuf &) = delete;
    DBuf(DBuf &&o) noexcept : p(o.p), n(o.n), pooled(o.pooled) { o.p = nullptr; o.n = 0; o.pooled = false; }
    DBuf &operator=(DBuf &&o) noexcept {
        if (this != &o) {
            release();
            p = o.p; n = o.n; pooled = o.pooled;
            o.p = nullptr; o.n = 0; o.pooled = false;
        }
        return *this;
    }
    ~DBuf() { release(); }
    void alloc(size_t count) {
        release();
        n = count;
        p = count ? static_cast<T *>(dmalloc(count * sizeof(T), &pooled)) : nullptr;
    }
    void release() { if (p) dfree(p, pooled); p = nullptr; n = 0; pooled = false; }
    T *get() const { return p; }
    size_t bytes() const { return n * sizeof(T); }
};

// ------------------------------------------------------------------ device CSR
struct DCsr {
    int n = 0;
    int nnz = 0;
    DBuf<int> rp;       // [n+1]
    DBuf<int> ci;       // [nnz]
    DBuf<double> v;     // [nnz]
};

// SELL-32 copy of a CSR matrix: slices of 32 consecutive rows, each slice
// padded to its longest row and stored column-major (entry k of row r of
// slice s at ptr[s] + 32 k + r), so a warp's load of entry k is contiguous.
// Padding repeats the row's diagonal column with value 0.
struct Sell {
    int n = 0, nslices = 0;
    int64_t padded = 0;
    DBuf<int64_t> ptr;      // [nslices + 1]
    DBuf<int> ci;           // [padded]
    DBuf<double> v;         // [padded]
    int block = 256, unroll = 4;   // launch geometry of the SpMV (autotuned at setup)
};
void build_sell(const DCsr &A, const double *vals, Sell &S, cudaStream_t s);

// Row-scheduled triangular factor for one sweep direction.
struct Sweep {
    int nlev = 0;                   // schedule levels
    std::vector<int> lev_ptr;       // host copy [nlev+1] into rows
    DBuf<int> dlev;                 // device copy of lev_ptr
    DBuf<int> rows;                 // [n] row ids in schedule order
    DBuf<int> rp;                   // [n+1] entries of rows[k] at rp[k]..rp[k+1]
    DBuf<int> ci;                   // [nnzf] column ids
    DBuf<double> v64;               // [nnzf]
    DBuf<float> v32;
    DBuf<__nv_bfloat16> v16;
    DBuf<double> d64;               // backward only: diagonal u_ii per schedule position
    DBuf<float> d32;
    int maxlev = 0;                 // widest level
};

// ------------------------------------------------------------------ kernels: primitives
void exclusive_scan_int(const int *in, int *out, int n, int *total_host, cudaStream_t s);
void iota_int(int *p, int n, cudaStream_t s);
void fill_int(int *p, int v, int n, cudaStream_t s);
void fill_double(double *p, double v, size_t n, cudaStream_t s);

// Stable LSD radix sort of (key, value) pairs by the low key_bits bits.
void radix_sort_pairs(uint32_t *keys, int *vals, int n, int key_bits, cudaStream_t s);
int bits_for(uint32_t maxval);
// dst[i] = src[idx[i]]
void gather_int(const int *src, const int *idx, int *dst, int n, cudaStream_t s);
// Segment pointers [nseg+1] of a sorted key array.
void segment_ptr(const uint32_t *sorted_keys, int n, int nseg, DBuf<int> &ptr, cudaStream_t s);

// CSR transpose (pattern + the source position of each transposed entry),
// rows of the transpose ascending.  Allocates outputs.
void csr_transpose(int n, int nnz, const int *rp, const int *ci, DBuf<int> &trp, DBuf<int> &tci,
                   DBuf<int> &tsrc, cudaStream_t s);

// ------------------------------------------------------------------ kernels: setup
// Validates a CSR (columns in range, strictly ascending, diagonal present).
// Returns the number of bad rows.
int csr_validate(int n, const int *rp, const int *ci, cudaStream_t s);

// Symmetrised off-diagonal adjacency of the pattern (A + A^T, no diagonal).
void sym_adjacency(const DCsr &A, DBuf<int> &arp, DBuf<int> &aci, int &annz, cudaStream_t s);

// One heavy-edge matching pass; mate[u] = partner or -1.  scaled: edge
// weights divided by the geometric mean of their endpoints' diagonal
// magnitudes.
// Returns rounds or throws AMG_ERR_LIMIT.
int match_pass(const DCsr &A, const int *arp, const int *aci, int annz, uint64_t seed, int scaled,
               int *mate, cudaStream_t s);

// Aggregates from a matching: agg[u], returns N_c.
int aggregates_from_mate(int n, const int *mate, int *agg, cudaStream_t s);

// members CSR of a map agg: ptr [nc+1], idx [n] ascending within an aggregate.
void members_of(int n, int nc, const int *agg, DBuf<int> &ptr, DBuf<int> &idx, cudaStream_t s);

// Galerkin product of A by the aggregation (agg, members): fills C.
void galerkin(const DCsr &A, int nc, const int *agg, const int *mptr, const int *midx, DCsr &C,
              cudaStream_t s);

// Greedy colouring by Jones-Plassmann rounds; returns colours.
int color_jp(int n, const int *arp, const int *aci, int mode, uint64_t seed, int *color,
             cudaStream_t s);

// Elimination positions pos[i] = rank of (label[i], i).
void elimination_positions(int n, const int *label, int nlabels, int *pos, cudaStream_t s);

// ILU(0) in the elimination order given by pos; lu receives the factors on
// A's layout.  Also builds the forward/backward sweep schedules.
void ilu0_factor(const DCsr &A, const int *pos, DBuf<double> &lu, Sweep &fwd, Sweep &bwd,
                 cudaStream_t s);

// Sweep schedules of factors already computed on the pattern of F (values lu
// on F's layout; L part: pos(j) < pos(i), U part with the diagonal).
void factor_sweeps(const DCsr &F, const int *pos, const double *lu, Sweep &fwd, Sweep &bwd, cudaStream_t s);

// ILUT(tau) of a host CSR matrix (ilut.cu): rows of L~ (unit diagonal implied)
// then U~, ascending columns.  Returns false on a zero or non-finite pivot.
bool ilut_factor_host(int n, const int64_t *rp, const int32_t *ci, const double *val, double tau,
                      std::vector<int64_t> &frp, std::vector<int32_t> &fci, std::vector<double> &fv);

// Dense inverse (Gauss-Jordan with partial pivoting, FP64) of a CSR matrix.
void dense_inverse(const DCsr &A, DBuf<double> &inv, cudaStream_t s);

// Casts
void cast_f64_f32(const double *in, float *out, size_t n, cudaStream_t s);
void cast_f64_bf16(const double *in, __nv_bfloat16 *out, size_t n, cudaStream_t s);

// FV assembly / gradient (device pointers).
int64_t fv_assemble(int dim, int nx, int ny, int nz, const double *kx, const double *ky,
                    const double *kz, const double *fx, const double *fy, const double *fz,
                    const double *f, int64_t *rp, int *ci, double *v, double *b, cudaStream_t s);
// gy == nullptr: isotropic conductivity kx per cell; gx receives the
// derivative with respect to log kx (the sum of the three axis terms).
void fv_grad_logk(int dim, int nx, int ny, int nz, const double *kx, const double *ky,
                  const double *kz, const double *lam, const double *x, double *gx, double *gy,
                  double *gz, cudaStream_t s);
void exp_f64(long n, const double *in, double *out, cudaStream_t s);

// ------------------------------------------------------------------ kernels: solve
// Grid sizing helper: blocks for n items at `tpb` threads, capped to a
// multiple of the SM count.
int grid_for(size_t n, int tpb);
int sm_count();

}  // namespace amg
