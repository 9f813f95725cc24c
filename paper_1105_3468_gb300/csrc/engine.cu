// engine.cu -- the C ABI of libamg_gb (include/amg.h): the handle, the
// setup pipeline (Algorithm 1, setup, applied level by level), the
// recursive preconditioner (Algorithm 1, the two-grid and coarse-solve applications,
// with the inexact coarse solve read as Richardson steps preconditioned by
// the coarse level's own two-grid construction), and right-preconditioned
// FGMRES(m) (Algorithm 1, Krylov iteration, flexible form).
#include "../../include/amg.h"
#include "solve.cuh"
#include <type_traits>

#include <atomic>
#include <chrono>
#include <cmath>
#include <thread>
#include <cstdio>
#include <cstring>
#include <memory>
#include <string>
#include <vector>

namespace amg {

static thread_local std::string t_last_error;

// ------------------------------------------------------------------ level data
struct PassData {
    DCsr mat;            // Galerkin product after this pass (except the last pass)
    DBuf<int> agg;       // map of this pass
    int n_in = 0, n_out = 0;
};

struct Level {
    DCsr A;                                   // FP64
    DBuf<float> v32;
    DBuf<__nv_bfloat16> v16;
    // transposed matrix (adjoint)
    DCsr AT;
    DBuf<float> vt32;
    DBuf<__nv_bfloat16> vt16;
    // aggregation to the next level
    std::vector<PassData> passes;
    DBuf<int> agg, mptr, midx;
    int n_next = -1;
    // smoother
    int order = AMG_ORDER_COLOR, ncol = 0;
    DBuf<int> label, pos;
    DBuf<double> lu;
    Sweep fwd, bwd, fwdT, bwdT;
    // level 1 of the ILUT two-grid: the factors' pattern (values in lu)
    bool ilut_level = false;
    DCsr fpat;
    // dense last level
    bool dense = false;
    DBuf<double> inv;
    DBuf<float> inv32;                    // FP32 copy for the FP32 / BF16 V-cycles
    // SELL-32 copies for the outer FP64 SpMV (level 0 only)
    Sell sell, sellT;
    // SELL-32 copy for the V-cycle's forward residual of a level with at
    // least RSELL_MIN rows (FP64 values in the FP64 V-cycle, else FP32 in rsv32)
    Sell rsell;
    DBuf<float> rsv32;
    // workspace (vector type of the V-cycle, allocated as bytes)
    DBuf<char> wt, wy, wr, wres, wh, wg, wf;
    int wy_sent = 0;                      // element size of the sentinel wy holds (dataflow sweeps), 0: none
    // the smoother in grid tiles (finest level, natural-order stencil, persistent 5)
    std::unique_ptr<TilePlan> tiles;
    int sweep_kind[2] = {-1, -1};         // smoother variant of the last application (SWEEP_KIND_*), forward / transposed
};

}  // namespace amg

struct amg_handle {
    amg_options_t opt;
    cudaStream_t stream = nullptr;        // internal non-blocking stream (all library work)
    cudaStream_t ustream = nullptr;       // the caller's stream given to amg_setup
    cudaEvent_t entry_ev = nullptr;
    std::vector<std::unique_ptr<amg::Level>> lev;
    int n = 0;
    // FGMRES storage
    amg::DBuf<double> V, Zd, w, r, xb, bb, hist, partials, zin64, zout64;
    amg::DBuf<float> Zf, zin32, zout32;
    int *hflags = nullptr;                // pinned: stop flag, status
    cudaGraphExec_t gexec[2] = {nullptr, nullptr};   // inner iteration (solve, adjoint)
    // device-driven solve loop (graph conditional nodes): the whole FGMRES
    // loop of this handle (lexec) or of all members of a batch (bexec)
    cudaGraphExec_t lexec[2] = {nullptr, nullptr};
    cudaGraphExec_t bexec[2] = {nullptr, nullptr};
    int64_t loop_nodes[2][2] = {{0, 0}, {0, 0}};   // kernels per pass and per cycle end
    cudaStream_t aux = nullptr;           // captures the cycle-end body
    size_t gpairs[2] = {0, 0};            // timing event pairs recorded by each graph
    int64_t gnodes[2] = {0, 0};           // kernels in each graph
    double gbytes[2] = {0.0, 0.0};        // timed-class bytes of one replay
    amg::DBuf<amg::FgState> st;
    amg::DBuf<unsigned int> ticket, bar;   // reduction ticket; grid-barrier words
    amg::DBuf<int> err;                      // set when a device wait gives up
    amg::FgState *hst = nullptr;          // pinned host mirror
    std::vector<double> last_hist;
    double setup_ms = 0.0;
    bool adjoint_ready = false;
    int deep_first = 1 << 30;             // first level run by the single-block V-cycle
    std::vector<amg_handle *> subs;       // batch: one handle per system
    std::vector<int64_t> offs;            // batch: row offsets of the systems [count+1]
    amg::DBuf<char> deep_desc;            // DeepLevel<T, V>[nlev - deep_first]
    // kernel timing of one kernel class (CUDA events around each launch)
    int tclass = 0;
    std::vector<std::pair<cudaEvent_t, cudaEvent_t>> tev;
    size_t tused = 0;
    double t_ms = 0.0, t_bytes = 0.0;
    int64_t t_launches = 0;
    double t_bytes_per_launch = 0.0;
};

namespace amg {

// ------------------------------------------------------------------ helpers
static bool is_device_ptr(const void *p) {
    if (!p) return false;
    cudaPointerAttributes a;
    cudaError_t e = cudaPointerGetAttributes(&a, p);
    if (e != cudaSuccess) { cudaGetLastError(); return false; }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

// Orders the handle's internal stream after the work already queued on the
// caller's stream (inputs may still be in flight there).
static void enter(amg_handle *h) {
    CU(cudaEventRecord(h->entry_ev, h->ustream));
    CU(cudaStreamWaitEvent(h->stream, h->entry_ev, 0));
}

template <typename T>
static const T *to_device(const T *p, size_t n, DBuf<T> &tmp, cudaStream_t s) {
    if (is_device_ptr(p)) return p;
    tmp.alloc(n ? n : 1);
    if (n) CU(cudaMemcpyAsync(tmp.get(), p, n * sizeof(T), cudaMemcpyHostToDevice, s));
    return tmp.get();
}

__global__ void k_rp64_to_32(int n, int64_t nnz, const int64_t *rp64, int *rp32, int *bad) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i <= n; i += gridDim.x * blockDim.x) {
        int64_t v = rp64[i];
        bool ok = v >= 0 && v <= nnz && v < (int64_t)0x7fffffff;
        if (i == 0 && v != 0) ok = false;
        if (i == n && v != nnz) ok = false;
        if (i < n && rp64[i + 1] < v) ok = false;
        if (!ok) atomicAdd(bad, 1);
        rp32[i] = (int)(v < 0 ? 0 : (v > nnz ? nnz : v));   // a bad entry never becomes an index
    }
}

__global__ void k_rp32_to_64(int n, const int *rp32, int64_t *rp64) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i <= n; i += gridDim.x * blockDim.x) rp64[i] = rp32[i];
}

static void load_csr(const amg_csr_t *A, DCsr &out, cudaStream_t s) {
    if (!A || A->n <= 0 || A->nnz < 0 || !A->row_ptr || (A->nnz > 0 && (!A->col || !A->val)))
        fail(AMG_ERR_INVALID_ARG, "CSR: null pointer or non-positive size");
    if (A->nnz >= (int64_t)0x7fffffff) fail(AMG_ERR_INVALID_ARG, "CSR: nnz >= 2^31 is not supported");
    const int n = A->n;
    const int nnz = (int)A->nnz;
    DBuf<int64_t> trp;
    DBuf<int> tci;
    DBuf<double> tv;
    const int64_t *rp64 = to_device(A->row_ptr, (size_t)n + 1, trp, s);
    const int *ci = to_device(A->col, (size_t)nnz, tci, s);
    const double *v = to_device(A->val, (size_t)nnz, tv, s);
    out.n = n;
    out.nnz = nnz;
    out.rp.alloc(n + 1);
    out.ci.alloc(nnz > 0 ? nnz : 1);
    out.v.alloc(nnz > 0 ? nnz : 1);
    DBuf<int> bad(1);
    CU(cudaMemsetAsync(bad.get(), 0, sizeof(int), s));
    k_rp64_to_32<<<grid_for((size_t)n + 1, 256), 256, 0, s>>>(n, A->nnz, rp64, out.rp.get(), bad.get());
    CU_LAUNCH("k_rp64_to_32"); count_launch();
    if (nnz) {
        CU(cudaMemcpyAsync(out.ci.get(), ci, sizeof(int) * nnz, cudaMemcpyDeviceToDevice, s));
        CU(cudaMemcpyAsync(out.v.get(), v, sizeof(double) * nnz, cudaMemcpyDeviceToDevice, s));
    }
    int hbad = 0;
    CU(cudaMemcpyAsync(&hbad, bad.get(), sizeof(int), cudaMemcpyDeviceToHost, s));
    CU(cudaStreamSynchronize(s));
    if (hbad) fail(AMG_ERR_INVALID_ARG, "CSR: row pointers are not a valid non-decreasing sequence from 0 to nnz");
    if (csr_validate(n, out.rp.get(), out.ci.get(), s))
        fail(AMG_ERR_INVALID_ARG, "CSR: columns out of range or not strictly ascending, or a missing diagonal");
}

__global__ void k_gather_double(const double *src, const int *idx, double *dst, int n) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) dst[i] = src[idx[i]];
}

// Transpose with values: T = M^T (rows ascending).
static void transpose_values(const DCsr &M, const double *vals, DCsr &T, cudaStream_t s) {
    DBuf<int> tsrc;
    csr_transpose(M.n, M.nnz, M.rp.get(), M.ci.get(), T.rp, T.ci, tsrc, s);
    T.n = M.n;
    T.nnz = M.nnz;
    T.v.alloc(M.nnz > 0 ? M.nnz : 1);
    if (M.nnz) {
        k_gather_double<<<grid_for(M.nnz, 256), 256, 0, s>>>(vals, tsrc.get(), T.v.get(), M.nnz);
        CU_LAUNCH("k_gather_double"); count_launch();
    }
    CU(cudaStreamSynchronize(s));
}

// Sweep schedules of the transposed factors: row j of (LU)^T holds U_ij
// (pos(i) < pos(j), forward, divided by u_jj) and L_ij (pos(i) > pos(j),
// backward, unit diagonal).
void build_transposed_sweeps(const DCsr &A, const int *pos, const double *lu, Sweep &fwdT, Sweep &bwdT,
                             cudaStream_t s);

// ------------------------------------------------------------------ setup
// frozen: per-pass maps to reuse instead of matching (amg_update_values),
// or nullptr.
static void coarsen(Level &L, const amg_options_t &o, DBuf<int> &adj_rp, DBuf<int> &adj_ci, int &adj_nnz,
                    DCsr &next, cudaStream_t s, std::vector<PassData> *frozen = nullptr) {
    const int n = L.A.n;
    L.agg.alloc(n);
    iota_int(L.agg.get(), n, s);
    const DCsr *cur = &L.A;
    DCsr last;
    L.passes.clear();
    L.passes.resize(o.passes);
    for (int p = 0; p < o.passes; ++p) {
        PassData &P = L.passes[p];
        DBuf<int> arp, aci;
        int annz = 0;
        sym_adjacency(*cur, arp, aci, annz, s);
        P.n_in = cur->n;
        int nc = 0;
        if (frozen) {
            PassData &F = (*frozen)[p];
            if (F.n_in != cur->n) fail(AMG_ERR_INVALID_ARG, "amg_update_values: hierarchy shape changed");
            P.agg = std::move(F.agg);
            nc = F.n_out;
        } else {
            DBuf<int> mate(cur->n);
            match_pass(*cur, arp.get(), aci.get(), annz, o.seed, o.match_weight, mate.get(), s);
            P.agg.alloc(cur->n);
            nc = aggregates_from_mate(cur->n, mate.get(), P.agg.get(), s);
        }
        P.n_out = nc;
        DBuf<int> mp, mi;
        members_of(cur->n, nc, P.agg.get(), mp, mi, s);
        DCsr C;
        galerkin(*cur, nc, P.agg.get(), mp.get(), mi.get(), C, s);
        DBuf<int> comp(n);
        gather_int(P.agg.get(), L.agg.get(), comp.get(), n, s);
        CU(cudaStreamSynchronize(s));
        L.agg = std::move(comp);
        if (p == 0) { adj_rp = std::move(arp); adj_ci = std::move(aci); adj_nnz = annz; }
        if (p + 1 < o.passes) {
            P.mat = std::move(C);
            cur = &P.mat;
        } else {
            next = std::move(C);
        }
    }
    L.n_next = next.n;
    members_of(n, next.n, L.agg.get(), L.mptr, L.midx, s);
}

static void build_smoother(Level &L, int order, const amg_options_t &o, const int *arp, const int *aci,
                           cudaStream_t s) {
    const int n = L.A.n;
    L.order = order;
    L.label.alloc(n);
    L.pos.alloc(n);
    int nlabels = 1;
    if (order == AMG_ORDER_NATURAL) {
        fill_int(L.label.get(), 0, n, s);
        L.ncol = 0;
    } else {
        DBuf<int> tr, tc;
        int tn = 0;
        if (!arp) {
            sym_adjacency(L.A, tr, tc, tn, s);
            arp = tr.get();
            aci = tc.get();
        }
        L.ncol = color_jp(n, arp, aci, o.coloring, o.seed, L.label.get(), s);
        nlabels = L.ncol;
    }
    elimination_positions(n, L.label.get(), nlabels, L.pos.get(), s);
    ilu0_factor(L.A, L.pos.get(), L.lu, L.fwd, L.bwd, s);
}

// Level 1 of the paper's two-grid form (Section 2, Algorithm 1 setup):
// A~_c = ILUT(A_c) on the host, the factors uploaded with their own pattern
// and scheduled for the same triangular sweeps as ILU(0) (natural order).
static void build_ilut_level(Level &L, const amg_options_t &o, cudaStream_t s) {
    const int n = L.A.n;
    std::vector<int> hrp(n + 1), hci(L.A.nnz);
    std::vector<double> hv(L.A.nnz);
    CU(cudaMemcpyAsync(hrp.data(), L.A.rp.get(), sizeof(int) * (n + 1), cudaMemcpyDeviceToHost, s));
    CU(cudaMemcpyAsync(hci.data(), L.A.ci.get(), sizeof(int) * L.A.nnz, cudaMemcpyDeviceToHost, s));
    CU(cudaMemcpyAsync(hv.data(), L.A.v.get(), sizeof(double) * L.A.nnz, cudaMemcpyDeviceToHost, s));
    CU(cudaStreamSynchronize(s));
    std::vector<int64_t> rp64(hrp.begin(), hrp.end());
    std::vector<int64_t> frp;
    std::vector<int32_t> fci;
    std::vector<double> fv;
    if (!ilut_factor_host(n, rp64.data(), hci.data(), hv.data(), o.ilut_tau, frp, fci, fv))
        fail(AMG_ERR_BREAKDOWN, "ILUT of the coarse level: zero or non-finite pivot");
    const int64_t nnz = frp[n];
    if (nnz >= (int64_t)0x7fffffff) fail(AMG_ERR_INVALID_ARG, "ILUT of the coarse level: factors with >= 2^31 entries");
    std::vector<int> frp32(frp.begin(), frp.end());
    DCsr &F = L.fpat;
    F.n = n;
    F.nnz = (int)nnz;
    F.rp.alloc(n + 1);
    F.ci.alloc(nnz > 0 ? nnz : 1);
    F.v.alloc(nnz > 0 ? nnz : 1);
    CU(cudaMemcpyAsync(F.rp.get(), frp32.data(), sizeof(int) * (n + 1), cudaMemcpyHostToDevice, s));
    CU(cudaMemcpyAsync(F.ci.get(), fci.data(), sizeof(int) * nnz, cudaMemcpyHostToDevice, s));
    CU(cudaMemcpyAsync(F.v.get(), fv.data(), sizeof(double) * nnz, cudaMemcpyHostToDevice, s));
    L.lu.alloc(nnz > 0 ? nnz : 1);
    CU(cudaMemcpyAsync(L.lu.get(), fv.data(), sizeof(double) * nnz, cudaMemcpyHostToDevice, s));
    L.order = AMG_ORDER_NATURAL;
    L.ncol = 0;
    L.label.alloc(n);
    L.pos.alloc(n);
    fill_int(L.label.get(), 0, n, s);
    elimination_positions(n, L.label.get(), 1, L.pos.get(), s);
    factor_sweeps(F, L.pos.get(), L.lu.get(), L.fwd, L.bwd, s);
    CU(cudaStreamSynchronize(s));   // the host vectors above are the copies' sources
    L.ilut_level = true;
}

// Storage precision of level l's factors for a V-cycle precision.
static int level_prec(int vcycle_prec, size_t l) {
    if (vcycle_prec == AMG_BF16_ALL) return AMG_BF16;
    if (vcycle_prec == AMG_BF16 && l > 0) return AMG_FP32;
    return vcycle_prec;
}

static void cast_sweep(Sweep &S, int prec, cudaStream_t s) {
    const size_t nnzf = S.v64.n;
    if (prec == AMG_FP32 || prec == AMG_BF16) {
        S.v32.alloc(nnzf);
        cast_f64_f32(S.v64.get(), S.v32.get(), nnzf, s);
        if (S.d64.n) {
            S.d32.alloc(S.d64.n);
            cast_f64_f32(S.d64.get(), S.d32.get(), S.d64.n, s);
        }
    }
    if (prec == AMG_BF16) {
        S.v16.alloc(nnzf);
        cast_f64_bf16(S.v64.get(), S.v16.get(), nnzf, s);
    }
}

template <typename T, typename V>
static void build_deep(amg_handle *h);

// SpMV autotuner: times every (threads per block, unroll) pair not fixed by
// the options on this matrix (one warm-up and three timed launches each, x in
// the V-cycle's output type) and keeps the fastest.  Results do not depend on
// the choice.
static void tune_sell(Sell &SL, const amg_options_t &o, cudaStream_t s) {
    static const int blocks[] = {64, 128, 256, 512};
    static const int unrolls[] = {2, 4, 8};
    SL.block = o.spmv_block ? o.spmv_block : 256;
    SL.unroll = o.spmv_unroll ? o.spmv_unroll : 4;
    if (o.spmv_block && o.spmv_unroll) return;
    const bool f64 = o.vcycle_prec == AMG_FP64;
    const size_t n = (size_t)SL.n;
    DBuf<char> xb(n * (f64 ? sizeof(double) : sizeof(float)));
    DBuf<double> y(n);
    CU(cudaMemsetAsync(xb.get(), 0, xb.n, s));
    cudaEvent_t e0, e1;
    CU(cudaEventCreate(&e0));
    CU(cudaEventCreate(&e1));
    float best = 1e30f;
    int bb = SL.block, bu = SL.unroll;
    try {
        for (int blk : blocks) {
            if (o.spmv_block && blk != o.spmv_block) continue;
            for (int u : unrolls) {
                if (o.spmv_unroll && u != o.spmv_unroll) continue;
                auto run = [&] {
                    if (f64)
                        sell_spmv<double>(SL.n, SL.nslices, SL.ptr.get(), SL.ci.get(), SL.v.get(),
                                          reinterpret_cast<const double *>(xb.get()), nullptr, y.get(), 0, s, blk, u);
                    else
                        sell_spmv<float>(SL.n, SL.nslices, SL.ptr.get(), SL.ci.get(), SL.v.get(),
                                         reinterpret_cast<const float *>(xb.get()), nullptr, y.get(), 0, s, blk, u);
                };
                run();
                CU(cudaEventRecord(e0, s));
                for (int r = 0; r < 3; ++r) run();
                CU(cudaEventRecord(e1, s));
                CU(cudaEventSynchronize(e1));
                float ms = 0.f;
                CU(cudaEventElapsedTime(&ms, e0, e1));
                if (ms < best) { best = ms; bb = blk; bu = u; }
            }
        }
    } catch (...) {
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        throw;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    SL.block = bb;
    SL.unroll = bu;
}

// frozen (amg_update_values): the previous hierarchy's per-level, per-pass
// maps; levels keep the same shape, only the numbers are recomputed.
// Levels with at least this many rows keep a SELL-32 copy for the V-cycle's
// forward residual (smaller ones are bound by launch latency).
constexpr int RSELL_MIN = 32768;

static void build_tiles(amg_handle *h, cudaStream_t s);

static void setup_impl(amg_handle *h, const amg_csr_t *Ain,
                       std::vector<std::vector<PassData>> *frozen = nullptr) {
    const amg_options_t &o = h->opt;
    cudaStream_t s = h->stream;
    auto L0 = std::make_unique<Level>();
    load_csr(Ain, L0->A, s);
    h->n = L0->A.n;
    h->lev.push_back(std::move(L0));
    for (int l = 0;; ++l) {
        Level &L = *h->lev[l];
        const bool two_grid = o.coarse_solver == AMG_COARSE_ILUT;
        bool last = two_grid ? l >= 1 : ((l > 0 && L.A.n <= o.dense_max) || (l + 1 >= o.max_levels));
        if (frozen) last = l >= (int)frozen->size() || (*frozen)[l].empty();
        DBuf<int> arp, aci;
        int annz = 0;
        if (!last) {
            auto N = std::make_unique<Level>();
            coarsen(L, o, arp, aci, annz, N->A, s, frozen ? &(*frozen)[l] : nullptr);
            if (!frozen && l > 0 && (double)N->A.n > 0.9 * (double)L.A.n) {
                last = true;
                L.passes.clear();
                L.agg.release(); L.mptr.release(); L.midx.release();
                L.n_next = -1;
            } else {
                h->lev.push_back(std::move(N));
            }
        }
        if (two_grid && l == 1) {
            build_ilut_level(L, o, s);
        } else if (last && L.A.n <= o.dense_max) {
            L.dense = true;
            dense_inverse(L.A, L.inv, s);
        } else {
            const int order = l == 0 ? o.order_fine : o.order_coarse;
            build_smoother(L, order, o, arp.n ? arp.get() : nullptr, aci.n ? aci.get() : nullptr, s);
        }
        if (last) break;
    }
    // precision copies (BF16: the finest level's ILU(0) factors only; BF16_ALL:
    // the factors of every smoothed level)
    for (size_t l = 0; l < h->lev.size(); ++l) {
        Level &L = *h->lev[l];
        const int prec = level_prec(o.vcycle_prec, l);
        if (prec != AMG_FP64) {
            L.v32.alloc(L.A.nnz);
            cast_f64_f32(L.A.v.get(), L.v32.get(), L.A.nnz, s);
        }
        if (!L.dense) {
            cast_sweep(L.fwd, prec, s);
            cast_sweep(L.bwd, prec, s);
        } else if (prec != AMG_FP64) {
            const size_t nn = (size_t)L.A.n * L.A.n;
            L.inv32.alloc(nn);
            cast_f64_f32(L.inv.get(), L.inv32.get(), nn, s);
        }
    }
    // adjoint structures
    if (o.build_adjoint) {
        for (size_t l = 0; l < h->lev.size(); ++l) {
            Level &L = *h->lev[l];
            const int prec = level_prec(o.vcycle_prec, l);
            transpose_values(L.A, L.A.v.get(), L.AT, s);
            if (prec != AMG_FP64) {
                L.vt32.alloc(L.AT.nnz);
                cast_f64_f32(L.AT.v.get(), L.vt32.get(), L.AT.nnz, s);
            }
            if (!L.dense) {
                build_transposed_sweeps(L.ilut_level ? L.fpat : L.A, L.pos.get(), L.lu.get(), L.fwdT, L.bwdT, s);
                cast_sweep(L.fwdT, prec, s);
                cast_sweep(L.bwdT, prec, s);
            }
        }
        h->adjoint_ready = true;
    }
    build_tiles(h, s);
    // SELL-32 copies of the larger levels for the V-cycle's forward residuals
    for (size_t l = 0; l < h->lev.size(); ++l) {
        Level &L = *h->lev[l];
        if (L.dense || L.ilut_level || L.A.n < RSELL_MIN) continue;
        build_sell(L.A, L.A.v.get(), L.rsell, s);
        if (o.vcycle_prec != AMG_FP64) {
            L.rsv32.alloc((size_t)L.rsell.padded);
            cast_f64_f32(L.rsell.v.get(), L.rsv32.get(), (size_t)L.rsell.padded, s);
            CU(cudaStreamSynchronize(s));
            L.rsell.v.release();
        }
    }
    // SELL-32 copies of A (and A^T) for the outer FP64 products
    build_sell(h->lev[0]->A, h->lev[0]->A.v.get(), h->lev[0]->sell, s);
    if (o.build_adjoint) build_sell(h->lev[0]->AT, h->lev[0]->AT.v.get(), h->lev[0]->sellT, s);
    tune_sell(h->lev[0]->sell, o, s);
    if (o.build_adjoint) {
        h->lev[0]->sellT.block = h->lev[0]->sell.block;
        h->lev[0]->sellT.unroll = h->lev[0]->sell.unroll;
    }
    // workspaces
    const size_t tsz = o.vcycle_prec == AMG_FP64 ? sizeof(double) : sizeof(float);
    for (auto &Lp : h->lev) {
        Level &L = *Lp;
        const size_t b = tsz * (size_t)L.A.n;
        L.wt.alloc(b); L.wy.alloc(b); L.wr.alloc(b); L.wres.alloc(b); L.wh.alloc(b); L.wg.alloc(b); L.wf.alloc(b);
        if (o.persistent >= 2) {   // dataflow sweeps expect wy to hold the sentinel on entry
            if (tsz == sizeof(double)) fill_sentinel<double>(reinterpret_cast<double *>(L.wy.get()), L.A.n, s);
            else fill_sentinel<float>(reinterpret_cast<float *>(L.wy.get()), L.A.n, s);
            L.wy_sent = (int)tsz;
        }
    }
    const size_t n = h->n, m = o.restart;
    h->V.alloc((m + 1) * n);
    if (o.vcycle_prec == AMG_FP64) { h->Zd.alloc(m * n); h->zin64.alloc(n); h->zout64.alloc(n); }
    else { h->Zf.alloc(m * n); h->zin32.alloc(n); h->zout32.alloc(n); }
    CU(cudaMallocHost(&h->hflags, 2 * sizeof(int)));
    switch (o.vcycle_prec) {
    case AMG_FP64: build_deep<double, double>(h); break;
    case AMG_FP32: build_deep<float, float>(h); break;
    default: build_deep<float, float>(h); break;   // BF16 mode: coarse levels are FP32
    }
    h->w.alloc(n); h->r.alloc(n); h->xb.alloc(n); h->bb.alloc(n);
    h->hist.alloc((size_t)o.maxit + 2);
    h->partials.alloc((size_t)reduce_grid() * KMAX1);
    h->st.alloc(1);
    h->ticket.alloc(1);
    CU(cudaMemsetAsync(h->ticket.get(), 0, sizeof(unsigned int), s));
    h->bar.alloc(2);
    CU(cudaMemsetAsync(h->bar.get(), 0, 2 * sizeof(unsigned int), s));
    h->err.alloc(1);
    CU(cudaMemsetAsync(h->err.get(), 0, sizeof(int), s));
    CU(cudaMallocHost(&h->hst, sizeof(FgState)));
    CU(cudaStreamSynchronize(s));
}

// ------------------------------------------------------------------ kernel timing
static void tmark_begin(amg_handle *h, int kclass) {
    if (h->tclass != kclass) return;
    if (h->tused == h->tev.size()) {
        cudaEvent_t a, b;
        CU(cudaEventCreate(&a));
        CU(cudaEventCreate(&b));
        h->tev.emplace_back(a, b);
    }
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    CU(cudaStreamIsCapturing(h->stream, &cs));
    // inside a capture the record must become a node of the graph
    CU(cudaEventRecordWithFlags(h->tev[h->tused].first, h->stream,
                                cs == cudaStreamCaptureStatusActive ? cudaEventRecordExternal : 0));
}
static void tmark_end(amg_handle *h, int kclass, double bytes) {
    if (h->tclass != kclass) return;
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    CU(cudaStreamIsCapturing(h->stream, &cs));
    CU(cudaEventRecordWithFlags(h->tev[h->tused].second, h->stream,
                                cs == cudaStreamCaptureStatusActive ? cudaEventRecordExternal : 0));
    ++h->tused;
    h->t_bytes += bytes;
    h->t_bytes_per_launch = bytes;
}
// after a synchronisation: fold the recorded pairs into the totals
static void tcollect(amg_handle *h, size_t count) {
    for (size_t i = 0; i < count; ++i) {
        float ms = 0.f;
        CU(cudaEventElapsedTime(&ms, h->tev[i].first, h->tev[i].second));
        h->t_ms += ms;
        ++h->t_launches;
    }
}
static void tcollect(amg_handle *h) {
    tcollect(h, h->tused);
    h->tused = 0;
}

// ------------------------------------------------------------------ preconditioner
// Accurate (Dot2) inner products: on by default with the FP64 V-cycle.
static bool use_dot2(const amg_handle *h) {
    return h->opt.dot2 < 0 ? h->opt.vcycle_prec == AMG_FP64 : h->opt.dot2 != 0;
}

template <typename T, typename V>
struct VCycle {
    amg_handle *h;
    cudaStream_t s;

    Level &L(int l) { return *h->lev[l]; }
    static T *ws(DBuf<char> &b) { return reinterpret_cast<T *>(b.get()); }

    const V *vals(Level &Lv, bool tr);
    LevelMats<V> mats(int l, bool tr) {
        Level &Lv = L(l);
        const DCsr &M = tr ? Lv.AT : Lv.A;
        return LevelMats<V>{M.n, M.nnz, M.rp.get(), M.ci.get(), vals(Lv, tr)};
    }
    SweepView<T, V> view(Sweep &S);

    int nlev() const { return (int)h->lev.size(); }

    // the dense last level's rows as Dot2 inner products in the FP64 V-cycle
    // when the Arnoldi inner products are Dot2 too (the dot2 option)
    bool dense_dot2() const { return std::is_same<T, double>::value && use_dot2(h); }

    // g = A_L^{-1} h (transpose: A_L^{-T} h) on the dense last level: the FP64
    // inverse in the FP64 V-cycle, its FP32 copy in the FP32 / BF16 ones
    void dense_apply(Level &Lv, const T *hrhs, T *g, int transpose) {
        if constexpr (std::is_same<T, float>::value) {
            if (Lv.inv32.n) { dense_solve_f32(Lv.A.n, Lv.inv32.get(), hrhs, g, transpose, s); return; }
        }
        dense_solve<T>(Lv.A.n, Lv.inv.get(), hrhs, g, transpose, 0, dense_dot2(), s);
    }

    // t = S^{-1} in (transpose: S^{-T} in); y is scratch for the first solve
    void smooth(Level &Lv, const T *in, T *y, T *t, bool transpose) {
        Sweep &F = transpose ? Lv.fwdT : Lv.fwd;
        Sweep &B = transpose ? Lv.bwdT : Lv.bwd;
        const int fd = transpose ? 1 : 0, bd = transpose ? 0 : 1;
        // persistent 5: as 3, the finest level in grid tiles when its matrix
        // is a natural-order grid stencil (tiles.cu)
        const TilePlan *P = Lv.tiles.get();
        const bool tiled = h->opt.persistent == 5 && P && P->tsz == sizeof(T) && P->vsz == sizeof(V) &&
                           (transpose ? P->fwdT.c.n : P->fwd.c.n);
        // algorithmic bytes: factor values (+ columns and schedule
        // rows/pointers, which the tiled solve does not read), the diagonal,
        // in read once, y written and read, out written
        const double n = Lv.A.n;
        const double bytes = (sizeof(V) + (tiled ? 0.0 : 4.0)) * (double)(F.v64.n + B.v64.n) +
                             (tiled ? 0.0 : 12.0 * 2.0 * n) +
                             sizeof(T) * (1.0 + (B.d64.n || F.d64.n ? 1.0 : 0.0) + 3.0) * n;
        tmark_begin(h, 2);
        // persistent 2: dataflow solve (no level barriers) on every level
        // (3: on the finest level only, the others as with 1; 4: on every
        // level too large for the shared-memory cluster kernel);
        // persistent 1: one cooperative launch with level barriers where there
        // are many schedule levels (natural order), colour classes as
        // separate launches; persistent 0: one launch per schedule level
        const bool finest = &Lv == h->lev[0].get();
        const bool dataflow = h->opt.persistent == 2 ||
                              ((h->opt.persistent == 3 || h->opt.persistent == 5) && finest) ||
                              (h->opt.persistent == 4 && !sweep_fits_dsm(Lv.A.n, F.nlev, B.nlev, sizeof(T)));
        int kind;
        if (tiled) {
            sweep_pair_tiles<T, V>(*P, transpose ? P->fwdT : P->fwd, transpose ? P->bwdT : P->bwd, in, y, t,
                                   h->bar.get(), h->err.get(), s);
            kind = SWEEP_KIND_TILES;
        } else if (dataflow) {
            if (Lv.wy_sent != (int)sizeof(T)) {
                fill_sentinel<T>(y, (size_t)Lv.A.n, s);
                Lv.wy_sent = (int)sizeof(T);
            }
            sweep_pair_df<T, V>(view(F), fd, view(B), bd, in, y, t, h->bar.get(), h->err.get(), s);
            kind = SWEEP_KIND_DATAFLOW;
        } else if (h->opt.persistent && F.nlev + B.nlev > PERSISTENT_MIN_LEVELS) {
            kind = sweep_pair_coop<T, V>(view(F), fd, view(B), bd, in, y, t, h->bar.get(), h->err.get(), s);
        } else {
            sweep<T, V>(view(F), in, y, fd, s);
            sweep<T, V>(view(B), y, t, bd, s);
            kind = SWEEP_KIND_LEVELS;
        }
        Lv.sweep_kind[transpose ? 1 : 0] = kind;
        tmark_end(h, 2, bytes);
    }
    bool has_child(int l) { return l + 1 < nlev() && L(l).n_next > 0; }

    // r = b - A_l x (tr: A_l^T).  In BF16 mode only the ILU(0) factors are
    // BF16; the residual keeps FP32 values (8-bit mantissas cannot resolve
    // the small residual of smooth errors of a near-singular diffusion
    // operator, which the coarse correction needs).
    void residual(int l, bool tr, const T *x, const T *b, T *r) {
        Level &Lr = L(l);
        if (!tr && Lr.rsell.n > 0) {              // SELL-32 copy of a larger level
            if constexpr (std::is_same<T, double>::value)
                level_residual_sell<double, double>(Lr.rsell.n, Lr.rsell.ptr.get(), Lr.rsell.ci.get(),
                                                    Lr.rsell.v.get(), x, b, r, s);
            else
                level_residual_sell<float, float>(Lr.rsell.n, Lr.rsell.ptr.get(), Lr.rsell.ci.get(),
                                                  Lr.rsv32.get(), x, b, r, s);
            return;
        }
        if constexpr (std::is_same<V, __nv_bfloat16>::value) {
            Level &Lv = L(l);
            const DCsr &M = tr ? Lv.AT : Lv.A;
            level_residual<float, float>(
                LevelMats<float>{M.n, M.nnz, M.rp.get(), M.ci.get(), tr ? Lv.vt32.get() : Lv.v32.get()}, x, b, r, s);
        } else {
            level_residual<T, V>(mats(l, tr), x, b, r, s);
        }
    }

    // q (mode 0: =, mode 1: +=) B_l^{-1} z
    void precond(int l, const T *z, T *q, int mode) {
        Level &Lv = L(l);
        const int n = Lv.A.n;
        T *y = ws(Lv.wy), *t = ws(Lv.wt), *r = ws(Lv.wr);
        smooth(Lv, z, y, t, false);
        residual(l, false, t, z, r);
        Level &C = L(l + 1);
        T *hc = ws(C.wh), *gc = ws(C.wg);
        restrict_to<T>(C.A.n, Lv.mptr.get(), Lv.midx.get(), r, hc, s);
        level_solve(l + 1, hc, gc);
        prolong<T, T>(n, Lv.agg.get(), t, gc, q, mode, s);
    }

    // g = C_l(h): the inexact solve of level l >= 1
    void level_solve(int l, const T *hrhs, T *g) {
        if constexpr (std::is_same<V, __nv_bfloat16>::value) {
            // BF16 factors on the finest level only (AMG_BF16) or on levels
            // run by the single-block deep V-cycle: the coarse levels run in
            // FP32.  AMG_BF16_ALL keeps BF16 factors on every level; the
            // residuals always use FP32 matrix values (rounding Galerkin sums
            // with near-zero row sums to 8 bits made the coarse Richardson
            // steps diverge).
            if (h->opt.vcycle_prec != AMG_BF16_ALL || l >= h->deep_first) {
                VCycle<float, float>{h, s}.level_solve(l, hrhs, g);
                return;
            }
        }
        Level &Lv = L(l);
        if (l >= h->deep_first) {
            const DeepLevel<T, V> *d = reinterpret_cast<const DeepLevel<T, V> *>(h->deep_desc.get()) +
                                       (l - h->deep_first);
            deep_vcycle<T, V>(d, nlev() - l, s);
            return;
        }
        if (Lv.dense) { dense_apply(Lv, hrhs, g, 0); return; }
        if (Lv.ilut_level) { smooth(Lv, hrhs, ws(Lv.wy), g, false); return; }   // g = (L~ U~)^{-1} h
        const int k = l == 1 ? h->opt.coarse_inner : h->opt.deep_inner;
        T *res = ws(Lv.wres);
        for (int it = 0; it < k; ++it) {
            const T *in = hrhs;
            if (it > 0) {
                residual(l, false, g, hrhs, res);
                in = res;
            }
            if (has_child(l)) {
                precond(l, in, g, it == 0 ? 0 : 1);
            } else {
                T *y = ws(Lv.wy), *t = ws(Lv.wt);
                smooth(Lv, in, y, t, false);
                vec_acc<T>(Lv.A.n, t, g, it == 0 ? 0 : 1, s);
            }
        }
    }

    // q (mode) = B_l^{-T} z = f + S^{-T}(z - A^T f), f = P C^T P^T z
    void precondT(int l, const T *z, T *q, int mode) {
        Level &Lv = L(l);
        const int n = Lv.A.n;
        Level &C = L(l + 1);
        T *hc = ws(C.wh), *gc = ws(C.wg);
        T *f = ws(Lv.wf), *r = ws(Lv.wr), *y = ws(Lv.wy), *t = ws(Lv.wt);
        restrict_to<T>(C.A.n, Lv.mptr.get(), Lv.midx.get(), z, hc, s);
        level_solveT(l + 1, hc, gc);
        prolong<T, T>(n, Lv.agg.get(), nullptr, gc, f, 2, s);
        residual(l, true, f, z, r);
        smooth(Lv, r, y, t, true);
        // q (mode)= f + t
        prolong<T, T>(n, nullptr, f, t, q, mode == 0 ? 3 : 4, s);
    }

    void level_solveT(int l, const T *hrhs, T *g) {
        if constexpr (std::is_same<V, __nv_bfloat16>::value) {
            if (h->opt.vcycle_prec != AMG_BF16_ALL || l >= h->deep_first) {
                VCycle<float, float>{h, s}.level_solveT(l, hrhs, g);
                return;
            }
        }
        Level &Lv = L(l);
        if (Lv.dense) { dense_apply(Lv, hrhs, g, 1); return; }
        if (Lv.ilut_level) { smooth(Lv, hrhs, ws(Lv.wy), g, true); return; }    // g = (L~ U~)^{-T} h
        const int k = l == 1 ? h->opt.coarse_inner : h->opt.deep_inner;
        T *res = ws(Lv.wres);
        for (int it = 0; it < k; ++it) {
            const T *in = hrhs;
            if (it > 0) {
                residual(l, true, g, hrhs, res);
                in = res;
            }
            if (has_child(l)) {
                precondT(l, in, g, it == 0 ? 0 : 1);
            } else {
                T *y = ws(Lv.wy), *t = ws(Lv.wt);
                smooth(Lv, in, y, t, true);
                vec_acc<T>(Lv.A.n, t, g, it == 0 ? 0 : 1, s);
            }
        }
    }
};

template <> const double *VCycle<double, double>::vals(Level &Lv, bool tr) { return tr ? Lv.AT.v.get() : Lv.A.v.get(); }
template <> const float *VCycle<float, float>::vals(Level &Lv, bool tr) { return tr ? Lv.vt32.get() : Lv.v32.get(); }
template <> const __nv_bfloat16 *VCycle<float, __nv_bfloat16>::vals(Level &Lv, bool tr) {
    return tr ? Lv.vt16.get() : Lv.v16.get();
}
template <> SweepView<double, double> VCycle<double, double>::view(Sweep &S) {
    return SweepView<double, double>{S.nlev, S.lev_ptr.data(), S.dlev.get(), S.rows.get(), S.rp.get(), S.ci.get(),
                                     S.v64.get(), S.d64.n ? S.d64.get() : nullptr};
}
template <> SweepView<float, float> VCycle<float, float>::view(Sweep &S) {
    return SweepView<float, float>{S.nlev, S.lev_ptr.data(), S.dlev.get(), S.rows.get(), S.rp.get(), S.ci.get(),
                                   S.v32.get(), S.d32.n ? S.d32.get() : nullptr};
}
template <> SweepView<float, __nv_bfloat16> VCycle<float, __nv_bfloat16>::view(Sweep &S) {
    return SweepView<float, __nv_bfloat16>{S.nlev, S.lev_ptr.data(), S.dlev.get(), S.rows.get(), S.rp.get(),
                                           S.ci.get(), S.v16.get(), S.d32.n ? S.d32.get() : nullptr};
}

// The finest level's smoother in tile layout (persistent 5): built when the
// level is in natural order and its matrix a 2D / 3D grid stencil; without
// a plan the level keeps the dataflow solve.
template <typename T, typename V>
static void build_tiles_t(amg_handle *h, Level &L, cudaStream_t s) {
    std::unique_ptr<TilePlan> P(new TilePlan());
    if (!tile_plan_build(L.A, *P, sizeof(T), sizeof(V), s)) return;
    tile_prepare<T, V>(*P);
    VCycle<T, V> vc{h, s};
    if (!tile_factor_build<T, V>(*P, vc.view(L.fwd), false, P->fwd, s)) return;
    if (!tile_factor_build<T, V>(*P, vc.view(L.bwd), true, P->bwd, s)) return;
    if (h->opt.build_adjoint) {
        if (!tile_factor_build<T, V>(*P, vc.view(L.fwdT), false, P->fwdT, s)) return;
        if (!tile_factor_build<T, V>(*P, vc.view(L.bwdT), true, P->bwdT, s)) return;
    }
    L.tiles = std::move(P);
}
static void build_tiles(amg_handle *h, cudaStream_t s) {
    Level &L = *h->lev[0];
    L.tiles.reset();
    if (h->opt.persistent != 5 || L.dense || L.ilut_level || L.order != AMG_ORDER_NATURAL) return;
    switch (level_prec(h->opt.vcycle_prec, 0)) {
    case AMG_FP64: build_tiles_t<double, double>(h, L, s); break;
    case AMG_FP32: build_tiles_t<float, float>(h, L, s); break;
    default: build_tiles_t<float, __nv_bfloat16>(h, L, s); break;
    }
}

// Device descriptors of the levels run by the single-block V-cycle.
template <typename T, typename V>
static void build_deep(amg_handle *h) {
    const int nl = (int)h->lev.size();
    const auto &o = h->opt;
    h->deep_first = 1 << 30;
    if (!o.deep_block_max || o.deep_inner != 1) return;
    int first = nl;
    for (int l = nl - 1; l >= 2; --l) {
        if (h->lev[l]->A.n > o.deep_block_max) break;
        first = l;
    }
    if (first >= nl) return;
    VCycle<T, V> vc{h, h->stream};
    std::vector<DeepLevel<T, V>> d(nl - first);
    for (int l = first; l < nl; ++l) {
        Level &Lv = *h->lev[l];
        DeepLevel<T, V> &D = d[l - first];
        memset(&D, 0, sizeof(D));
        D.n = Lv.A.n;
        D.dense = Lv.dense ? 1 : 0;
        D.has_child = vc.has_child(l) ? 1 : 0;
        D.rp = Lv.A.rp.get();
        D.ci = Lv.A.ci.get();
        D.v = vc.vals(Lv, false);
        if (!Lv.dense) { D.fwd = vc.view(Lv.fwd); D.bwd = vc.view(Lv.bwd); }
        D.inv = Lv.inv.get();
        D.agg = Lv.agg.get();
        D.mptr = Lv.mptr.get();
        D.midx = Lv.midx.get();
        D.h = VCycle<T, V>::ws(Lv.wh);
        D.g = VCycle<T, V>::ws(Lv.wg);
        D.t = VCycle<T, V>::ws(Lv.wt);
        D.y = VCycle<T, V>::ws(Lv.wy);
        D.r = VCycle<T, V>::ws(Lv.wr);
    }
    h->deep_desc.alloc(sizeof(DeepLevel<T, V>) * d.size());
    CU(cudaMemcpyAsync(h->deep_desc.get(), d.data(), sizeof(DeepLevel<T, V>) * d.size(), cudaMemcpyHostToDevice,
                       h->stream));
    CU(cudaStreamSynchronize(h->stream));
    h->deep_first = first;
}

// q = B~^{-1} zin (or B~^{-T} zin) at level 0 in the V-cycle type.
template <typename T, typename V>
static void precond0(amg_handle *h, const T *zin, T *zout, bool transpose) {
    if (h->lev.size() < 2) fail(AMG_ERR_NOT_SUPPORTED, "hierarchy has a single level");
    VCycle<T, V> vc{h, h->stream};
    if (transpose) vc.precondT(0, zin, zout, 0);
    else vc.precond(0, zin, zout, 0);
}

static void apply_precond_vtype(amg_handle *h, bool transpose) {
    switch (h->opt.vcycle_prec) {
    case AMG_FP64: precond0<double, double>(h, h->zin64.get(), h->zout64.get(), transpose); break;
    case AMG_FP32: precond0<float, float>(h, h->zin32.get(), h->zout32.get(), transpose); break;
    default: precond0<float, __nv_bfloat16>(h, h->zin32.get(), h->zout32.get(), transpose); break;
    }
}

// ------------------------------------------------------------------ FGMRES
// One inner FGMRES iteration (column j = st->j, read on the device):
// z_j = B~^{-1} v_j, w = A z_j, modified Gram-Schmidt (or CGS2) against
// v_0..v_j, ||w||, Givens, v_{j+1} = w / ||w||, and the stop flag copied to
// pinned host memory.
static void enqueue_iteration(amg_handle *h, bool transpose, bool host_flag = true) {
    cudaStream_t s = h->stream;
    const size_t n = h->n;
    FgState *dst = h->st.get();
    Level &L0 = *h->lev[0];
    const DCsr &M = transpose ? L0.AT : L0.A;
    const bool f64 = h->opt.vcycle_prec == AMG_FP64;
    if (f64) load_vj<double>(n, dst, h->V.get(), h->zin64.get(), s);
    else load_vj<float>(n, dst, h->V.get(), h->zin32.get(), s);
    apply_precond_vtype(h, transpose);
    // algorithmic bytes of w = A z: values + columns, row pointers, z once, w once
    const double bytes = 12.0 * M.nnz + 4.0 * (M.n + 1) + (f64 ? 8.0 : 4.0) * M.n + 8.0 * M.n;
    const Sell &SL = transpose ? L0.sellT : L0.sell;
    tmark_begin(h, 1);
    if (f64) sell_spmv<double>(SL.n, SL.nslices, SL.ptr.get(), SL.ci.get(), SL.v.get(), h->zout64.get(), nullptr,
                               h->w.get(), 0, s, SL.block, SL.unroll);
    else sell_spmv<float>(SL.n, SL.nslices, SL.ptr.get(), SL.ci.get(), SL.v.get(), h->zout32.get(), nullptr,
                          h->w.get(), 0, s, SL.block, SL.unroll);
    tmark_end(h, 1, bytes);
    (void)M;
    if (f64) store_zj<double>(n, dst, h->zout64.get(), h->Zd.get(), s);
    else store_zj<float>(n, dst, h->zout32.get(), h->Zf.get(), s);
    // K = j+1 basis vectors are known only on the device, so the bytes use
    // the cycle's mean K = (m+1)/2
    const double K = 0.5 * (h->opt.restart + 1);
    if (h->opt.orthog == AMG_ORTHO_MGS) {
        // step k reads w, v_k, v_{k+1} and writes w; the first dot reads w, v_0
        tmark_begin(h, 3);
        mgs(n, dst, h->w.get(), h->V.get(), n, h->partials.get(), h->bar.get(), h->err.get(), use_dot2(h), s);
        tmark_end(h, 3, 8.0 * (double)n * (4.0 * K + 2.0));
    } else {
        mdot(n, dst, h->w.get(), h->V.get(), n, h->partials.get(), h->ticket.get(), dst->h1, s);
        // a CGS2 pass reads the K basis vectors and w and writes w
        tmark_begin(h, 3);
        cgs_update(n, dst, dst->h1, h->w.get(), h->V.get(), n, 1, h->partials.get(), h->ticket.get(), dst->h2, s);
        tmark_end(h, 3, 8.0 * (double)n * (K + 2.0));
        cgs_update(n, dst, dst->h2, h->w.get(), h->V.get(), n, 0, h->partials.get(), h->ticket.get(), dst->nrm2, s);
    }
    givens(dst, s);
    scale_next(n, h->w.get(), h->V.get(), dst, s);
    if (host_flag) CU(cudaMemcpyAsync(h->hflags, &dst->stop, 2 * sizeof(int), cudaMemcpyDeviceToHost, s));
}

// Queues one inner iteration, replaying a captured CUDA graph when enabled
// (captured on first use, once per handle and direction).  No synchronisation.
static void launch_iteration(amg_handle *h, bool transpose) {
    const int d = transpose ? 1 : 0;
    if (!h->opt.use_graphs) {
        enqueue_iteration(h, transpose);
        return;
    }
    if (!h->gexec[d]) {
        const size_t before = h->tused;
        const int64_t l0 = launch_count();
        const double b0 = h->t_bytes;
        cudaGraph_t g = nullptr;
        CU(cudaStreamBeginCapture(h->stream, cudaStreamCaptureModeThreadLocal));
        try {
            enqueue_iteration(h, transpose);
        } catch (...) {
            cudaStreamEndCapture(h->stream, &g);
            if (g) cudaGraphDestroy(g);
            cudaGetLastError();
            h->tused = before;
            throw;
        }
        CU(cudaStreamEndCapture(h->stream, &g));
        cudaError_t e = cudaGraphInstantiate(&h->gexec[d], g, 0);
        cudaGraphDestroy(g);
        CU(e);
        h->gpairs[d] = h->tused - before;
        h->tused = before;
        h->gnodes[d] = launch_count() - l0;
        count_launch(-h->gnodes[d]);          // counted again at each replay
        h->gbytes[d] = h->t_bytes - b0;
        h->t_bytes = b0;                      // added again at each replay
    }
    CU(cudaGraphLaunch(h->gexec[d], h->stream));
    count_launch(h->gnodes[d]);
    h->t_bytes += h->gbytes[d];
}

// Waits for the queued iteration and folds its kernel timings.
static void collect_iteration(amg_handle *h, bool transpose) {
    CU(cudaStreamSynchronize(h->stream));
    if (h->opt.use_graphs) tcollect(h, h->gpairs[transpose ? 1 : 0]);
    else tcollect(h);
}

static void outer_residual(amg_handle *h, const double *b, const double *x, double *r, bool transpose) {
    Level &L0 = *h->lev[0];
    const Sell &SL = transpose ? L0.sellT : L0.sell;
    sell_spmv<double>(SL.n, SL.nslices, SL.ptr.get(), SL.ci.get(), SL.v.get(), x, b, r, 1, h->stream, SL.block,
                      SL.unroll);
}

static double read_norm(amg_handle *h, const double *v) {
    cudaStream_t s = h->stream;
    norm2(h->n, v, h->partials.get(), h->ticket.get(), h->st.get()->nrm2, use_dot2(h), s);
    double r = 0.0;
    CU(cudaMemcpyAsync(&r, h->st.get()->nrm2, sizeof(double), cudaMemcpyDeviceToHost, s));
    CU(cudaStreamSynchronize(s));
    return std::sqrt(r);
}

// One FGMRES(m) solve as a host-side state machine, so that the batched
// driver can advance many systems (each on its own stream) together:
// begin() computes ||b|| and the initial residual and starts a cycle;
// launch()/collect() run one inner iteration; at the end of a cycle the
// solution is updated, the true residual decides convergence, and a new
// cycle starts.  Kernels and their order are those of a single solve.
struct Run {
    amg_handle *h = nullptr;
    const double *b_in = nullptr, *b = nullptr;
    double *x_io = nullptr;
    bool x_dev = false, transpose = false, done = false;
    double tol = 0.0, bnorm = 0.0, relres = 0.0;
    int status = AMG_OK, total = 0, restarts = 0, j = 0;
    int64_t launches0 = 0;
    std::chrono::steady_clock::time_point t0;
};

static void start_cycle(Run &R) {
    amg_handle *h = R.h;
    if (R.relres <= R.tol) { R.done = true; return; }
    if (R.total >= h->opt.maxit) { R.status = AMG_ERR_NOT_CONVERGED; R.done = true; return; }
    // the state's nrm2 holds ||r||^2 from read_norm
    restart_scale(h->n, h->r.get(), h->V.get(), h->st.get(), h->stream);
    R.j = 0;
}

static void run_begin(Run &R) {
    amg_handle *h = R.h;
    R.t0 = std::chrono::steady_clock::now();
    R.launches0 = launch_count();
    enter(h);
    cudaStream_t s = h->stream;
    const size_t n = h->n;
    R.x_dev = is_device_ptr(R.x_io);
    // b in the handle's own buffer, so that a captured solve loop reads it
    CU(cudaMemcpyAsync(h->bb.get(), R.b_in, n * sizeof(double),
                       is_device_ptr(R.b_in) ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, s));
    R.b = h->bb.get();
    double *x = h->xb.get();
    if (R.x_dev) CU(cudaMemcpyAsync(x, R.x_io, n * sizeof(double), cudaMemcpyDeviceToDevice, s));
    else CU(cudaMemcpyAsync(x, R.x_io, n * sizeof(double), cudaMemcpyHostToDevice, s));
    FgState &hs = *h->hst;
    memset(&hs, 0, sizeof(FgState));
    hs.m = h->opt.restart; hs.maxit = h->opt.maxit; hs.hist_cap = h->opt.maxit + 2; hs.tol = R.tol;
    hs.loop_cap = h->opt.maxit + 16;      // one inner iteration per loop pass
    hs.hist = h->hist.get();
    h->last_hist.clear();
    R.bnorm = read_norm(h, R.b);
    if (!std::isfinite(R.bnorm)) { R.status = AMG_ERR_NUMERIC; R.done = true; return; }
    if (R.bnorm == 0.0) {
        CU(cudaMemsetAsync(x, 0, n * sizeof(double), s));
        h->last_hist.push_back(0.0);
        R.done = true;
        return;
    }
    hs.bnorm = R.bnorm;
    hs.hist_len = 1;
    CU(cudaMemcpyAsync(h->st.get(), &hs, sizeof(FgState), cudaMemcpyHostToDevice, s));
    outer_residual(h, R.b, x, h->r.get(), R.transpose);
    const double beta = read_norm(h, h->r.get());      // leaves ||r0||^2 in the state for the restart
    R.relres = beta / R.bnorm;
    CU(cudaMemcpyAsync(h->hist.get(), &R.relres, sizeof(double), cudaMemcpyHostToDevice, s));
    CU(cudaMemcpyAsync(&h->st.get()->relres, &R.relres, sizeof(double), cudaMemcpyHostToDevice, s));
    CU(cudaStreamSynchronize(s));
    if (!std::isfinite(R.relres)) { R.status = AMG_ERR_NUMERIC; R.done = true; return; }
    start_cycle(R);
}

static void end_cycle(Run &R) {
    amg_handle *h = R.h;
    cudaStream_t s = h->stream;
    FgState &hs = *h->hst;
    FgState *dst = h->st.get();
    CU(cudaMemcpyAsync(&hs, dst, sizeof(FgState), cudaMemcpyDeviceToHost, s));
    CU(cudaStreamSynchronize(s));
    R.total = hs.total;
    if (hs.status) { R.status = hs.status; R.done = true; return; }
    const size_t n = h->n;
    double *x = h->xb.get();
    backsolve(dst, s);
    if (h->opt.vcycle_prec == AMG_FP64) update_x<double>(n, dst, h->Zd.get(), n, x, s);
    else update_x<float>(n, dst, h->Zf.get(), n, x, s);
    outer_residual(h, R.b, x, h->r.get(), R.transpose);
    const double beta = read_norm(h, h->r.get());
    R.relres = beta / R.bnorm;
    if (!std::isfinite(R.relres)) { R.status = AMG_ERR_NUMERIC; R.done = true; return; }
    if (R.relres <= R.tol) { R.done = true; return; }
    if (R.total >= h->opt.maxit) { R.status = AMG_ERR_NOT_CONVERGED; R.done = true; return; }
    ++R.restarts;
    start_cycle(R);
}

static void run_launch(Run &R) { launch_iteration(R.h, R.transpose); }

static void run_collect(Run &R) {
    collect_iteration(R.h, R.transpose);
    ++R.j;
    if (R.h->hflags[0] || R.j >= R.h->opt.restart) end_cycle(R);
}

static int run_end(Run &R, amg_stats_t *stats) {
    amg_handle *h = R.h;
    cudaStream_t s = h->stream;
    const size_t n = h->n;
    FgState &hs = *h->hst;
    if (h->last_hist.empty() && R.bnorm != 0.0 && std::isfinite(R.bnorm)) {
        CU(cudaMemcpyAsync(&hs, h->st.get(), sizeof(FgState), cudaMemcpyDeviceToHost, s));
        CU(cudaStreamSynchronize(s));
        h->last_hist.resize(hs.hist_len);
        if (hs.hist_len)
            CU(cudaMemcpyAsync(h->last_hist.data(), h->hist.get(), sizeof(double) * hs.hist_len,
                               cudaMemcpyDeviceToHost, s));
    }
    double *x = h->xb.get();
    if (R.x_dev) CU(cudaMemcpyAsync(R.x_io, x, n * sizeof(double), cudaMemcpyDeviceToDevice, s));
    else CU(cudaMemcpyAsync(R.x_io, x, n * sizeof(double), cudaMemcpyDeviceToHost, s));
    int derr = 0;
    CU(cudaMemcpyAsync(&derr, h->err.get(), sizeof(int), cudaMemcpyDeviceToHost, s));
    CU(cudaStreamSynchronize(s));
    if (derr) {
        CU(cudaMemsetAsync(h->err.get(), 0, sizeof(int), s));
        CU(cudaMemsetAsync(h->bar.get(), 0, 2 * sizeof(unsigned int), s));
        CU(cudaStreamSynchronize(s));
        // a wait that gave up leaves values in place of sentinels: restore
        // them here (a captured graph does not refill them)
        for (auto &L : h->lev) {
            if (L->wy_sent == (int)sizeof(double))
                fill_sentinel<double>(reinterpret_cast<double *>(L->wy.get()), L->A.n, s);
            else if (L->wy_sent == (int)sizeof(float))
                fill_sentinel<float>(reinterpret_cast<float *>(L->wy.get()), L->A.n, s);
            if (L->tiles) tile_mailbox_reset(*L->tiles, s);
        }
        CU(cudaStreamSynchronize(s));
        t_last_error = "a grid-barrier, dataflow or tile wait gave up (results invalid)";
        R.status = AMG_ERR_LIMIT;
    }
    const auto t1 = std::chrono::steady_clock::now();
    if (stats) {
        stats->status = R.status;
        stats->iters = R.total;
        stats->restarts = R.restarts;
        stats->nlevels = (int)h->lev.size();
        stats->rel_res_true = R.relres;
        stats->setup_ms = h->setup_ms;
        stats->solve_ms = std::chrono::duration<double, std::milli>(t1 - R.t0).count();
        stats->n_coarse = h->lev.size() > 1 ? h->lev[1]->A.n : 0;
        stats->nnz_coarse = h->lev.size() > 1 ? h->lev[1]->A.nnz : 0;
        stats->n_colors = h->lev[0]->fwd.nlev;
        stats->kernel_launches = launch_count() - R.launches0;
    }
    return R.status;
}

// ------------------------------------------------------------------ device-driven loop
// The loop of run_collect / end_cycle as one CUDA graph per handle (or per
// batch): a WHILE conditional node whose body is one inner iteration (the
// kernels of enqueue_iteration) followed by an IF conditional node, taken
// when the iteration ended the cycle, holding the update x += Z y, the true
// residual, its norm, the convergence decision and the restart.  The loop
// ends on convergence, at the iteration cap, on a breakdown, or when a
// device wait gave up; the host reads the state once, after the loop.
// Kernel timing (event nodes) is not allowed in conditional bodies, so a
// handle with a timed kernel class runs the host-driven loop.
static bool device_loop_ok(const amg_handle *h) {
    return h->opt.solve_loop == AMG_LOOP_DEVICE && h->opt.use_graphs && h->tclass == 0;
}

static void capture_into(cudaStream_t s, cudaGraph_t g) {
    CU(cudaStreamBeginCaptureToGraph(s, g, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal));
}
static void end_capture(cudaStream_t s) {
    cudaGraph_t g = nullptr;
    CU(cudaStreamEndCapture(s, &g));
}
static cudaGraph_t capture_graph(cudaStream_t s) {
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    cudaGraph_t g = nullptr;
    CU(cudaStreamGetCaptureInfo(s, &cs, nullptr, &g, nullptr, nullptr, nullptr));
    if (cs != cudaStreamCaptureStatusActive || !g) fail(AMG_ERR_CUDA, "device loop: stream is not capturing");
    return g;
}
// Adds a conditional node after the capture's current tail on stream s and
// makes it the new tail; returns its body graph.
static cudaGraph_t add_conditional(cudaStream_t s, cudaGraphConditionalHandle c, cudaGraphConditionalNodeType type) {
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    cudaGraph_t g = nullptr;
    const cudaGraphNode_t *deps = nullptr;
    size_t nd = 0;
    CU(cudaStreamGetCaptureInfo(s, &cs, nullptr, &g, &deps, nullptr, &nd));
    if (cs != cudaStreamCaptureStatusActive || !g) fail(AMG_ERR_CUDA, "device loop: stream is not capturing");
    std::vector<cudaGraphNode_t> dv(deps, deps + nd);
    cudaGraphNodeParams p = {};
    p.type = cudaGraphNodeTypeConditional;
    p.conditional.handle = c;
    p.conditional.type = type;
    p.conditional.size = 1;
    cudaGraphNode_t node = nullptr;
    CU(cudaGraphAddNode(&node, g, dv.empty() ? nullptr : dv.data(), nullptr, dv.size(), &p));
    CU(cudaStreamUpdateCaptureDependencies(s, &node, nullptr, 1, cudaStreamSetCaptureDependencies));
    return p.conditional.phGraph_out[0];
}

// End of a cycle on stream s (the same kernels and order as end_cycle and
// start_cycle of the host-driven loop).
static void enqueue_cycle_end(amg_handle *h, bool transpose, cudaStream_t s) {
    const size_t n = h->n;
    FgState *dst = h->st.get();
    double *x = h->xb.get();
    backsolve(dst, s);
    if (h->opt.vcycle_prec == AMG_FP64) update_x<double>(n, dst, h->Zd.get(), n, x, s);
    else update_x<float>(n, dst, h->Zf.get(), n, x, s);
    Level &L0 = *h->lev[0];
    const Sell &SL = transpose ? L0.sellT : L0.sell;
    sell_spmv<double>(SL.n, SL.nslices, SL.ptr.get(), SL.ci.get(), SL.v.get(), x, h->bb.get(), h->r.get(), 1, s,
                      SL.block, SL.unroll);
    norm2(n, h->r.get(), h->partials.get(), h->ticket.get(), dst->nrm2, use_dot2(h), s);
    end_cycle_dev(dst, s);
    restart_scale(n, h->r.get(), h->V.get(), dst, s);
}

// Appends handle h's solve loop to graph G as a new root chain:
// loop_init -> WHILE { iteration; cycle_flag; IF { cycle end }; loop_flag }.
static void add_member_loop(amg_handle *h, bool transpose, cudaGraph_t G) {
    const int d = transpose ? 1 : 0;
    cudaStream_t s = h->stream;
    if (!h->aux) CU(cudaStreamCreateWithFlags(&h->aux, cudaStreamNonBlocking));
    FgState *dst = h->st.get();
    const int64_t l0 = launch_count();
    cudaGraphConditionalHandle w;
    CU(cudaGraphConditionalHandleCreate(&w, G, 0, 0));
    capture_into(s, G);
    loop_init(dst, w, s);
    cudaGraph_t body = add_conditional(s, w, cudaGraphCondTypeWhile);
    end_capture(s);
    const int64_t l1 = launch_count();
    capture_into(s, body);
    enqueue_iteration(h, transpose, false);
    cudaGraphConditionalHandle c;
    CU(cudaGraphConditionalHandleCreate(&c, capture_graph(s), 0, 0));
    cycle_flag(dst, c, s);
    cudaGraph_t endg = add_conditional(s, c, cudaGraphCondTypeIf);
    const int64_t l2 = launch_count();
    capture_into(h->aux, endg);
    enqueue_cycle_end(h, transpose, h->aux);
    end_capture(h->aux);
    const int64_t l3 = launch_count();
    loop_flag(dst, h->err.get(), w, s);
    end_capture(s);
    const int64_t l4 = launch_count();
    h->loop_nodes[d][0] = (l2 - l1) + (l4 - l3);     // kernels of one pass
    h->loop_nodes[d][1] = l3 - l2;                   // kernels of one cycle end
    count_launch(-(l4 - l0));                        // counted per executed node after the run
}

// Runs the solve loops of `runs` (begun with run_begin) as one graph on
// `owner`'s stream, built on first use and kept in `exec`.
static void run_device_loop(const std::vector<Run *> &runs, amg_handle *owner, cudaGraphExec_t &exec,
                            bool transpose) {
    if (!exec) {
        cudaGraph_t G = nullptr;
        CU(cudaGraphCreate(&G, 0));
        try {
            for (Run *R : runs) add_member_loop(R->h, transpose, G);
            CU(cudaGraphInstantiate(&exec, G, 0));
        } catch (...) {
            cudaGraphDestroy(G);
            exec = nullptr;
            throw;
        }
        cudaGraphDestroy(G);
    }
    static const int one = 1;
    for (Run *R : runs)
        if (R->done)        // finished in run_begin: its loop must not run
            CU(cudaMemcpyAsync(&R->h->st.get()->done, &one, sizeof(int), cudaMemcpyHostToDevice, R->h->stream));
    for (Run *R : runs) CU(cudaStreamSynchronize(R->h->stream));
    CU(cudaGraphLaunch(exec, owner->stream));
    count_launch(1);
    CU(cudaStreamSynchronize(owner->stream));
    const int d = transpose ? 1 : 0;
    for (Run *R : runs) {
        if (R->done) continue;
        amg_handle *h = R->h;
        FgState &hs = *h->hst;
        CU(cudaMemcpyAsync(&hs, h->st.get(), sizeof(FgState), cudaMemcpyDeviceToHost, owner->stream));
        CU(cudaStreamSynchronize(owner->stream));
        R->total = hs.total;
        R->restarts = hs.restarts;
        R->relres = hs.relres;
        R->status = hs.status;
        R->done = true;
        count_launch(hs.passes * h->loop_nodes[d][0] + (hs.restarts + (hs.passes > 0 ? 1 : 0)) * h->loop_nodes[d][1]);
    }
}

static int fgmres(amg_handle *h, const double *b_in, double *x_io, double tol, amg_stats_t *stats, bool transpose) {
    Run R;
    R.h = h; R.b_in = b_in; R.x_io = x_io; R.tol = tol; R.transpose = transpose;
    run_begin(R);
    if (!R.done && device_loop_ok(h)) {
        run_device_loop({&R}, h, h->lexec[transpose ? 1 : 0], transpose);
    } else {
        while (!R.done) {
            run_launch(R);
            run_collect(R);
        }
    }
    return run_end(R, stats);
}

}  // namespace amg

// Lets the other translation units of the ABI report a message through
// amg_last_error().
const char *amg_noalloc_set_error(const char *msg) {
    amg::t_last_error = msg;
    return amg::t_last_error.c_str();
}

// =================================================================== C ABI
using namespace amg;

#define ABI_TRY try {
#define ABI_CATCH                                                     \
    }                                                                 \
    catch (const amg::Error &e) {                                     \
        t_last_error = e.msg;                                         \
        return e.status;                                              \
    }                                                                 \
    catch (const std::bad_alloc &) {                                  \
        t_last_error = "host allocation failed";                      \
        return AMG_ERR_OOM;                                           \
    }                                                                 \
    catch (...) {                                                     \
        t_last_error = "unexpected exception";                        \
        return AMG_ERR_CUDA;                                          \
    }

extern "C" {

const char *amg_version(void) { return "amg_gb 0.1 (sm_103a)"; }

const char *amg_status_string(int st) {
    switch (st) {
    case AMG_OK: return "ok";
    case AMG_ERR_INVALID_ARG: return "invalid argument";
    case AMG_ERR_CUDA: return "CUDA error";
    case AMG_ERR_OOM: return "out of device memory";
    case AMG_ERR_NOT_SUPPORTED: return "not supported";
    case AMG_ERR_BREAKDOWN: return "breakdown (zero or non-finite pivot)";
    case AMG_ERR_NUMERIC: return "non-finite residual";
    case AMG_ERR_NOT_CONVERGED: return "not converged";
    case AMG_ERR_LIMIT: return "device loop limit reached";
    default: return "unknown status";
    }
}

const char *amg_last_error(void) { return t_last_error.c_str(); }

int amg_default_options(amg_options_t *o) {
    if (!o) return AMG_ERR_INVALID_ARG;
    memset(o, 0, sizeof(*o));
    o->passes = 2;
    o->coarse_inner = 5;
    o->deep_inner = 1;
    o->dense_max = 4096;
    o->max_levels = 12;
    o->order_fine = AMG_ORDER_NATURAL;
    o->order_coarse = AMG_ORDER_COLOR;
    o->coloring = AMG_COLOR_HASH_JP;
    o->restart = 30;
    o->maxit = 600;
    o->vcycle_prec = AMG_FP64;
    o->build_adjoint = 0;
    o->use_graphs = 1;
    o->persistent = 5;
    o->deep_block_max = 0;
    o->orthog = AMG_ORTHO_MGS;
    o->spmv_block = 0;
    o->spmv_unroll = 0;
    o->dot2 = -1;
    o->match_weight = AMG_MATCH_SCALED;
    o->seed = 0;
    o->coarse_solver = AMG_COARSE_RECURSIVE;
    o->solve_loop = AMG_LOOP_DEVICE;
    o->ilut_tau = 1e-6;
    return AMG_OK;
}

static void check_options(const amg_options_t &o) {
    if (o.passes < 1 || o.passes > 8 || o.coarse_inner < 1 || o.deep_inner < 1 || o.dense_max < 0 ||
        o.dense_max > 4096 || o.max_levels < 2 || o.max_levels > 24 || o.restart < 1 || o.restart > KMAX1 - 1 ||
        o.maxit < 0 || o.vcycle_prec < 0 || o.vcycle_prec > 3 || o.order_fine < 0 || o.order_fine > 1 ||
        o.order_coarse < 0 || o.order_coarse > 1 || o.coloring < 0 || o.coloring > 1 || o.deep_block_max < 0 ||
        o.persistent < 0 || o.persistent > 5 || o.orthog < 0 || o.orthog > 1 ||
        (o.spmv_block != 0 && o.spmv_block != 64 && o.spmv_block != 128 && o.spmv_block != 256 &&
         o.spmv_block != 512) ||
        (o.spmv_unroll != 0 && o.spmv_unroll != 2 && o.spmv_unroll != 4 && o.spmv_unroll != 8) || o.dot2 < -1 ||
        o.dot2 > 1 || o.match_weight < 0 || o.match_weight > 1 || o.solve_loop < 0 || o.solve_loop > 1 || o.coarse_solver < 0 || o.coarse_solver > 1 || !(o.ilut_tau >= 0.0) ||
        !std::isfinite(o.ilut_tau))
        fail(AMG_ERR_INVALID_ARG, "option out of range (restart <= 31, dense_max <= 4096, 2 <= max_levels <= 24)");
}

int amg_setup(const amg_csr_t *A, const amg_options_t *opt, void *stream, amg_handle_t **out) {
    if (out) *out = nullptr;
    ABI_TRY
    if (!A || !out) fail(AMG_ERR_INVALID_ARG, "amg_setup: null argument");
    auto t0 = std::chrono::steady_clock::now();
    std::unique_ptr<amg_handle> h(new amg_handle());
    if (opt) h->opt = *opt;
    else amg_default_options(&h->opt);
    check_options(h->opt);
    h->ustream = (cudaStream_t)stream;
    CU(cudaStreamCreateWithFlags(&h->stream, cudaStreamNonBlocking));
    CU(cudaEventCreateWithFlags(&h->entry_ev, cudaEventDisableTiming));
    enter(h.get());
    {
        AllocScope scope(h->stream);       // setup buffers: stream-ordered pool on the handle's stream
        setup_impl(h.get(), A);
    }
    h->setup_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    *out = h.release();
    return AMG_OK;
    ABI_CATCH
}

int amg_update_values(amg_handle_t *h, const double *val) {
    ABI_TRY
    if (!h || !val) fail(AMG_ERR_INVALID_ARG, "amg_update_values: null argument");
    if (!h->subs.empty()) fail(AMG_ERR_INVALID_ARG, "amg_update_values: batched handle");
    auto t0 = std::chrono::steady_clock::now();
    CU(cudaStreamSynchronize(h->stream));
    Level &L0 = *h->lev[0];
    const int n = L0.A.n;
    // copies of every level's per-pass maps: the aggregation, frozen (the
    // handle stays intact if the update fails)
    std::vector<std::vector<PassData>> frozen(h->lev.size());
    for (size_t l = 0; l < h->lev.size(); ++l)
        for (PassData &P : h->lev[l]->passes) {
            PassData f;
            f.agg.alloc((size_t)P.n_in);
            CU(cudaMemcpyAsync(f.agg.get(), P.agg.get(), sizeof(int) * (size_t)P.n_in, cudaMemcpyDeviceToDevice,
                               h->stream));
            f.n_in = P.n_in;
            f.n_out = P.n_out;
            frozen[l].push_back(std::move(f));
        }
    CU(cudaStreamSynchronize(h->stream));
    std::unique_ptr<amg_handle> nh(new amg_handle());
    nh->opt = h->opt;
    nh->ustream = h->ustream;
    CU(cudaStreamCreateWithFlags(&nh->stream, cudaStreamNonBlocking));
    CU(cudaEventCreateWithFlags(&nh->entry_ev, cudaEventDisableTiming));
    enter(nh.get());
    DBuf<int64_t> rp64((size_t)n + 1);
    k_rp32_to_64<<<grid_for((size_t)n + 1, 256), 256, 0, nh->stream>>>(n, L0.A.rp.get(), rp64.get());
    CU_LAUNCH("k_rp32_to_64"); count_launch();
    amg_csr_t A{n, (int64_t)L0.A.nnz, rp64.get(), L0.A.ci.get(), val};
    try {
        AllocScope scope(nh->stream);
        setup_impl(nh.get(), &A, &frozen);
        CU(cudaStreamSynchronize(nh->stream));
    } catch (...) {
        amg_destroy(nh.release());          // the handle keeps its previous hierarchy
        throw;
    }
    std::swap(h->lev, nh->lev);
    std::swap(h->n, nh->n);
    std::swap(h->V, nh->V); std::swap(h->Zd, nh->Zd); std::swap(h->w, nh->w); std::swap(h->r, nh->r);
    std::swap(h->xb, nh->xb); std::swap(h->bb, nh->bb); std::swap(h->hist, nh->hist);
    std::swap(h->partials, nh->partials); std::swap(h->zin64, nh->zin64); std::swap(h->zout64, nh->zout64);
    std::swap(h->Zf, nh->Zf); std::swap(h->zin32, nh->zin32); std::swap(h->zout32, nh->zout32);
    std::swap(h->hflags, nh->hflags);
    for (int d = 0; d < 2; ++d) {
        std::swap(h->gexec[d], nh->gexec[d]);
        std::swap(h->lexec[d], nh->lexec[d]);
        std::swap(h->gpairs[d], nh->gpairs[d]);
        std::swap(h->gnodes[d], nh->gnodes[d]);
        std::swap(h->gbytes[d], nh->gbytes[d]);
    }
    std::swap(h->st, nh->st); std::swap(h->ticket, nh->ticket); std::swap(h->bar, nh->bar);
    std::swap(h->err, nh->err); std::swap(h->hst, nh->hst);
    std::swap(h->adjoint_ready, nh->adjoint_ready);
    std::swap(h->deep_first, nh->deep_first);
    std::swap(h->deep_desc, nh->deep_desc);
    h->last_hist.clear();
    h->setup_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    amg_destroy(nh.release());              // frees the previous hierarchy and its graphs
    return AMG_OK;
    ABI_CATCH
}

void amg_destroy(amg_handle_t *h) {
    if (!h) return;
    for (amg_handle *sub : h->subs) amg_destroy(sub);
    h->subs.clear();
    try {
        cudaStreamSynchronize(h->stream);
        if (h->hst) cudaFreeHost(h->hst);
        if (h->hflags) cudaFreeHost(h->hflags);
        for (auto &g : h->gexec) if (g) cudaGraphExecDestroy(g);
        for (auto &g : h->lexec) if (g) cudaGraphExecDestroy(g);
        for (auto &g : h->bexec) if (g) cudaGraphExecDestroy(g);
        if (h->aux) cudaStreamDestroy(h->aux);
        h->lev.clear();
        h->V.release(); h->Zd.release(); h->Zf.release();
        if (h->entry_ev) cudaEventDestroy(h->entry_ev);
        if (h->stream) cudaStreamDestroy(h->stream);
        for (auto &e : h->tev) { cudaEventDestroy(e.first); cudaEventDestroy(e.second); }
        delete h;
    } catch (...) {
    }
}

int amg_solve(amg_handle_t *h, const double *b, double *x, double tol, amg_stats_t *stats) {
    ABI_TRY
    if (!h || !b || !x) fail(AMG_ERR_INVALID_ARG, "amg_solve: null argument");
    if (!h->subs.empty()) fail(AMG_ERR_INVALID_ARG, "amg_solve: batched handle (use amg_solve_batched)");
    if (!(tol >= 0.0)) fail(AMG_ERR_INVALID_ARG, "amg_solve: tol must be >= 0");
    return fgmres(h, b, x, tol, stats, false);
    ABI_CATCH
}

int amg_adjoint(amg_handle_t *h, const double *g, double *lambda, double tol, amg_stats_t *stats) {
    ABI_TRY
    if (!h || !g || !lambda) fail(AMG_ERR_INVALID_ARG, "amg_adjoint: null argument");
    if (!h->subs.empty()) fail(AMG_ERR_INVALID_ARG, "amg_adjoint: batched handle");
    if (!h->adjoint_ready) fail(AMG_ERR_INVALID_ARG, "amg_adjoint: setup without build_adjoint");
    if (!(tol >= 0.0)) fail(AMG_ERR_INVALID_ARG, "amg_adjoint: tol must be >= 0");
    return fgmres(h, g, lambda, tol, stats, true);
    ABI_CATCH
}

int amg_setup_batched(const amg_csr_t *systems, int32_t count, const amg_options_t *opt, void *stream,
                      amg_handle_t **out) {
    if (out) *out = nullptr;
    ABI_TRY
    if (!systems || count <= 0 || !out) fail(AMG_ERR_INVALID_ARG, "amg_setup_batched: bad argument");
    auto t0 = std::chrono::steady_clock::now();
    std::unique_ptr<amg_handle> B(new amg_handle());
    if (opt) B->opt = *opt;
    else amg_default_options(&B->opt);
    check_options(B->opt);
    B->ustream = (cudaStream_t)stream;
    CU(cudaStreamCreateWithFlags(&B->stream, cudaStreamNonBlocking));
    B->subs.assign(count, nullptr);
    // independent systems: set up concurrently from a few host threads, each
    // system on its own internal stream
    int dev = 0;
    CU(cudaGetDevice(&dev));
    std::vector<int> st(count, AMG_OK);
    std::vector<std::string> msg(count);
    std::atomic<int> next{0};
    std::atomic<int64_t> launches{0};
    // 8 host threads: each member's setup is a chain of short launches and
    // synchronisations, so members overlap on the GPU (16 threads measured
    // slower on the batch workload: setup 3.72 s against 3.47 s)
    const int nth = std::max(1, std::min<int>(count, 8));
    auto work = [&]() {
        cudaSetDevice(dev);
        const int64_t l0 = launch_count();
        for (;;) {
            const int k = next.fetch_add(1);
            if (k >= count) break;
            amg_handle_t *sub = nullptr;
            st[k] = amg_setup(&systems[k], &B->opt, stream, &sub);
            if (st[k] != AMG_OK) msg[k] = amg_last_error();
            B->subs[k] = sub;
        }
        launches += launch_count() - l0;
    };
    std::vector<std::thread> th;
    for (int t = 0; t < nth; ++t) th.emplace_back(work);
    for (auto &t : th) t.join();
    count_launch(launches.load());
    for (int k = 0; k < count; ++k)
        if (st[k] != AMG_OK) {
            const int code = st[k];
            const std::string m = "system " + std::to_string(k) + ": " + msg[k];
            for (amg_handle *sub : B->subs) amg_destroy(sub);
            B->subs.clear();
            fail(code, m);
        }
    B->offs.assign(count + 1, 0);
    for (int k = 0; k < count; ++k) B->offs[k + 1] = B->offs[k] + systems[k].n;
    B->n = (int)std::min<int64_t>(B->offs[count], 0x7fffffff);
    B->setup_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    *out = B.release();
    return AMG_OK;
    ABI_CATCH
}

int amg_solve_batched(amg_handle_t *h, const double *b_cat, double *x_cat, double tol, amg_stats_t *per_system) {
    ABI_TRY
    if (!h || h->subs.empty() || !b_cat || !x_cat) fail(AMG_ERR_INVALID_ARG, "amg_solve_batched: bad argument");
    if (!(tol >= 0.0)) fail(AMG_ERR_INVALID_ARG, "amg_solve_batched: tol must be >= 0");
    const int count = (int)h->subs.size();
    std::vector<Run> R(count);
    CU(cudaStreamSynchronize(h->ustream));
    for (int k = 0; k < count; ++k) {
        R[k].h = h->subs[k];
        R[k].b_in = b_cat + h->offs[k];
        R[k].x_io = x_cat + h->offs[k];
        R[k].tol = tol;
        R[k].h->ustream = h->ustream;
        run_begin(R[k]);
    }
    bool device = true;
    for (int k = 0; k < count; ++k) device = device && device_loop_ok(h->subs[k]);
    if (device) {
        // every member's loop in one graph (parallel root chains), masks in
        // device memory: one launch and one synchronisation for the batch
        std::vector<Run *> runs(count);
        for (int k = 0; k < count; ++k) runs[k] = &R[k];
        run_device_loop(runs, h, h->bexec[0], false);
    } else {
        // host-driven: every active system queues its inner iteration on its
        // own stream, then each is collected; converged systems drop out
        for (;;) {
            bool any = false;
            for (int k = 0; k < count; ++k)
                if (!R[k].done) { run_launch(R[k]); any = true; }
            if (!any) break;
            for (int k = 0; k < count; ++k)
                if (!R[k].done) run_collect(R[k]);
        }
    }
    int status = AMG_OK;
    for (int k = 0; k < count; ++k) {
        const int sk = run_end(R[k], per_system ? per_system + k : nullptr);
        if (sk != AMG_OK && (status == AMG_OK || status == AMG_ERR_NOT_CONVERGED)) status = sk;
    }
    return status;
    ABI_CATCH
}

int amg_batch_size(amg_handle_t *h, int32_t *count, int64_t *offsets) {
    ABI_TRY
    if (!h || !count) fail(AMG_ERR_INVALID_ARG, "amg_batch_size: null argument");
    *count = (int32_t)h->subs.size();
    if (offsets)
        for (size_t k = 0; k < h->offs.size(); ++k) offsets[k] = h->offs[k];
    return AMG_OK;
    ABI_CATCH
}

amg_handle_t *amg_batch_member(amg_handle_t *h, int32_t k) {
    if (!h || k < 0 || k >= (int)h->subs.size()) return nullptr;
    return h->subs[k];
}

int amg_get_history(amg_handle_t *h, double *out, int32_t cap, int32_t *len) {
    ABI_TRY
    if (!h || !len) fail(AMG_ERR_INVALID_ARG, "amg_get_history: null argument");
    *len = (int32_t)h->last_hist.size();
    if (out) for (int i = 0; i < cap && i < *len; ++i) out[i] = h->last_hist[i];
    return AMG_OK;
    ABI_CATCH
}

int amg_precond_apply(amg_handle_t *h, const double *z, double *q, int32_t transpose) {
    ABI_TRY
    if (!h || !z || !q) fail(AMG_ERR_INVALID_ARG, "amg_precond_apply: null argument");
    if (transpose && !h->adjoint_ready) fail(AMG_ERR_INVALID_ARG, "amg_precond_apply: no adjoint structures");
    if (!is_device_ptr(z) || !is_device_ptr(q)) fail(AMG_ERR_INVALID_ARG, "amg_precond_apply: device pointers required");
    enter(h);
    const size_t n = h->n;
    if (h->opt.vcycle_prec == AMG_FP64) {
        CU(cudaMemcpyAsync(h->zin64.get(), z, n * sizeof(double), cudaMemcpyDeviceToDevice, h->stream));
        apply_precond_vtype(h, transpose != 0);
        CU(cudaMemcpyAsync(q, h->zout64.get(), n * sizeof(double), cudaMemcpyDeviceToDevice, h->stream));
    } else {
        convert_f64_f32(n, z, h->zin32.get(), h->stream);
        apply_precond_vtype(h, transpose != 0);
        convert_f32_f64(n, h->zout32.get(), q, h->stream);
    }
    CU(cudaStreamSynchronize(h->stream));
    return AMG_OK;
    ABI_CATCH
}

int amg_spmv(const amg_csr_t *A, const double *x, double *y, void *stream) {
    ABI_TRY
    if (!A || !x || !y || A->n <= 0 || !A->row_ptr) fail(AMG_ERR_INVALID_ARG, "amg_spmv: bad argument");
    if (A->nnz >= (int64_t)0x7fffffff) fail(AMG_ERR_INVALID_ARG, "amg_spmv: nnz >= 2^31");
    cudaStream_t s = (cudaStream_t)stream;
    DBuf<int> rp32(A->n + 1), bad(1);
    CU(cudaMemsetAsync(bad.get(), 0, sizeof(int), s));
    k_rp64_to_32<<<grid_for((size_t)A->n + 1, 256), 256, 0, s>>>(A->n, A->nnz, A->row_ptr, rp32.get(), bad.get());
    CU_LAUNCH("k_rp64_to_32"); count_launch();
    spmv_f64_checked(A->n, (int)A->nnz, rp32.get(), A->col, A->val, x, y, bad.get(), s);
    int hbad = 0;
    CU(cudaMemcpyAsync(&hbad, bad.get(), sizeof(int), cudaMemcpyDeviceToHost, s));
    CU(cudaStreamSynchronize(s));
    if (hbad) fail(AMG_ERR_INVALID_ARG, "amg_spmv: row pointers not a valid sequence from 0 to nnz, or columns out of range");
    return AMG_OK;
    ABI_CATCH
}

int amg_set_kernel_timing(amg_handle_t *h, int32_t kclass) {
    ABI_TRY
    if (!h || kclass < 0 || kclass > 3) fail(AMG_ERR_INVALID_ARG, "amg_set_kernel_timing: bad argument");
    h->tclass = kclass;
    h->t_ms = 0.0; h->t_bytes = 0.0; h->t_launches = 0; h->tused = 0;
    return AMG_OK;
    ABI_CATCH
}

int amg_get_kernel_timing(amg_handle_t *h, double *ms_total, int64_t *launches, double *bytes_total) {
    ABI_TRY
    if (!h || !ms_total || !launches || !bytes_total) fail(AMG_ERR_INVALID_ARG, "amg_get_kernel_timing: null");
    CU(cudaStreamSynchronize(h->stream));
    tcollect(h);
    *ms_total = h->t_ms;
    *launches = h->t_launches;
    *bytes_total = h->t_bytes;
    return AMG_OK;
    ABI_CATCH
}

int64_t amg_launch_counter(void) { return launch_count(); }

int amg_num_levels(amg_handle_t *h, int32_t *nlevels) {
    if (!h || !nlevels) return AMG_ERR_INVALID_ARG;
    *nlevels = (int32_t)h->lev.size();
    return AMG_OK;
}

static Level &level_of(amg_handle_t *h, int l) {
    if (!h || l < 0 || l >= (int)h->lev.size()) fail(AMG_ERR_INVALID_ARG, "level out of range");
    return *h->lev[l];
}

int amg_get_spmv_config(amg_handle_t *h, int32_t *block, int32_t *unroll) {
    ABI_TRY
    if (!h || !block || !unroll) fail(AMG_ERR_INVALID_ARG, "amg_get_spmv_config: null argument");
    if (h->lev.empty()) fail(AMG_ERR_INVALID_ARG, "amg_get_spmv_config: batch handle (ask a member)");
    *block = h->lev[0]->sell.block;
    *unroll = h->lev[0]->sell.unroll;
    return AMG_OK;
    ABI_CATCH
}

int amg_get_level_info(amg_handle_t *h, int32_t level, int64_t *info) {
    ABI_TRY
    if (!info) fail(AMG_ERR_INVALID_ARG, "null info");
    Level &L = level_of(h, level);
    info[0] = L.A.n;
    info[1] = L.A.nnz;
    info[2] = L.dense ? 0 : L.fwd.nlev;
    info[3] = L.dense ? 1 : 0;
    info[4] = L.passes.empty() ? -1 : L.passes[0].n_out;
    info[5] = L.n_next;
    info[6] = L.ncol;
    info[7] = L.dense ? 0 : L.bwd.nlev;
    return AMG_OK;
    ABI_CATCH
}

int amg_get_tile_grid(amg_handle_t *h, int64_t *info) {
    ABI_TRY
    if (!h || !info) fail(AMG_ERR_INVALID_ARG, "null argument");
    if (!h->subs.empty()) fail(AMG_ERR_INVALID_ARG, "amg_get_tile_grid: batched handle");
    const TilePlan *P = h->lev[0]->tiles.get();
    for (int q = 0; q < 8; ++q) info[q] = 0;
    if (P) {
        const TileGeom &g = P->g;
        info[0] = 1;
        info[1] = g.nx; info[2] = g.ny; info[3] = g.nz;
        info[4] = g.tx; info[5] = g.ty; info[6] = g.tz;
        info[7] = g.ntiles;
    }
    return AMG_OK;
    ABI_CATCH
}

int amg_get_sweep_kind(amg_handle_t *h, int32_t level, int32_t *kind) {
    ABI_TRY
    if (!kind) fail(AMG_ERR_INVALID_ARG, "null kind");
    Level &L = level_of(h, level);
    kind[0] = L.sweep_kind[0];
    kind[1] = L.sweep_kind[1];
    return AMG_OK;
    ABI_CATCH
}

int amg_get_aggregates(amg_handle_t *h, int32_t level, int32_t pass, int32_t *out) {
    ABI_TRY
    Level &L = level_of(h, level);
    if (!out || L.n_next < 0) fail(AMG_ERR_INVALID_ARG, "no aggregation on this level");
    if (pass == 0) {
        CU(cudaMemcpy(out, L.agg.get(), sizeof(int) * L.A.n, cudaMemcpyDeviceToHost));
    } else {
        if (pass < 1 || pass > (int)L.passes.size()) fail(AMG_ERR_INVALID_ARG, "pass out of range");
        const PassData &P = L.passes[pass - 1];
        CU(cudaMemcpy(out, P.agg.get(), sizeof(int) * P.n_in, cudaMemcpyDeviceToHost));
    }
    return AMG_OK;
    ABI_CATCH
}

static void csr_to_host(const DCsr &M, int64_t *rp, int32_t *col, double *val) {
    std::vector<int> r32(M.n + 1);
    CU(cudaMemcpy(r32.data(), M.rp.get(), sizeof(int) * (M.n + 1), cudaMemcpyDeviceToHost));
    for (int i = 0; i <= M.n; ++i) rp[i] = r32[i];
    if (M.nnz) {
        CU(cudaMemcpy(col, M.ci.get(), sizeof(int) * M.nnz, cudaMemcpyDeviceToHost));
        CU(cudaMemcpy(val, M.v.get(), sizeof(double) * M.nnz, cudaMemcpyDeviceToHost));
    }
}

int amg_get_matrix(amg_handle_t *h, int32_t level, int64_t *rp, int32_t *col, double *val) {
    ABI_TRY
    Level &L = level_of(h, level);
    if (!rp || !col || !val) fail(AMG_ERR_INVALID_ARG, "null output");
    csr_to_host(L.A, rp, col, val);
    return AMG_OK;
    ABI_CATCH
}

int amg_get_pass_matrix(amg_handle_t *h, int32_t level, int32_t pass, int64_t *info, int64_t *rp, int32_t *col,
                        double *val) {
    ABI_TRY
    Level &L = level_of(h, level);
    if (pass < 1 || pass >= (int)L.passes.size()) fail(AMG_ERR_INVALID_ARG, "pass out of range");
    const DCsr &M = L.passes[pass - 1].mat;
    if (info) { info[0] = M.n; info[1] = M.nnz; }
    if (rp) {
        if (!col || !val) fail(AMG_ERR_INVALID_ARG, "null output");
        csr_to_host(M, rp, col, val);
    }
    return AMG_OK;
    ABI_CATCH
}

int amg_get_colors(amg_handle_t *h, int32_t level, int32_t *out) {
    ABI_TRY
    Level &L = level_of(h, level);
    if (!out || L.dense) fail(AMG_ERR_INVALID_ARG, "no elimination order on this level");
    CU(cudaMemcpy(out, L.label.get(), sizeof(int) * L.A.n, cudaMemcpyDeviceToHost));
    return AMG_OK;
    ABI_CATCH
}

int amg_get_ilu(amg_handle_t *h, int32_t level, double *out) {
    ABI_TRY
    Level &L = level_of(h, level);
    if (!out || L.dense || L.ilut_level)   // ILUT factors have their own pattern
        fail(AMG_ERR_INVALID_ARG, "no ILU(0) factors on this level");
    CU(cudaMemcpy(out, L.lu.get(), sizeof(double) * L.A.nnz, cudaMemcpyDeviceToHost));
    return AMG_OK;
    ABI_CATCH
}

int amg_fv_assemble(int32_t dim, int32_t nx, int32_t ny, int32_t nz, const double *kx, const double *ky,
                    const double *kz, const double *fx, const double *fy, const double *fz, const double *f,
                    int64_t *row_ptr, int32_t *col, double *val, double *b, int64_t *nnz_out, void *stream) {
    ABI_TRY
    if ((dim != 2 && dim != 3) || nx <= 0 || ny <= 0 || nz <= 0 || (dim == 2 && nz != 1))
        fail(AMG_ERR_INVALID_ARG, "amg_fv_assemble: bad grid");
    if ((int64_t)nx * ny * nz * (2 * dim + 1) >= (int64_t)0x7fffffff) fail(AMG_ERR_INVALID_ARG, "grid too large");
    if (!kx || !ky || !fx || !fy || !f || !row_ptr || !col || !val || !b || !nnz_out || (dim == 3 && (!kz || !fz)))
        fail(AMG_ERR_INVALID_ARG, "amg_fv_assemble: null pointer");
    *nnz_out = fv_assemble(dim, nx, ny, nz, kx, ky, kz, fx, fy, fz, f, row_ptr, col, val, b, (cudaStream_t)stream);
    return AMG_OK;
    ABI_CATCH
}

int amg_fv_assemble_logk(int32_t dim, int32_t nx, int32_t ny, int32_t nz, const double *logk, double *kappa,
                         const double *fx, const double *fy, const double *fz, const double *f, int64_t *row_ptr,
                         int32_t *col, double *val, double *b, int64_t *nnz_out, void *stream) {
    ABI_TRY
    if ((dim != 2 && dim != 3) || nx <= 0 || ny <= 0 || nz <= 0 || (dim == 2 && nz != 1))
        fail(AMG_ERR_INVALID_ARG, "amg_fv_assemble_logk: bad grid");
    if ((int64_t)nx * ny * nz * (2 * dim + 1) >= (int64_t)0x7fffffff) fail(AMG_ERR_INVALID_ARG, "grid too large");
    if (!logk || !kappa || !fx || !fy || !f || !row_ptr || !col || !val || !b || !nnz_out || (dim == 3 && !fz))
        fail(AMG_ERR_INVALID_ARG, "amg_fv_assemble_logk: null pointer");
    cudaStream_t s = (cudaStream_t)stream;
    exp_f64((long)nx * ny * nz, logk, kappa, s);
    *nnz_out = fv_assemble(dim, nx, ny, nz, kappa, kappa, kappa, fx, fy, fz, f, row_ptr, col, val, b, s);
    return AMG_OK;
    ABI_CATCH
}

__global__ void k_csr_outer_grad(int n, const int64_t *rp, const int32_t *ci, const double *lam, const double *x,
                                 double *g) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const double li = lam[i];
        for (int64_t e = rp[i]; e < rp[i + 1]; ++e) g[e] = -li * x[ci[e]];
    }
}

int amg_csr_value_grad(const amg_csr_t *A, const double *lambda, const double *x, double *grad_val, void *stream) {
    ABI_TRY
    if (!A || !A->row_ptr || !A->col || !lambda || !x || !grad_val || A->n <= 0)
        fail(AMG_ERR_INVALID_ARG, "amg_csr_value_grad: bad argument");
    cudaStream_t s = (cudaStream_t)stream;
    k_csr_outer_grad<<<grid_for(A->n, 256), 256, 0, s>>>(A->n, A->row_ptr, A->col, lambda, x, grad_val);
    CU_LAUNCH("k_csr_outer_grad"); count_launch();
    return AMG_OK;
    ABI_CATCH
}

int amg_fv_grad_logk(int32_t dim, int32_t nx, int32_t ny, int32_t nz, const double *kx, const double *ky,
                     const double *kz, const double *lambda, const double *x, double *gx, double *gy, double *gz,
                     void *stream) {
    ABI_TRY
    if ((dim != 2 && dim != 3) || nx <= 0 || ny <= 0 || nz <= 0 || (dim == 2 && nz != 1))
        fail(AMG_ERR_INVALID_ARG, "amg_fv_grad_logk: bad grid");
    if (!kx || !ky || !lambda || !x || !gx || !gy || (dim == 3 && (!kz || !gz)))
        fail(AMG_ERR_INVALID_ARG, "amg_fv_grad_logk: null pointer");
    fv_grad_logk(dim, nx, ny, nz, kx, ky, kz, lambda, x, gx, gy, gz, (cudaStream_t)stream);
    CU(cudaStreamSynchronize((cudaStream_t)stream));
    return AMG_OK;
    ABI_CATCH
}

int amg_fv_grad_logk_iso(int32_t dim, int32_t nx, int32_t ny, int32_t nz, const double *kappa,
                         const double *lambda, const double *x, double *g, void *stream) {
    ABI_TRY
    if ((dim != 2 && dim != 3) || nx <= 0 || ny <= 0 || nz <= 0 || (dim == 2 && nz != 1))
        fail(AMG_ERR_INVALID_ARG, "amg_fv_grad_logk_iso: bad grid");
    if (!kappa || !lambda || !x || !g) fail(AMG_ERR_INVALID_ARG, "amg_fv_grad_logk_iso: null pointer");
    fv_grad_logk(dim, nx, ny, nz, kappa, kappa, kappa, lambda, x, g, nullptr, nullptr, (cudaStream_t)stream);
    CU(cudaStreamSynchronize((cudaStream_t)stream));
    return AMG_OK;
    ABI_CATCH
}

}  // extern "C"
