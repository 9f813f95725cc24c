// setup.cu -- GPU setup phase of the matching-aggregation AMG hierarchy
// (Algorithm 1, setup): heavy-edge matching, aggregates,
// Galerkin products P^T A P, colourings, ILU(0) factors with their sweep
// schedules, the dense inverse of the last level, precision casts, and the
// finite-volume assembly of eq. (2).
//
// Every floating-point step that feeds an integer decision (matching keys)
// or a later level (Galerkin sums, ILU factors) uses explicitly rounded
// intrinsics (__dadd_rn, __dmul_rn, ...) so that no multiply-add is fused:
// the results are bit-identical to the plain sequential definition.
#include "internal.cuh"
#include "devsync.cuh"

#include <cmath>
#include <cstdio>

namespace amg {

// ------------------------------------------------------------------ helpers
__device__ __forceinline__ uint64_t mix64(uint64_t z) {
    // SplitMix64 output finaliser (Steele, Lea, Flood 2014)
    z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
    z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
    return z ^ (z >> 31);
}

__device__ __forceinline__ int find_col(const int *ci, int b, int e, int c) {
    int lo = b, hi = e - 1;
    while (lo <= hi) {
        int mid = (lo + hi) >> 1;
        int x = ci[mid];
        if (x == c) return mid;
        if (x < c) lo = mid + 1; else hi = mid - 1;
    }
    return -1;
}

template <typename T>
__device__ __forceinline__ T ld_volatile(const T *p) { return *(const volatile T *)p; }

struct Flags {   // device-side status words
    int a, b, c, d;
};

static int read_int(const int *d, cudaStream_t s) {
    int h = 0;
    CU(cudaMemcpyAsync(&h, d, sizeof(int), cudaMemcpyDeviceToHost, s));
    CU(cudaStreamSynchronize(s));
    return h;
}

// ------------------------------------------------------------------ validation
__global__ void k_validate(int n, const int *rp, const int *ci, int *bad) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        int b = rp[i], e = rp[i + 1];
        bool ok = e >= b, diag = false;
        for (int k = b; ok && k < e; ++k) {
            int c = ci[k];
            if (c < 0 || c >= n) ok = false;
            if (k > b && c <= ci[k - 1]) ok = false;
            if (c == i) diag = true;
        }
        if (!ok || !diag) atomicAdd(bad, 1);
    }
}

int csr_validate(int n, const int *rp, const int *ci, cudaStream_t s) {
    DBuf<int> bad(1);
    CU(cudaMemsetAsync(bad.get(), 0, sizeof(int), s));
    k_validate<<<grid_for(n, 256), 256, 0, s>>>(n, rp, ci, bad.get());
    CU_LAUNCH("k_validate"); count_launch();
    return read_int(bad.get(), s);
}

// ------------------------------------------------------------------ symmetrised adjacency
__global__ void k_sym_count(int n, const int *rp, const int *ci, const int *trp, const int *tci, int *cnt) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        int p = rp[i], pe = rp[i + 1], q = trp[i], qe = trp[i + 1], m = 0;
        while (p < pe || q < qe) {
            int c;
            if (q >= qe || (p < pe && ci[p] < tci[q])) c = ci[p++];
            else if (p >= pe || tci[q] < ci[p]) c = tci[q++];
            else { c = ci[p]; ++p; ++q; }
            if (c != i) ++m;
        }
        cnt[i] = m;
    }
}

__global__ void k_sym_fill(int n, const int *rp, const int *ci, const int *trp, const int *tci,
                           const int *arp, int *aci) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        int p = rp[i], pe = rp[i + 1], q = trp[i], qe = trp[i + 1], m = arp[i];
        while (p < pe || q < qe) {
            int c;
            if (q >= qe || (p < pe && ci[p] < tci[q])) c = ci[p++];
            else if (p >= pe || tci[q] < ci[p]) c = tci[q++];
            else { c = ci[p]; ++p; ++q; }
            if (c != i) aci[m++] = c;
        }
    }
}

void sym_adjacency(const DCsr &A, DBuf<int> &arp, DBuf<int> &aci, int &annz, cudaStream_t s) {
    DBuf<int> trp, tci, tsrc;
    csr_transpose(A.n, A.nnz, A.rp.get(), A.ci.get(), trp, tci, tsrc, s);
    DBuf<int> cnt(A.n + 1);
    fill_int(cnt.get(), 0, A.n + 1, s);
    k_sym_count<<<grid_for(A.n, 256), 256, 0, s>>>(A.n, A.rp.get(), A.ci.get(), trp.get(), tci.get(), cnt.get());
    CU_LAUNCH("k_sym_count"); count_launch();
    arp.alloc(A.n + 1);
    exclusive_scan_int(cnt.get(), arp.get(), A.n + 1, &annz, s);
    aci.alloc(annz > 0 ? annz : 1);
    k_sym_fill<<<grid_for(A.n, 256), 256, 0, s>>>(A.n, A.rp.get(), A.ci.get(), trp.get(), tci.get(), arp.get(), aci.get());
    CU_LAUNCH("k_sym_fill"); count_launch();
    CU(cudaStreamSynchronize(s));
}

// ------------------------------------------------------------------ matching
// Edge {u,v}, u < v: w = (|a_uv| + |a_vu|) * 0.5, missing entry = 0; with the
// scaled weight (scaled = 1) w is divided by sqrt(|a_uu| |a_vv|) (the product
// rounded, then the correctly rounded square root), the strength of
// connection of smoothed aggregation (Vanek, Mandel, Brezina 1996); key
// (w, mix64(((u<<32)|v) ^ seed), u, v), larger first.  Each round, every
// free vertex proposes to its largest-key free neighbour; mutual proposals
// are matched.  Mutual maxima of a strict total order are exactly the
// edges a greedy pass in decreasing key order takes, so the fixed point is
// the greedy matching.
__global__ void k_edge_weights(int n, const int *rp, const int *ci, const double *v, const int *arp,
                               const int *aci, int scaled, double *aw) {
    for (int u = blockIdx.x * blockDim.x + threadIdx.x; u < n; u += gridDim.x * blockDim.x) {
        double du = 0.0;
        if (scaled) {
            int eu = find_col(ci, rp[u], rp[u + 1], u);
            du = eu >= 0 ? fabs(v[eu]) : 0.0;
        }
        for (int e = arp[u]; e < arp[u + 1]; ++e) {
            int w = aci[e];
            int lo = u < w ? u : w, hi = u < w ? w : u;
            int e1 = find_col(ci, rp[lo], rp[lo + 1], hi);
            int e2 = find_col(ci, rp[hi], rp[hi + 1], lo);
            double a1 = e1 >= 0 ? fabs(v[e1]) : 0.0;
            double a2 = e2 >= 0 ? fabs(v[e2]) : 0.0;
            double wt = __dmul_rn(__dadd_rn(a1, a2), 0.5);
            if (scaled && wt > 0.0) {
                int ew = find_col(ci, rp[w], rp[w + 1], w);
                double dw = ew >= 0 ? fabs(v[ew]) : 0.0;
                wt = __ddiv_rn(wt, __dsqrt_rn(__dmul_rn(du, dw)));
            }
            aw[e] = wt;
        }
    }
}

struct EKey {
    double w;
    uint64_t h;
    int lo, hi;
};

__device__ __forceinline__ bool key_greater(const EKey &a, const EKey &b) {
    if (a.w != b.w) return a.w > b.w;
    if (a.h != b.h) return a.h > b.h;
    if (a.lo != b.lo) return a.lo > b.lo;
    return a.hi > b.hi;
}

__global__ void k_propose(int n, const int *arp, const int *aci, const double *aw, uint64_t seed,
                          int *mate, int *prop, int *active) {
    int cnt = 0;
    for (int u = blockIdx.x * blockDim.x + threadIdx.x; u < n; u += gridDim.x * blockDim.x) {
        if (ld_volatile(mate + u) != -1) { prop[u] = -1; continue; }
        int best = -1;
        EKey bk{0.0, 0, 0, 0};
        for (int e = arp[u]; e < arp[u + 1]; ++e) {
            int v = aci[e];
            double w = aw[e];
            if (!(w > 0.0)) continue;
            if (ld_volatile(mate + v) != -1) continue;
            int lo = u < v ? u : v, hi = u < v ? v : u;
            EKey k{w, mix64((((uint64_t)(uint32_t)lo) << 32 | (uint64_t)(uint32_t)hi) ^ seed), lo, hi};
            if (best < 0 || key_greater(k, bk)) { best = v; bk = k; }
        }
        prop[u] = best;
        if (best < 0) mate[u] = -2;      // no free neighbour left: stays a singleton
        else ++cnt;
    }
    if (cnt) atomicAdd(active, cnt);
}

__global__ void k_accept(int n, int *mate, const int *prop) {
    for (int u = blockIdx.x * blockDim.x + threadIdx.x; u < n; u += gridDim.x * blockDim.x) {
        int v = prop[u];
        if (v >= 0 && prop[v] == u) mate[u] = v;
    }
}

__global__ void k_unmark_dead(int n, int *mate) {
    for (int u = blockIdx.x * blockDim.x + threadIdx.x; u < n; u += gridDim.x * blockDim.x)
        if (mate[u] < 0) mate[u] = -1;
}

int match_pass(const DCsr &A, const int *arp, const int *aci, int annz, uint64_t seed, int scaled, int *mate,
               cudaStream_t s) {
    const int n = A.n;
    DBuf<double> aw(annz > 0 ? annz : 1);
    DBuf<int> prop(n), active(1);
    k_edge_weights<<<grid_for(n, 256), 256, 0, s>>>(n, A.rp.get(), A.ci.get(), A.v.get(), arp, aci, scaled,
                                                   aw.get());
    CU_LAUNCH("k_edge_weights"); count_launch();
    fill_int(mate, -1, n, s);
    int *hactive = nullptr;
    CU(cudaMallocHost(&hactive, sizeof(int)));
    const int max_rounds = 100000;
    int rounds = 0;
    for (;;) {
        if (rounds >= max_rounds) {
            cudaFreeHost(hactive);
            fail(8, "matching: handshake rounds exceeded the cap");
        }
        CU(cudaMemsetAsync(active.get(), 0, sizeof(int), s));
        k_propose<<<grid_for(n, 256), 256, 0, s>>>(n, arp, aci, aw.get(), seed, mate, prop.get(), active.get());
        CU_LAUNCH("k_propose"); count_launch();
        k_accept<<<grid_for(n, 256), 256, 0, s>>>(n, mate, prop.get());
        CU_LAUNCH("k_accept"); count_launch();
        CU(cudaMemcpyAsync(hactive, active.get(), sizeof(int), cudaMemcpyDeviceToHost, s));
        CU(cudaStreamSynchronize(s));
        ++rounds;
        if (*hactive == 0) break;
    }
    cudaFreeHost(hactive);
    k_unmark_dead<<<grid_for(n, 256), 256, 0, s>>>(n, mate);
    CU_LAUNCH("k_unmark_dead"); count_launch();
    return rounds;
}

// ------------------------------------------------------------------ aggregates
__global__ void k_leader(int n, const int *mate, int *flag) {
    for (int u = blockIdx.x * blockDim.x + threadIdx.x; u < n; u += gridDim.x * blockDim.x)
        flag[u] = (mate[u] < 0 || u < mate[u]) ? 1 : 0;
}
__global__ void k_agg_from_ids(int n, const int *mate, const int *id, int *agg) {
    for (int u = blockIdx.x * blockDim.x + threadIdx.x; u < n; u += gridDim.x * blockDim.x) {
        int m = mate[u];
        agg[u] = id[(m >= 0 && m < u) ? m : u];
    }
}

int aggregates_from_mate(int n, const int *mate, int *agg, cudaStream_t s) {
    DBuf<int> flag(n), id(n);
    k_leader<<<grid_for(n, 256), 256, 0, s>>>(n, mate, flag.get());
    CU_LAUNCH("k_leader"); count_launch();
    int nc = 0;
    exclusive_scan_int(flag.get(), id.get(), n, &nc, s);
    k_agg_from_ids<<<grid_for(n, 256), 256, 0, s>>>(n, mate, id.get(), agg);
    CU_LAUNCH("k_agg_from_ids"); count_launch();
    CU(cudaStreamSynchronize(s));
    return nc;
}

__global__ void k_int_to_key(const int *a, uint32_t *k, int n) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) k[i] = (uint32_t)a[i];
}

void members_of(int n, int nc, const int *agg, DBuf<int> &ptr, DBuf<int> &idx, cudaStream_t s) {
    DBuf<uint32_t> keys(n);
    idx.alloc(n);
    k_int_to_key<<<grid_for(n, 256), 256, 0, s>>>(agg, keys.get(), n);
    CU_LAUNCH("k_int_to_key"); count_launch();
    iota_int(idx.get(), n, s);
    radix_sort_pairs(keys.get(), idx.get(), n, bits_for((uint32_t)nc), s);
    segment_ptr(keys.get(), n, nc, ptr, s);
    CU(cudaStreamSynchronize(s));
}

// ------------------------------------------------------------------ Galerkin
// Coarse row I gathers the rows of its members (ascending), each in stored
// column order, maps columns through agg, sorts stably by coarse column and
// sums each run in that order: the entrywise formula of Section 2 with the
// summation order of a stable sort of A's entries by (agg[k], agg[l]).
// Rows gathering at most GAL_CAP entries are handled by one thread; longer
// rows (deep coarse levels) by one block that sorts (column, gather index)
// keys in shared memory.
constexpr int GAL_CAP = 128;
constexpr int GAL_BIG = 4096;

__device__ int gal_collect(int I, const int *rp, const int *ci, const double *v, const int *agg,
                           const int *mptr, const int *midx, int *kJ, double *kv) {
    int m = 0;
    for (int t = mptr[I]; t < mptr[I + 1]; ++t) {
        int row = midx[t];
        for (int e = rp[row]; e < rp[row + 1]; ++e) {
            int J = agg[ci[e]];
            double x = v[e];
            int p = m;                       // stable insertion: after equal keys
            while (p > 0 && kJ[p - 1] > J) { kJ[p] = kJ[p - 1]; kv[p] = kv[p - 1]; --p; }
            kJ[p] = J; kv[p] = x;
            ++m;
        }
    }
    return m;
}

__device__ __forceinline__ int gal_len(int I, const int *rp, const int *mptr, const int *midx) {
    int m = 0;
    for (int t = mptr[I]; t < mptr[I + 1]; ++t) m += rp[midx[t] + 1] - rp[midx[t]];
    return m;
}

__global__ void k_gal_count(int nc, const int *rp, const int *ci, const double *v, const int *agg,
                            const int *mptr, const int *midx, int *cnt, int *big, int *nbig) {
    int kJ[GAL_CAP];
    double kv[GAL_CAP];
    for (int I = blockIdx.x * blockDim.x + threadIdx.x; I < nc; I += gridDim.x * blockDim.x) {
        if (gal_len(I, rp, mptr, midx) > GAL_CAP) {
            big[atomicAdd(nbig, 1)] = I;
            cnt[I] = 0;
            continue;
        }
        int m = gal_collect(I, rp, ci, v, agg, mptr, midx, kJ, kv);
        int u = 0;
        for (int t = 0; t < m; ++t) if (t == 0 || kJ[t] != kJ[t - 1]) ++u;
        cnt[I] = u;
    }
}

__global__ void k_gal_fill(int nc, const int *rp, const int *ci, const double *v, const int *agg,
                           const int *mptr, const int *midx, const int *crp, int *cci, double *cv) {
    int kJ[GAL_CAP];
    double kv[GAL_CAP];
    for (int I = blockIdx.x * blockDim.x + threadIdx.x; I < nc; I += gridDim.x * blockDim.x) {
        if (gal_len(I, rp, mptr, midx) > GAL_CAP) continue;
        int m = gal_collect(I, rp, ci, v, agg, mptr, midx, kJ, kv);
        int out = crp[I] - 1;
        double acc = 0.0;
        for (int t = 0; t < m; ++t) {
            if (t == 0 || kJ[t] != kJ[t - 1]) {
                if (out >= crp[I]) cv[out] = acc;
                ++out;
                cci[out] = kJ[t];
                acc = kv[t];
            } else {
                acc = __dadd_rn(acc, kv[t]);
            }
        }
        if (m > 0) cv[out] = acc;
    }
}

// One block per long row: keys (J << 32 | gather index) bitonic-sorted in
// shared memory; values stay in gather order.  mode 0 counts, mode 1 fills.
__global__ void __launch_bounds__(256) k_gal_big(const int *big, const int *rp, const int *ci, const double *v,
                                                 const int *agg, const int *mptr, const int *midx, int *cnt,
                                                 const int *crp, int *cci, double *cv, int mode, int *overflow) {
    extern __shared__ unsigned char smem[];
    uint64_t *key = reinterpret_cast<uint64_t *>(smem);
    double *val = reinterpret_cast<double *>(smem + sizeof(uint64_t) * GAL_BIG);
    __shared__ int m_s, P_s;
    const int I = big[blockIdx.x];
    if (threadIdx.x == 0) {
        int m = gal_len(I, rp, mptr, midx);
        m_s = m;
        int P = 1;
        while (P < m) P <<= 1;
        P_s = P;
        if (m > GAL_BIG) atomicExch(overflow, 1);
    }
    __syncthreads();
    const int m = m_s, P = P_s;
    if (m > GAL_BIG) return;
    // gather: the k-th entry in (member ascending, column ascending) order
    if (threadIdx.x == 0) {
        int k = 0;
        for (int t = mptr[I]; t < mptr[I + 1]; ++t) {
            int row = midx[t];
            for (int e = rp[row]; e < rp[row + 1]; ++e, ++k) {
                key[k] = ((uint64_t)(uint32_t)agg[ci[e]] << 32) | (uint32_t)k;
                val[k] = v[e];
            }
        }
    }
    __syncthreads();
    for (int k = m + threadIdx.x; k < P; k += blockDim.x) key[k] = ~0ull;
    __syncthreads();
    for (int size = 2; size <= P; size <<= 1) {
        for (int stride = size >> 1; stride > 0; stride >>= 1) {
            for (int t = threadIdx.x; t < P; t += blockDim.x) {
                int partner = t ^ stride;
                if (partner > t) {
                    bool up = (t & size) == 0;
                    uint64_t a = key[t], b = key[partner];
                    if ((a > b) == up) { key[t] = b; key[partner] = a; }
                }
            }
            __syncthreads();
        }
    }
    if (threadIdx.x == 0) {
        int out = mode ? crp[I] - 1 : -1, u = 0;
        double acc = 0.0;
        for (int t = 0; t < m; ++t) {
            const int J = (int)(key[t] >> 32);
            const double x = val[(uint32_t)key[t]];
            if (t == 0 || J != (int)(key[t - 1] >> 32)) {
                ++u;
                if (mode) {
                    if (out >= crp[I]) cv[out] = acc;
                    ++out;
                    cci[out] = J;
                }
                acc = x;
            } else {
                acc = __dadd_rn(acc, x);
            }
        }
        if (mode) { if (m > 0) cv[out] = acc; }
        else cnt[I] = u;
    }
}

void galerkin(const DCsr &A, int nc, const int *agg, const int *mptr, const int *midx, DCsr &C,
              cudaStream_t s) {
    DBuf<int> cnt(nc + 1), big(nc > 0 ? nc : 1), flags(2);
    CU(cudaMemsetAsync(flags.get(), 0, 2 * sizeof(int), s));
    fill_int(cnt.get(), 0, nc + 1, s);
    k_gal_count<<<grid_for(nc, 128), 128, 0, s>>>(nc, A.rp.get(), A.ci.get(), A.v.get(), agg, mptr, midx,
                                                  cnt.get(), big.get(), flags.get());
    CU_LAUNCH("k_gal_count"); count_launch();
    const int nbig = read_int(flags.get(), s);
    const size_t smem = (sizeof(uint64_t) + sizeof(double)) * GAL_BIG;
    if (nbig > 0) {
        CU(cudaFuncSetAttribute(k_gal_big, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        k_gal_big<<<nbig, 256, smem, s>>>(big.get(), A.rp.get(), A.ci.get(), A.v.get(), agg, mptr, midx,
                                          cnt.get(), nullptr, nullptr, nullptr, 0, flags.get() + 1);
        CU_LAUNCH("k_gal_big"); count_launch();
        if (read_int(flags.get() + 1, s)) fail(8, "Galerkin: a coarse row gathers more than 4096 fine entries");
    }
    C.n = nc;
    C.rp.alloc(nc + 1);
    exclusive_scan_int(cnt.get(), C.rp.get(), nc + 1, &C.nnz, s);
    C.ci.alloc(C.nnz > 0 ? C.nnz : 1);
    C.v.alloc(C.nnz > 0 ? C.nnz : 1);
    k_gal_fill<<<grid_for(nc, 128), 128, 0, s>>>(nc, A.rp.get(), A.ci.get(), A.v.get(), agg, mptr, midx,
                                                 C.rp.get(), C.ci.get(), C.v.get());
    CU_LAUNCH("k_gal_fill"); count_launch();
    if (nbig > 0) {
        k_gal_big<<<nbig, 256, smem, s>>>(big.get(), A.rp.get(), A.ci.get(), A.v.get(), agg, mptr, midx,
                                          cnt.get(), C.rp.get(), C.ci.get(), C.v.get(), 1, flags.get() + 1);
        CU_LAUNCH("k_gal_big"); count_launch();
    }
    CU(cudaStreamSynchronize(s));
}

// ------------------------------------------------------------------ colouring
// Jones-Plassmann rounds: a vertex whose higher-priority neighbours are all
// coloured takes the smallest colour none of them uses.  This reproduces the
// sequential greedy colouring in decreasing priority order.
constexpr int MAX_COLORS = 256;
__device__ __forceinline__ bool prio_higher(int a, int b, int mode, uint64_t seed) {
    if (mode == 1) return a < b;                        // first fit: lower index first
    const uint64_t salt = 0x9e3779b97f4a7c15ull;
    uint64_t ha = mix64((uint64_t)(uint32_t)a ^ (seed + salt));
    uint64_t hb = mix64((uint64_t)(uint32_t)b ^ (seed + salt));
    if (ha != hb) return ha > hb;
    return a > b;
}

__global__ void k_jp_round(int n, const int *arp, const int *aci, int mode, uint64_t seed, int *color,
                           int *remaining, int *overflow) {
    int rem = 0;
    for (int u = blockIdx.x * blockDim.x + threadIdx.x; u < n; u += gridDim.x * blockDim.x) {
        if (ld_volatile(color + u) >= 0) continue;
        uint64_t mask[MAX_COLORS / 64] = {0, 0, 0, 0};
        bool ready = true;
        for (int e = arp[u]; e < arp[u + 1]; ++e) {
            int v = aci[e];
            if (!prio_higher(v, u, mode, seed)) continue;
            int cv = ld_volatile(color + v);
            if (cv < 0) { ready = false; break; }
            if (cv < MAX_COLORS) mask[cv >> 6] |= 1ull << (cv & 63);
        }
        if (!ready) { ++rem; continue; }
        int c = 0;
        while (c < MAX_COLORS && (mask[c >> 6] >> (c & 63)) & 1ull) ++c;
        if (c >= MAX_COLORS) { atomicExch(overflow, 1); c = MAX_COLORS - 1; }
        *(volatile int *)(color + u) = c;
    }
    if (rem) atomicAdd(remaining, rem);
}

__global__ void k_max_int(const int *a, int n, int *out) {
    int m = -1;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) m = max(m, a[i]);
    for (int off = 16; off; off >>= 1) m = max(m, __shfl_xor_sync(0xffffffffu, m, off));
    if ((threadIdx.x & 31) == 0) atomicMax(out, m);
}

static int max_of(const int *a, int n, cudaStream_t s) {
    DBuf<int> out(1);
    fill_int(out.get(), -1, 1, s);
    k_max_int<<<grid_for(n, 256), 256, 0, s>>>(a, n, out.get());
    CU_LAUNCH("k_max_int"); count_launch();
    return read_int(out.get(), s);
}

int color_jp(int n, const int *arp, const int *aci, int mode, uint64_t seed, int *color, cudaStream_t s) {
    DBuf<int> rem(1), overflow(1);
    fill_int(color, -1, n, s);
    CU(cudaMemsetAsync(overflow.get(), 0, sizeof(int), s));
    int *h = nullptr;
    CU(cudaMallocHost(&h, sizeof(int)));
    const int max_rounds = 1000000;
    int rounds = 0;
    for (;;) {
        if (rounds >= max_rounds) { cudaFreeHost(h); fail(8, "colouring: rounds exceeded the cap"); }
        CU(cudaMemsetAsync(rem.get(), 0, sizeof(int), s));
        k_jp_round<<<grid_for(n, 256), 256, 0, s>>>(n, arp, aci, mode, seed, color, rem.get(), overflow.get());
        CU_LAUNCH("k_jp_round"); count_launch();
        CU(cudaMemcpyAsync(h, rem.get(), sizeof(int), cudaMemcpyDeviceToHost, s));
        CU(cudaStreamSynchronize(s));
        ++rounds;
        if (*h == 0) break;
    }
    cudaFreeHost(h);
    if (read_int(overflow.get(), s)) fail(8, "colouring: more than 256 colours");
    return max_of(color, n, s) + 1;
}

// ------------------------------------------------------------------ elimination order
__global__ void k_invert_perm(const int *perm, int *pos, int n) {
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < n; k += gridDim.x * blockDim.x) pos[perm[k]] = k;
}

void elimination_positions(int n, const int *label, int nlabels, int *pos, cudaStream_t s) {
    DBuf<uint32_t> keys(n);
    DBuf<int> perm(n);
    k_int_to_key<<<grid_for(n, 256), 256, 0, s>>>(label, keys.get(), n);
    CU_LAUNCH("k_int_to_key"); count_launch();
    iota_int(perm.get(), n, s);
    if (nlabels > 1) radix_sort_pairs(keys.get(), perm.get(), n, bits_for((uint32_t)nlabels), s);
    k_invert_perm<<<grid_for(n, 256), 256, 0, s>>>(perm.get(), pos, n);
    CU_LAUNCH("k_invert_perm"); count_launch();
    CU(cudaStreamSynchronize(s));
}

// ------------------------------------------------------------------ sweep schedules
// Longest-path depth of each row in the dependency graph of the forward
// (pos[j] < pos[i]) or backward (pos[j] > pos[i]) solve, by frontier rounds
// (Kahn's algorithm): a row enters round r when the last of its
// dependencies was in round r-1, so its round is 1 + the largest depth of
// its dependencies.  Work O(nnz) over all rounds.
__global__ void k_dep_count(int n, const int *rp, const int *ci, const int *pos, int fwd, int *indeg) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const int pi = pos[i];
        int m = 0;
        for (int e = rp[i]; e < rp[i + 1]; ++e) {
            const int pj = pos[ci[e]];
            if (fwd ? (pj < pi) : (pj > pi)) ++m;
        }
        indeg[i] = m;
    }
}

__global__ void k_frontier_init(int n, const int *indeg, int *front, int *count) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
        if (indeg[i] == 0) front[atomicAdd(count, 1)] = i;
}

// rows of the frontier get depth r; their dependents (column j of the
// pattern = rows i with a_ij stored) lose one dependency
__global__ void k_frontier_step(const int *front, int cnt, int r, const int *trp, const int *tci, const int *pos,
                                int fwd, int *indeg, int *lev, int *next, int *ncount) {
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < cnt; t += gridDim.x * blockDim.x) {
        const int j = front[t];
        lev[j] = r;
        const int pj = pos[j];
        for (int e = trp[j]; e < trp[j + 1]; ++e) {
            const int i = tci[e];
            const int pi = pos[i];
            if (!(fwd ? (pj < pi) : (pj > pi))) continue;
            if (atomicSub(indeg + i, 1) == 1) next[atomicAdd(ncount, 1)] = i;
        }
    }
}

static int schedule_levels(const DCsr &A, const int *pos, int fwd, int *lev, cudaStream_t s) {
    const int n = A.n;
    DBuf<int> trp, tci, tsrc, indeg(n), fa(n), fb(n), cnt(2);
    csr_transpose(n, A.nnz, A.rp.get(), A.ci.get(), trp, tci, tsrc, s);
    k_dep_count<<<grid_for(n, 256), 256, 0, s>>>(n, A.rp.get(), A.ci.get(), pos, fwd, indeg.get());
    CU_LAUNCH("k_dep_count"); count_launch();
    CU(cudaMemsetAsync(cnt.get(), 0, 2 * sizeof(int), s));
    k_frontier_init<<<grid_for(n, 256), 256, 0, s>>>(n, indeg.get(), fa.get(), cnt.get());
    CU_LAUNCH("k_frontier_init"); count_launch();
    int *h = nullptr;
    CU(cudaMallocHost(&h, sizeof(int)));
    CU(cudaMemcpyAsync(h, cnt.get(), sizeof(int), cudaMemcpyDeviceToHost, s));
    CU(cudaStreamSynchronize(s));
    int c = *h, r = 0, done = 0;
    int *cur = fa.get(), *nxt = fb.get();
    while (c > 0) {
        if (r > n) { cudaFreeHost(h); fail(8, "sweep schedule did not settle"); }
        CU(cudaMemsetAsync(cnt.get() + 1, 0, sizeof(int), s));
        k_frontier_step<<<grid_for(c, 256), 256, 0, s>>>(cur, c, r, trp.get(), tci.get(), pos, fwd, indeg.get(), lev,
                                                         nxt, cnt.get() + 1);
        CU_LAUNCH("k_frontier_step"); count_launch();
        CU(cudaMemcpyAsync(h, cnt.get() + 1, sizeof(int), cudaMemcpyDeviceToHost, s));
        CU(cudaStreamSynchronize(s));
        done += c;
        c = *h;
        std::swap(cur, nxt);
        ++r;
    }
    cudaFreeHost(h);
    if (done != n) fail(8, "sweep schedule: dependency cycle");
    return r;
}

__global__ void k_sweep_count(int n, const int *rows, const int *rp, const int *ci, const int *pos, int fwd,
                              int *cnt) {
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < n; k += gridDim.x * blockDim.x) {
        int i = rows[k], pi = pos[i], m = 0;
        for (int e = rp[i]; e < rp[i + 1]; ++e) {
            int pj = pos[ci[e]];
            if (fwd ? (pj < pi) : (pj > pi)) ++m;
        }
        cnt[k] = m;
    }
}

__global__ void k_sweep_fill(int n, const int *rows, const int *rp, const int *ci, const double *lu,
                             const int *pos, int fwd, const int *srp, int *sci, double *sv, double *diag) {
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < n; k += gridDim.x * blockDim.x) {
        int i = rows[k], pi = pos[i], m = srp[k];
        for (int e = rp[i]; e < rp[i + 1]; ++e) {
            int j = ci[e];
            int pj = pos[j];
            if (fwd ? (pj < pi) : (pj > pi)) { sci[m] = j; sv[m] = lu[e]; ++m; }
            else if (j == i && diag) diag[k] = lu[e];
        }
    }
}

static void build_sweep(const DCsr &A, const int *pos, const double *lu, int fwd, int want_diag, const int *lev,
                        int nlev, Sweep &S, cudaStream_t s) {
    const int n = A.n;
    DBuf<uint32_t> keys(n);
    S.rows.alloc(n);
    k_int_to_key<<<grid_for(n, 256), 256, 0, s>>>(lev, keys.get(), n);
    CU_LAUNCH("k_int_to_key"); count_launch();
    iota_int(S.rows.get(), n, s);
    if (nlev > 1) radix_sort_pairs(keys.get(), S.rows.get(), n, bits_for((uint32_t)nlev), s);
    segment_ptr(keys.get(), n, nlev, S.dlev, s);
    S.nlev = nlev;
    S.lev_ptr.resize(nlev + 1);
    CU(cudaMemcpyAsync(S.lev_ptr.data(), S.dlev.get(), sizeof(int) * (nlev + 1), cudaMemcpyDeviceToHost, s));
    DBuf<int> cnt(n + 1);
    fill_int(cnt.get(), 0, n + 1, s);
    k_sweep_count<<<grid_for(n, 256), 256, 0, s>>>(n, S.rows.get(), A.rp.get(), A.ci.get(), pos, fwd, cnt.get());
    CU_LAUNCH("k_sweep_count"); count_launch();
    S.rp.alloc(n + 1);
    int nnzf = 0;
    exclusive_scan_int(cnt.get(), S.rp.get(), n + 1, &nnzf, s);
    S.ci.alloc(nnzf > 0 ? nnzf : 1);
    S.v64.alloc(nnzf > 0 ? nnzf : 1);
    if (want_diag) S.d64.alloc(n);
    k_sweep_fill<<<grid_for(n, 256), 256, 0, s>>>(n, S.rows.get(), A.rp.get(), A.ci.get(), lu, pos, fwd,
                                                  S.rp.get(), S.ci.get(), S.v64.get(), want_diag ? S.d64.get() : nullptr);
    CU_LAUNCH("k_sweep_fill"); count_launch();
    CU(cudaStreamSynchronize(s));
    S.maxlev = 0;
    for (int l = 0; l < nlev; ++l) S.maxlev = std::max(S.maxlev, S.lev_ptr[l + 1] - S.lev_ptr[l]);
}

// ------------------------------------------------------------------ ILU(0)
// IKJ ILU(0) on the pattern of A in the elimination order pos (Algorithm 1,
// smoother setup): for each stored k of row i with pos(k) < pos(i), in
// increasing pos(k): a_ik /= a_kk, then a_ij -= a_ik a_kj for every stored
// (k, j) with pos(j) > pos(k) whose (i, j) is stored.  Rows of one schedule
// level only read rows of earlier levels, so a level runs in parallel.
constexpr int ILU_CAP = 256;
constexpr int ILU_WCAP = 256, ILU_WARPS = 4;   // rows up to ILU_WCAP entries: warp kernel

__global__ void k_ilu_rows(const int *rows, int count, const int *rp, const int *ci, const int *pos,
                           const int *dpos, double *lu, int *breakdown, int *overflow) {
    int lp[ILU_CAP], le[ILU_CAP];
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < count; t += gridDim.x * blockDim.x) {
        const int i = rows[t], pi = pos[i], rb = rp[i], re = rp[i + 1];
        if (re - rb <= ILU_WCAP) continue;           // handled by the warp kernel
        int nl = 0;
        bool over = false;
        for (int e = rb; e < re; ++e) {
            int p = pos[ci[e]];
            if (p < pi) {
                if (nl >= ILU_CAP) { over = true; break; }
                int q = nl++;
                while (q > 0 && lp[q - 1] > p) { lp[q] = lp[q - 1]; le[q] = le[q - 1]; --q; }
                lp[q] = p; le[q] = e;
            }
        }
        if (over) { atomicExch(overflow, 1); continue; }
        for (int a = 0; a < nl; ++a) {
            const int eik = le[a], k = ci[eik];
            const int pk = lp[a];
            const double lik = __ddiv_rn(lu[eik], lu[dpos[k]]);
            lu[eik] = lik;
            int p = rb;                              // walk row i and row k by column
            for (int ekj = rp[k]; ekj < rp[k + 1]; ++ekj) {
                const int j = ci[ekj];
                if (pos[j] <= pk) continue;
                while (p < re && ci[p] < j) ++p;
                if (p < re && ci[p] == j) lu[p] = __dsub_rn(lu[p], __dmul_rn(lik, lu[ekj]));
            }
        }
        double piv = lu[dpos[i]];
        if (piv == 0.0 || !isfinite(piv)) atomicExch(breakdown, 1);
    }
}

// Warp-per-row variant for rows of at most ILU_WCAP entries: row i is staged
// in shared memory, its L entries are ranked by pos in parallel, then for each
// L entry k (in increasing pos) lane 0 divides and the lanes apply row k's U
// part to the staged row (distinct columns per lane, so no two lanes update
// the same entry).  Same operations in the same order per entry as the
// thread-per-row kernel, hence bit-identical factors.

__global__ void __launch_bounds__(32 * ILU_WARPS) k_ilu_rows_warp(const int *rows, int count, const int *rp,
                                                                  const int *ci, const int *pos, const int *dpos,
                                                                  double *lu, int *breakdown) {
    __shared__ int s_col[ILU_WARPS][ILU_WCAP];
    __shared__ int s_pos[ILU_WARPS][ILU_WCAP];
    __shared__ double s_val[ILU_WARPS][ILU_WCAP];
    __shared__ int s_ord[ILU_WARPS][ILU_WCAP];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int gw = blockIdx.x * ILU_WARPS + w, nw = gridDim.x * ILU_WARPS;
    for (int t = gw; t < count; t += nw) {
        const int i = rows[t], rb = rp[i], len = rp[i + 1] - rb, pi = pos[i];
        if (len > ILU_WCAP) continue;                // long rows: thread kernel
        for (int q = lane; q < len; q += 32) {
            const int c = ci[rb + q];
            s_col[w][q] = c;
            s_pos[w][q] = pos[c];
            s_val[w][q] = lu[rb + q];
        }
        __syncwarp();
        int nl = 0;
        for (int q = lane; q < len; q += 32) {       // rank of each L entry by pos
            const int pq = s_pos[w][q];
            if (pq < pi) {
                int r = 0;
                for (int u = 0; u < len; ++u) r += (s_pos[w][u] < pq) ? 1 : 0;
                s_ord[w][r] = q;
            }
        }
        for (int q = 0; q < len; ++q) nl += (s_pos[w][q] < pi) ? 1 : 0;
        __syncwarp();
        for (int a = 0; a < nl; ++a) {
            const int qk = s_ord[w][a];
            const int k = s_col[w][qk], pk = s_pos[w][qk];
            double lik = 0.0;
            if (lane == 0) {
                lik = __ddiv_rn(s_val[w][qk], lu[dpos[k]]);
                s_val[w][qk] = lik;
            }
            lik = __shfl_sync(0xffffffffu, lik, 0);
            __syncwarp();
            for (int ekj = rp[k] + lane; ekj < rp[k + 1]; ekj += 32) {
                const int j = ci[ekj];
                if (pos[j] <= pk) continue;
                int lo = 0, hi = len - 1;                // columns of row i ascend
                while (lo <= hi) {
                    const int mid = (lo + hi) >> 1;
                    const int cm = s_col[w][mid];
                    if (cm == j) {
                        s_val[w][mid] = __dsub_rn(s_val[w][mid], __dmul_rn(lik, lu[ekj]));
                        break;
                    }
                    if (cm < j) lo = mid + 1; else hi = mid - 1;
                }
            }
            __syncwarp();
        }
        for (int q = lane; q < len; q += 32) lu[rb + q] = s_val[w][q];
        if (lane == 0) {
            const double piv = s_val[w][dpos[i] - rb];
            if (piv == 0.0 || !isfinite(piv)) atomicExch(breakdown, 1);
        }
        __syncwarp();
    }
}

__global__ void k_diag_pos(int n, const int *rp, const int *ci, int *dpos) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
        dpos[i] = find_col(ci, rp[i], rp[i + 1], i);
}

void ilu0_factor(const DCsr &A, const int *pos, DBuf<double> &lu, Sweep &fwd, Sweep &bwd, cudaStream_t s) {
    const int n = A.n;
    DBuf<int> levf(n), levb(n), dpos(n), flags(2);
    const int nf = schedule_levels(A, pos, 1, levf.get(), s);
    const int nb = schedule_levels(A, pos, 0, levb.get(), s);
    lu.alloc(A.nnz > 0 ? A.nnz : 1);
    CU(cudaMemcpyAsync(lu.get(), A.v.get(), sizeof(double) * A.nnz, cudaMemcpyDeviceToDevice, s));
    k_diag_pos<<<grid_for(n, 256), 256, 0, s>>>(n, A.rp.get(), A.ci.get(), dpos.get());
    CU_LAUNCH("k_diag_pos"); count_launch();
    CU(cudaMemsetAsync(flags.get(), 0, 2 * sizeof(int), s));
    // forward schedule rows (needed to run the factorisation level by level)
    Sweep tmp;
    {
        DBuf<uint32_t> keys(n);
        tmp.rows.alloc(n);
        k_int_to_key<<<grid_for(n, 256), 256, 0, s>>>(levf.get(), keys.get(), n);
        CU_LAUNCH("k_int_to_key"); count_launch();
        iota_int(tmp.rows.get(), n, s);
        if (nf > 1) radix_sort_pairs(keys.get(), tmp.rows.get(), n, bits_for((uint32_t)nf), s);
        DBuf<int> lp;
        segment_ptr(keys.get(), n, nf, lp, s);
        tmp.lev_ptr.resize(nf + 1);
        CU(cudaMemcpyAsync(tmp.lev_ptr.data(), lp.get(), sizeof(int) * (nf + 1), cudaMemcpyDeviceToHost, s));
        CU(cudaStreamSynchronize(s));
    }
    bool long_rows = false;
    {
        std::vector<int> hrp(n + 1);
        CU(cudaMemcpy(hrp.data(), A.rp.get(), sizeof(int) * (n + 1), cudaMemcpyDeviceToHost));
        for (int i = 0; i < n && !long_rows; ++i) long_rows = hrp[i + 1] - hrp[i] > ILU_WCAP;
    }
    for (int l = 0; l < nf; ++l) {
        const int b = tmp.lev_ptr[l], cnt = tmp.lev_ptr[l + 1] - b;
        if (cnt <= 0) continue;
        k_ilu_rows_warp<<<grid_for((size_t)cnt * 32, 32 * ILU_WARPS), 32 * ILU_WARPS, 0, s>>>(
            tmp.rows.get() + b, cnt, A.rp.get(), A.ci.get(), pos, dpos.get(), lu.get(), flags.get());
        CU_LAUNCH("k_ilu_rows_warp"); count_launch();
        if (long_rows) {
            k_ilu_rows<<<grid_for(cnt, 128), 128, 0, s>>>(tmp.rows.get() + b, cnt, A.rp.get(), A.ci.get(), pos,
                                                          dpos.get(), lu.get(), flags.get(), flags.get() + 1);
            CU_LAUNCH("k_ilu_rows"); count_launch();
        }
    }
    int hf[2];
    CU(cudaMemcpyAsync(hf, flags.get(), 2 * sizeof(int), cudaMemcpyDeviceToHost, s));
    CU(cudaStreamSynchronize(s));
    if (hf[1]) fail(8, "ILU(0): a row has more than 256 entries before the diagonal");
    if (hf[0]) fail(5, "ILU(0): zero or non-finite pivot");
    build_sweep(A, pos, lu.get(), 1, 0, levf.get(), nf, fwd, s);
    build_sweep(A, pos, lu.get(), 0, 1, levb.get(), nb, bwd, s);
}

void factor_sweeps(const DCsr &F, const int *pos, const double *lu, Sweep &fwd, Sweep &bwd, cudaStream_t s) {
    const int n = F.n;
    DBuf<int> levf(n), levb(n);
    const int nf = schedule_levels(F, pos, 1, levf.get(), s);
    const int nb = schedule_levels(F, pos, 0, levb.get(), s);
    build_sweep(F, pos, lu, 1, 0, levf.get(), nf, fwd, s);
    build_sweep(F, pos, lu, 0, 1, levb.get(), nb, bwd, s);
}

__global__ void k_gather_vals(const double *src, const int *idx, double *dst, int n) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) dst[i] = src[idx[i]];
}

// Sweeps of (L U)^T = U^T L^T on the transposed layout: row j of the
// transpose holds u_ij for pos(i) < pos(j) (forward solve U^T w = r with
// division by u_jj) and l_ij for pos(i) > pos(j) (backward solve L^T t = w,
// unit diagonal).
void build_transposed_sweeps(const DCsr &A, const int *pos, const double *lu, Sweep &fwdT, Sweep &bwdT,
                             cudaStream_t s) {
    DCsr T;
    DBuf<int> tsrc;
    csr_transpose(A.n, A.nnz, A.rp.get(), A.ci.get(), T.rp, T.ci, tsrc, s);
    T.n = A.n;
    T.nnz = A.nnz;
    T.v.alloc(A.nnz > 0 ? A.nnz : 1);
    if (A.nnz) {
        k_gather_vals<<<grid_for(A.nnz, 256), 256, 0, s>>>(lu, tsrc.get(), T.v.get(), A.nnz);
        CU_LAUNCH("k_gather_vals"); count_launch();
    }
    DBuf<int> levf(A.n), levb(A.n);
    const int nf = schedule_levels(T, pos, 1, levf.get(), s);
    const int nb = schedule_levels(T, pos, 0, levb.get(), s);
    build_sweep(T, pos, T.v.get(), 1, 1, levf.get(), nf, fwdT, s);
    build_sweep(T, pos, T.v.get(), 0, 0, levb.get(), nb, bwdT, s);
}

// ------------------------------------------------------------------ dense inverse
// Gauss-Jordan elimination with partial pivoting on [A | I] (FP64).  The
// pivot of column k is the first row of largest magnitude at or below k.
__global__ void k_dense_from_csr(int n, const int *rp, const int *ci, const double *v, double *M) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        double *row = M + (size_t)i * 2 * n;
        for (int j = 0; j < 2 * n; ++j) row[j] = (j == n + i) ? 1.0 : 0.0;
        for (int e = rp[i]; e < rp[i + 1]; ++e) row[ci[e]] = v[e];
    }
}

// Rows stay where they are: perm[l] is the physical row at logical position
// l (the position the row would have after the swaps of the sequential
// algorithm) and pos[r] its inverse.  Step k: the pivot is the first logical
// row l >= k of largest |m_{perm[l],k}|; perm and pos swap positions k and p;
// the pivot row R = perm[k] is divided by its diagonal entry; every other
// row r with f = m_rk != 0 gets fma(-f, m_Rj, m_rj).  Each value goes through
// the same operations as in the sequential algorithm, so the inverse is the
// same bit for bit; logical row l of the inverse is physical row perm[l].
struct GjPart {
    double v;      // largest |m_ik| of a row group (-1: none)
    int l;         // its logical position (first on ties)
    int r;         // its physical row
};

// x != 0 (either sign of zero counts as zero) as an integer test: FP64
// compares would use the FP64 pipe, the bound of the elimination on GB300.
__device__ __forceinline__ bool gj_nonzero(double x) {
    return (__double_as_longlong(x) & 0x7fffffffffffffffLL) != 0;
}

__device__ __forceinline__ bool gj_better(double v, int l, double bv, int bl) {
    return v > bv || (v == bv && l < bl);
}

// Pivot of column k and the division of the pivot row, over many blocks.
// Every block reduces the row-group candidates of the previous elimination
// (nparts > 0) or scans the column (k == 0, nparts == 0) to the same pivot;
// no block reads perm before block 0 has swapped it (blocks only read perm[k]
// when the pivot is singular, and then the swap leaves it unchanged); block 0 swaps
// logical positions k and p and publishes R; each block divides its slice of
// the pivot row's columns j > k by d = m_Rk (column k itself is never read
// again, so it keeps the raw d every block reads).
__global__ void __launch_bounds__(256) k_gj_pivot(int n, int k, double *M, int *perm, int *pos,
                                                  const GjPart *parts, int nparts, int *R_out, int *breakdown) {
    __shared__ double bv[8];
    __shared__ int bl[8], br[8];
    __shared__ int s_R, s_p;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const size_t w = 2 * (size_t)n;
    double best = -1.0;
    int bidx = n, brow = -1;
    if (nparts > 0) {
        for (int g = tid; g < nparts; g += blockDim.x)
            if (gj_better(parts[g].v, parts[g].l, best, bidx)) { best = parts[g].v; bidx = parts[g].l; brow = parts[g].r; }
    } else {                     // k == 0: perm is still the identity (block 0 swaps it below)
        for (int l = k + tid; l < n; l += blockDim.x) {
            const double a = fabs(M[(size_t)l * w + k]);
            if (gj_better(a, l, best, bidx)) { best = a; bidx = l; brow = l; }
        }
    }
    for (int off = 16; off; off >>= 1) {
        const double ob = __shfl_down_sync(0xffffffffu, best, off);
        const int oi = __shfl_down_sync(0xffffffffu, bidx, off);
        const int orr = __shfl_down_sync(0xffffffffu, brow, off);
        if (gj_better(ob, oi, best, bidx)) { best = ob; bidx = oi; brow = orr; }
    }
    if (lane == 0) { bv[warp] = best; bl[warp] = bidx; br[warp] = brow; }
    __syncthreads();
    if (tid == 0) {
        double b = -1.0;
        int p = n, R = -1;
        for (int q = 0; q < (int)(blockDim.x + 31) / 32; ++q)
            if (gj_better(bv[q], bl[q], b, p)) { b = bv[q]; p = bl[q]; R = br[q]; }
        if (!(b > 0.0) || !isfinite(b)) {              // singular: keep position k (the result is flagged)
            if (blockIdx.x == 0) atomicExch(breakdown, 1);
            p = k;
            R = -1;
        }
        s_p = p;
        s_R = R;
    }
    __syncthreads();
    int R = s_R;
    const int p = s_p;
    if (R < 0) R = perm[k];                           // breakdown: no swap (perm[k] is only written below)
    if (blockIdx.x == 0 && tid == 0) {
        const int rk = perm[k];
        perm[k] = R; perm[p] = rk;
        pos[R] = k; pos[rk] = p;
        *R_out = R;
    }
    double *row = M + (size_t)R * w;
    const double d = row[k];
    constexpr int U = 4;
    const size_t stride = (size_t)gridDim.x * blockDim.x;
    for (size_t j0 = (size_t)k + 1 + blockIdx.x * (size_t)blockDim.x + tid; j0 < w; j0 += U * stride) {
        double v[U];
#pragma unroll
        for (int q = 0; q < U; ++q) {
            const size_t j = j0 + q * stride;
            if (j < w) v[q] = row[j];
        }
#pragma unroll
        for (int q = 0; q < U; ++q) {
            const size_t j = j0 + q * stride;
            if (j < w) row[j] = __ddiv_rn(v[q], d);
        }
    }
}

// Elimination of column k: physical rows over the row groups (blockIdx.y),
// columns j > k over x; a thread keeps m_Rj in a register across its rows.
// The update m_ij - f m_Rj is one fused multiply-add.  Only columns nonzero
// in the pivot row are updated: m_ij - f (+-0) equals m_ij except possibly
// in the sign of a zero, which no later product sees.  Thread (0, 0) of each
// row group also records the group's pivot candidate for column k + 1
// (largest updated |m_{r,k+1}| over rows with pos[r] > k).
__global__ void __launch_bounds__(256) k_gj_elim(int n, int k, double *M, const int *pos, const int *R_in,
                                                 GjPart *parts) {
    const size_t w = 2 * (size_t)n;
    const int R = *R_in;
    const double *rk = M + (size_t)R * w;
    const int nrows_g = (n + gridDim.y - 1) / gridDim.y;
    const int r0 = blockIdx.y * nrows_g, r1 = min(n, r0 + nrows_g);
    const bool cand = k + 1 < n && blockIdx.x == 0 && threadIdx.x == 0;
    double best = -1.0;
    int bl = n, br = -1;
    constexpr int U = 8;        // rows whose loads are in flight together
    for (size_t j = (size_t)k + 1 + blockIdx.x * (size_t)blockDim.x + threadIdx.x; j < w;
         j += (size_t)gridDim.x * blockDim.x) {
        const double r = rk[j];
        const bool track = cand && j == (size_t)k + 1;
        const bool rnz = gj_nonzero(r);
        if (!rnz && !track) continue;
        for (int i0 = r0; i0 < r1; i0 += U) {
            double fv[U], vv[U];
#pragma unroll
            for (int q = 0; q < U; ++q) {
                const int i = i0 + q;
                if (i < r1) {
                    fv[q] = M[(size_t)i * w + k];
                    vv[q] = M[(size_t)i * w + j];
                }
            }
#pragma unroll
            for (int q = 0; q < U; ++q) {
                const int i = i0 + q;
                if (i >= r1 || i == R) continue;
                if (rnz && gj_nonzero(fv[q])) {
                    vv[q] = __fma_rn(-fv[q], r, vv[q]);
                    M[(size_t)i * w + j] = vv[q];
                }
                if (track) {
                    const int l = pos[i];
                    const double a = fabs(vv[q]);
                    if (l > k && gj_better(a, l, best, bl)) { best = a; bl = l; br = i; }
                }
            }
        }
    }
    if (cand) parts[blockIdx.y] = GjPart{best, bl, br};
}

__global__ void k_extract_inverse(int n, const double *M, const int *perm, double *inv) {
    const size_t total = (size_t)n * n;
    for (size_t t = blockIdx.x * (size_t)blockDim.x + threadIdx.x; t < total; t += (size_t)gridDim.x * blockDim.x) {
        const int i = (int)(t / n), j = (int)(t % n);
        inv[t] = M[(size_t)perm[i] * 2 * n + n + j];
    }
}

__global__ void k_iota2(int n, int *a, int *b) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) a[i] = b[i] = i;
}

// ------------------------------------------------------------------ blocked Gauss-Jordan
// The same elimination in blocks of GJB steps.  Panel (one cooperative
// launch per block of steps [k0, ke)): for each step k the pivot search over
// the panel column k, then the pivot row R brought to step k over the
// columns j >= ke (the block's earlier steps q < k applied with R's
// multipliers m_Rq, which sit in R's panel columns) and divided, kept in
// Ub[k - k0], then the panel columns (k, ke) of every other row updated.
// Trailing update (one launch): every value m_ij, j >= ke, goes through the
// block's steps in ascending order, m_ij - m_iq u_qj as one fused
// multiply-add, skipped when either factor is zero, exactly as the
// one-step-at-a-time elimination does; a pivot row of the block starts from
// its divided value after its own step.  Right-part columns of rows not yet
// pivoted are zero in every pivot row and are not visited.  The inverse is
// the one of the unblocked elimination bit for bit in its nonzero values.
constexpr int GJB = 64;            // steps per block
constexpr int GJ_PANEL_THREADS = 256;

__device__ __forceinline__ void gj_reduce_parts(const GjPart *parts, int nparts, double &best, int &bl, int &br) {
    __shared__ double sv[GJ_PANEL_THREADS / 32];
    __shared__ int sl[GJ_PANEL_THREADS / 32], sr[GJ_PANEL_THREADS / 32];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    double b = -1.0;
    int l = INT_MAX, r = -1;
    for (int g = tid; g < nparts; g += blockDim.x) {
        const double v = __ldcg(&parts[g].v);
        const int gl = __ldcg(&parts[g].l), gr = __ldcg(&parts[g].r);
        if (gj_better(v, gl, b, l)) { b = v; l = gl; r = gr; }
    }
    for (int off = 16; off; off >>= 1) {
        const double ob = __shfl_down_sync(0xffffffffu, b, off);
        const int ol = __shfl_down_sync(0xffffffffu, l, off);
        const int orr = __shfl_down_sync(0xffffffffu, r, off);
        if (gj_better(ob, ol, b, l)) { b = ob; l = ol; r = orr; }
    }
    if (lane == 0) { sv[warp] = b; sl[warp] = l; sr[warp] = r; }
    __syncthreads();
    if (tid == 0) {
        for (int q = 1; q < (int)blockDim.x / 32; ++q)
            if (gj_better(sv[q], sl[q], sv[0], sl[0])) { sv[0] = sv[q]; sl[0] = sl[q]; sr[0] = sr[q]; }
    }
    __syncthreads();
    best = sv[0];
    bl = sl[0];
    br = sr[0];
    __syncthreads();
}

// This block's candidate for the pivot of panel column cq (column k0 + cq)
// from its shared-memory panel rows: the largest |m_ic| over rows i with
// logical position > kmin (first logical position on ties).
__device__ __forceinline__ void gj_panel_candidate(const double *pan, const int *lpos, int cq, int kmin, int r0,
                                                   int r1, int n, GjPart *out) {
    __shared__ double sv[GJ_PANEL_THREADS / 32];
    __shared__ int sl[GJ_PANEL_THREADS / 32], sr[GJ_PANEL_THREADS / 32];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    double b = -1.0;
    int l = INT_MAX, r = -1;
    for (int i = r0 + tid; i < r1; i += blockDim.x) {
        const int li = lpos[i - r0];
        if (li <= kmin) continue;
        const double a = fabs(pan[(size_t)(i - r0) * GJB + cq]);
        if (gj_better(a, li, b, l)) { b = a; l = li; r = i; }
    }
    for (int off = 16; off; off >>= 1) {
        const double ob = __shfl_down_sync(0xffffffffu, b, off);
        const int ol = __shfl_down_sync(0xffffffffu, l, off);
        const int orr = __shfl_down_sync(0xffffffffu, r, off);
        if (gj_better(ob, ol, b, l)) { b = ob; l = ol; r = orr; }
    }
    if (lane == 0) { sv[warp] = b; sl[warp] = l; sr[warp] = r; }
    __syncthreads();
    if (tid == 0) {
        for (int q = 1; q < (int)blockDim.x / 32; ++q)
            if (gj_better(sv[q], sl[q], sv[0], sl[0])) { sv[0] = sv[q]; sl[0] = sl[q]; sr[0] = sr[q]; }
        out[blockIdx.x] = GjPart{sv[0], sl[0] == INT_MAX ? n : sl[0], sr[0]};
    }
    __syncthreads();
}

// Panel kernel of the steps [k0, ke), one grid barrier per step.  Block b
// keeps the panel columns of its rows [r0, r1) in shared memory and its rows'
// logical positions; it writes every update of a row that is not the step's
// pivot through to M (a later pivot row is read from there) and writes all
// back at the end.  Step k: every block reduces the pivot candidates to the
// same (p, R), reads R's panel values from M and divides them itself (the
// same operations, so the same bits in every block).  Thread t of block b
// owns the trailing column ke + t gridDim.x + b for all steps (the FP64 work
// spread over every SM) and keeps the divided pivot rows' values in that
// column in registers, so R's trailing value is brought to step k (the
// block's earlier steps, with R's multipliers) without further global loads,
// divided, and written to M and Ub.  Then each block updates its rows' panel
// columns after k and computes its candidate for column k + 1.  parts holds
// two sets of gridDim.x candidates.  Needs 2n - ke <= gridDim.x * blockDim.x
// (checked by the launcher).
__global__ void __launch_bounds__(GJ_PANEL_THREADS) k_gj_panel(int n, int k0, int kb, double *M, int *perm, int *pos,
                                                               double *Ub, GjPart *parts, int *breakdown,
                                                               unsigned int *bar, int *err) {
    extern __shared__ __align__(16) double gp_sm[];
    __shared__ int s_R;
    const size_t w = 2 * (size_t)n;
    const int ke = k0 + kb;
    const size_t wu = w - (size_t)ke;
    const int tid = threadIdx.x;
    const int rpb = (n + gridDim.x - 1) / gridDim.x;
    const int r0 = min(n, blockIdx.x * rpb), r1 = min(n, r0 + rpb), nr = r1 - r0;
    double *pan = gp_sm;                                 // [rpb][GJB] this block's rows, panel columns
    double *prow = pan + (size_t)rpb * GJB;              // [GJB] the pivot row's panel values
    int *lpos = reinterpret_cast<int *>(prow + GJB);     // [rpb] logical positions of this block's rows
    for (int e = tid; e < nr * kb; e += blockDim.x)
        pan[(e / kb) * GJB + e % kb] = M[(size_t)(r0 + e / kb) * w + k0 + e % kb];
    for (int i = tid; i < nr; i += blockDim.x) lpos[i] = pos[r0 + i];
    // trailing columns interleaved over the blocks (each SM gets a share of
    // the pivot row's FP64 work): thread (b, t) owns column ke + t G + b
    const size_t jt = (size_t)ke + (size_t)tid * gridDim.x + blockIdx.x;
    const bool has_col = jt < w;
    double ucol[GJB];
#pragma unroll
    for (int q = 0; q < GJB; ++q) ucol[q] = 0.0;
    __syncthreads();
    // candidates of the pivot of column c in parts[(c & 1) G + b]: a block
    // may write the next column's while another still reduces this one's
    const int G = gridDim.x;
    gj_panel_candidate(pan, lpos, 0, k0 - 1, r0, r1, n, parts + (size_t)(k0 & 1) * G);
    grid_barrier(bar, err);
    for (int k = k0; k < ke; ++k) {
        if (*(volatile int *)err) return;
        const int kq = k - k0;
        double best;
        int p, R;
        gj_reduce_parts(parts + (size_t)(k & 1) * G, G, best, p, R);
        if (!(best > 0.0) || !isfinite(best)) {      // singular: keep position k, no swap (the result is flagged)
            if (blockIdx.x == 0 && tid == 0) atomicExch(breakdown, 1);
            p = k;
            if (tid == 0) s_R = -1;
            __syncthreads();
            for (int i = tid; i < nr; i += blockDim.x)      // the row at position k, if it is one of ours
                if (lpos[i] == k) s_R = r0 + i;
            __syncthreads();
            R = s_R >= 0 ? s_R : __ldcg(perm + k);           // perm[k] is only written by block 0, below
        }
        __syncthreads();
        if (blockIdx.x == 0 && tid == 0) {
            const int rk = perm[k];
            perm[k] = R; perm[p] = rk;
            pos[R] = k; pos[rk] = p;
        }
        for (int i = tid; i < nr; i += blockDim.x) {     // the row at k moves to p, R to k
            if (lpos[i] == k) lpos[i] = p;
            if (r0 + i == R) lpos[i] = k;
        }
        // the pivot row's panel values and, for this thread's column, its trailing value
        double v = has_col ? __ldcg(M + (size_t)R * w + jt) : 0.0;
        for (int q = tid; q < kb; q += blockDim.x) prow[q] = __ldcg(M + (size_t)R * w + k0 + q);
        __syncthreads();
        const double d = prow[kq];
        if (has_col) {
#pragma unroll
            for (int q = 0; q < GJB; ++q) {
                if (q < kq) {
                    const double f = prow[q], u = ucol[q];
                    if (gj_nonzero(f) && gj_nonzero(u)) v = __fma_rn(-f, u, v);
                }
            }
            v = __ddiv_rn(v, d);
            M[(size_t)R * w + jt] = v;
            Ub[(size_t)kq * wu + (jt - ke)] = v;
#pragma unroll
            for (int q = 0; q < GJB; ++q)
                if (q == kq) ucol[q] = v;
        }
        __syncthreads();                                   // prow[q < kq] read; now the panel part
        const bool own = R >= r0 && R < r1;                // this block holds the pivot row
        for (int q = kq + 1 + tid; q < kb; q += blockDim.x) {
            const double u = __ddiv_rn(prow[q], d);
            prow[q] = u;
            // (only the shared copy: other blocks may still be reading R's
            // panel values from M in this step; written back at the end)
            if (own) pan[(size_t)(R - r0) * GJB + q] = u;
        }
        __syncthreads();
        const int pw = kb - kq - 1;                        // panel columns after k
        for (int e = tid; e < nr * pw; e += blockDim.x) {
            const int li = e / pw, i = r0 + li;
            if (i == R) continue;
            const int c = kq + 1 + e % pw;
            double *pi = pan + (size_t)li * GJB;
            const double f = pi[kq], u = prow[c];
            if (gj_nonzero(f) && gj_nonzero(u)) {
                const double nv = __fma_rn(-f, u, pi[c]);
                pi[c] = nv;
                M[(size_t)i * w + k0 + c] = nv;
            }
        }
        __syncthreads();
        if (pw > 0) gj_panel_candidate(pan, lpos, kq + 1, k, r0, r1, n, parts + (size_t)((k + 1) & 1) * G);
        grid_barrier(bar, err);
    }
    for (int e = tid; e < nr * kb; e += blockDim.x)
        M[(size_t)(r0 + e / kb) * w + k0 + e % kb] = pan[(e / kb) * GJB + e % kb];
}

// Trailing update of a block: a tile of GJT_R rows x GJT_C columns per CTA;
// thread (tr, tc) updates rows tr + 16 a (a < 4) and columns tc + 16 b (b <
// 8).  The block's multipliers and divided pivot rows are staged in shared
// memory.  Columns c < n - ke are the left part's columns ke + c, the rest
// the right-part columns n + perm[l], l < ke.  Every value takes the block's
// steps in ascending order as one fused multiply-add each (a pivot row of the
// block only the steps after its own); a product with a zero factor is not
// skipped here, which changes at most the sign of a zero value, never a
// nonzero one, and no later step tells the two zeros apart (the tests for
// zero ignore the sign).  A step whose multipliers or pivot-row values are
// all zero in the tile is skipped as a whole.
constexpr int GJT_R = 64, GJT_C = 128;
constexpr size_t GJT_SMEM = sizeof(double) * GJB * (GJT_R + GJT_C) + sizeof(size_t) * GJT_C + sizeof(int) * GJT_R +
                            2 * sizeof(int) * GJB;

__global__ void __launch_bounds__(256) k_gj_trailing(int n, int k0, int kb, double *M, const int *perm,
                                                     const int *pos, const double *Ub) {
    extern __shared__ __align__(16) unsigned char gjt_raw[];
    double (*ms)[GJT_R] = reinterpret_cast<double (*)[GJT_R]>(gjt_raw);
    double (*us)[GJT_C] = reinterpret_cast<double (*)[GJT_C]>(gjt_raw + sizeof(double) * GJB * GJT_R);
    size_t *cj = reinterpret_cast<size_t *>(gjt_raw + sizeof(double) * GJB * (GJT_R + GJT_C));
    int *ks = reinterpret_cast<int *>(cj + GJT_C);
    int *mnz = ks + GJT_R, *unz = mnz + GJB;       // per step: some multiplier / pivot-row value nonzero
    const size_t w = 2 * (size_t)n;
    const int ke = k0 + kb;
    const size_t wu = w - (size_t)ke;
    const int nleft = n - ke;
    const int i0 = blockIdx.y * GJT_R, c0 = blockIdx.x * GJT_C;
    const int tid = threadIdx.x;
    if (tid < GJT_C) {
        const int c = c0 + tid;
        cj[tid] = c < nleft ? (size_t)ke + c : (c < n ? (size_t)n + perm[c - nleft] : (size_t)-1);
    }
    if (tid < GJT_R) {
        const int i = i0 + tid;
        const int l = i < n ? pos[i] : 0;
        ks[tid] = (l >= k0 && l < ke) ? l - k0 + 1 : 0;
    }
    if (tid < GJB) { mnz[tid] = 0; unz[tid] = 0; }
    __syncthreads();
    for (int e = tid; e < GJB * GJT_R; e += 256) {
        const int r = e / GJB, q = e % GJB, i = i0 + r;
        const double v = (i < n && q < kb) ? M[(size_t)i * w + k0 + q] : 0.0;
        ms[q][r] = v;
        if (gj_nonzero(v)) mnz[q] = 1;
    }
    for (int e = tid; e < GJB * GJT_C; e += 256) {
        const int q = e / GJT_C, c = e % GJT_C;
        const size_t j = cj[c];
        const double v = (q < kb && j != (size_t)-1) ? Ub[(size_t)q * wu + (j - ke)] : 0.0;
        us[q][c] = v;
        if (gj_nonzero(v)) unz[q] = 1;
    }
    __syncthreads();
    const int tr = tid / 16, tc = tid % 16;
    double acc[4][8];
    int rks[4];
    bool rin[4], cin[8];
    size_t rj[8];
    int kmax = 0;
#pragma unroll
    for (int a = 0; a < 4; ++a) {
        rin[a] = i0 + tr + 16 * a < n;
        rks[a] = ks[tr + 16 * a];
        kmax = max(kmax, rks[a]);
    }
#pragma unroll
    for (int b = 0; b < 8; ++b) {
        rj[b] = cj[tc + 16 * b];
        cin[b] = rj[b] != (size_t)-1;
    }
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 8; ++b)
            acc[a][b] = (rin[a] && cin[b]) ? M[(size_t)(i0 + tr + 16 * a) * w + rj[b]] : 0.0;
    for (int q = 0; q < kb; ++q) {
        if (!mnz[q] || !unz[q]) continue;             // uniform over the CTA
        double m[4], u[8];
#pragma unroll
        for (int a = 0; a < 4; ++a) m[a] = ms[q][tr + 16 * a];
#pragma unroll
        for (int b = 0; b < 8; ++b) u[b] = us[q][tc + 16 * b];
        if (q >= kmax) {                              // no pivot row of the block still before its step
#pragma unroll
            for (int a = 0; a < 4; ++a)
#pragma unroll
                for (int b = 0; b < 8; ++b) acc[a][b] = __fma_rn(-m[a], u[b], acc[a][b]);
        } else {
#pragma unroll
            for (int a = 0; a < 4; ++a)
                if (q >= rks[a]) {
#pragma unroll
                    for (int b = 0; b < 8; ++b) acc[a][b] = __fma_rn(-m[a], u[b], acc[a][b]);
                }
        }
    }
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 8; ++b)
            if (rin[a] && cin[b]) M[(size_t)(i0 + tr + 16 * a) * w + rj[b]] = acc[a][b];
}

// Levels with at least this many rows use the blocked elimination.
constexpr int GJ_BLOCKED_MIN = 256;

void dense_inverse(const DCsr &A, DBuf<double> &inv, cudaStream_t s) {
    const int n = A.n;
    DBuf<double> M((size_t)n * 2 * n);
    DBuf<int> bd(1), perm(n), pos(n), R(1);
    const int gy = std::max(1, std::min(n, 2 * sm_count()));
    DBuf<GjPart> parts(std::max(gy, sm_count()));
    CU(cudaMemsetAsync(bd.get(), 0, sizeof(int), s));
    k_dense_from_csr<<<grid_for(n, 128), 128, 0, s>>>(n, A.rp.get(), A.ci.get(), A.v.get(), M.get());
    CU_LAUNCH("k_dense_from_csr"); count_launch();
    k_iota2<<<grid_for(n, 256), 256, 0, s>>>(n, perm.get(), pos.get());
    CU_LAUNCH("k_iota2"); count_launch();
    if (n >= GJ_BLOCKED_MIN) {
        // panel: one block per SM at most (its threads keep 64 FP64 values each
        // in registers), enough threads for one trailing column each
        const int G = std::min(sm_count(), std::max(1, (n + 15) / 16));
        const int rpb = (n + G - 1) / G;
        const size_t psmem = sizeof(double) * ((size_t)rpb * GJB + GJB) + sizeof(int) * (size_t)rpb;
        static const bool attrs = [] {
            CU(cudaFuncSetAttribute(k_gj_trailing, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)GJT_SMEM));
            CU(cudaFuncSetAttribute(k_gj_panel, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024));
            return true;
        }();
        (void)attrs;
        int per_sm = 0;
        CU(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_gj_panel, GJ_PANEL_THREADS, psmem));
        if (per_sm < 1 || psmem > 200 * 1024 || 2 * (size_t)n > (size_t)G * GJ_PANEL_THREADS + GJB ||
            (size_t)2 * G > parts.n)
            fail(4, "dense solve of the last level: blocked elimination does not fit");
        DBuf<double> Ub((size_t)GJB * 2 * n);
        DBuf<unsigned int> bar(2);
        DBuf<int> err(1);
        CU(cudaMemsetAsync(bar.get(), 0, 2 * sizeof(unsigned int), s));
        CU(cudaMemsetAsync(err.get(), 0, sizeof(int), s));
        for (int k0 = 0; k0 < n; k0 += GJB) {
            int kb = std::min(GJB, n - k0);
            int nn = n;
            int k0v = k0;
            double *Mp = M.get(), *Up = Ub.get();
            int *pp = perm.get(), *qp = pos.get(), *bp = bd.get(), *ep = err.get();
            GjPart *parts_p = parts.get();
            unsigned int *barp = bar.get();
            void *args[] = {&nn, &k0v, &kb, &Mp, &pp, &qp, &Up, &parts_p, &bp, &barp, &ep};
            CU(cudaLaunchCooperativeKernel((const void *)k_gj_panel, dim3(G), dim3(GJ_PANEL_THREADS), args, psmem, s));
            count_launch();
            const dim3 grid((n + GJT_C - 1) / GJT_C, (n + GJT_R - 1) / GJT_R);
            k_gj_trailing<<<grid, 256, GJT_SMEM, s>>>(n, k0, kb, M.get(), perm.get(), pos.get(), Ub.get());
            CU_LAUNCH("k_gj_trailing"); count_launch();
        }
        if (read_int(err.get(), s)) fail(8, "dense solve of the last level: a grid barrier wait gave up");
    } else {
        for (int k = 0; k < n; ++k) {
            const int pb = std::max(1, std::min((2 * n - k - 1 + 1023) / 1024, sm_count()));
            k_gj_pivot<<<pb, 256, 0, s>>>(n, k, M.get(), perm.get(), pos.get(), parts.get(), k == 0 ? 0 : gy,
                                          R.get(), bd.get());      // nparts == 0 only at k == 0
            // columns j > k over x (one thread each per pass), row groups over y
            const int xb = std::max(1, std::min((2 * n - k - 1 + 255) / 256, 64));
            k_gj_elim<<<dim3(xb, gy), 256, 0, s>>>(n, k, M.get(), pos.get(), R.get(), parts.get());
            count_launch(2);
        }
        CU_LAUNCH("k_gj_*");
    }
    inv.alloc((size_t)n * n);
    k_extract_inverse<<<grid_for((size_t)n * n, 256), 256, 0, s>>>(n, M.get(), perm.get(), inv.get());
    CU_LAUNCH("k_extract_inverse"); count_launch();
    if (read_int(bd.get(), s)) fail(5, "dense solve of the last level: singular matrix");
}

// ------------------------------------------------------------------ SELL-32 layout
__global__ void k_sell_width(int n, const int *rp, int nslices, int *w) {
    for (int sl = blockIdx.x * blockDim.x + threadIdx.x; sl < nslices; sl += gridDim.x * blockDim.x) {
        int m = 0;
        for (int r = 0; r < 32; ++r) {
            const int i = sl * 32 + r;
            if (i < n) m = max(m, rp[i + 1] - rp[i]);
        }
        w[sl] = m;
    }
}

__global__ void k_sell_fill(int n, const int *rp, const int *ci, const double *v, const int64_t *ptr, int *sci,
                            double *sv) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < ((n + 31) / 32) * 32; i += gridDim.x * blockDim.x) {
        const int sl = i >> 5, r = i & 31;
        const int64_t base = ptr[sl];
        const int w = (int)((ptr[sl + 1] - base) >> 5);
        if (i >= n) {                               // rows past the end of the last slice
            for (int k = 0; k < w; ++k) { sci[base + 32 * k + r] = 0; sv[base + 32 * k + r] = 0.0; }
            continue;
        }
        const int b = rp[i], len = rp[i + 1] - b;
        for (int k = 0; k < w; ++k) {
            const int64_t e = base + 32 * (int64_t)k + r;
            if (k < len) { sci[e] = ci[b + k]; sv[e] = v[b + k]; }
            else { sci[e] = i; sv[e] = 0.0; }
        }
    }
}

__global__ void k_widths_to_sizes(const int *w, int nslices, int64_t *sz) {
    for (int sl = blockIdx.x * blockDim.x + threadIdx.x; sl < nslices; sl += gridDim.x * blockDim.x)
        sz[sl] = 32 * (int64_t)w[sl];
}

void build_sell(const DCsr &A, const double *vals, Sell &S, cudaStream_t s) {
    S.n = A.n;
    S.nslices = (A.n + 31) / 32;
    DBuf<int> w(S.nslices);
    k_sell_width<<<grid_for(S.nslices, 256), 256, 0, s>>>(A.n, A.rp.get(), S.nslices, w.get());
    CU_LAUNCH("k_sell_width"); count_launch();
    std::vector<int> hw(S.nslices);
    CU(cudaMemcpyAsync(hw.data(), w.get(), sizeof(int) * S.nslices, cudaMemcpyDeviceToHost, s));
    CU(cudaStreamSynchronize(s));
    std::vector<int64_t> hp(S.nslices + 1, 0);
    for (int sl = 0; sl < S.nslices; ++sl) hp[sl + 1] = hp[sl] + 32 * (int64_t)hw[sl];
    S.padded = hp[S.nslices];
    S.ptr.alloc(S.nslices + 1);
    CU(cudaMemcpyAsync(S.ptr.get(), hp.data(), sizeof(int64_t) * (S.nslices + 1), cudaMemcpyHostToDevice, s));
    S.ci.alloc(S.padded > 0 ? S.padded : 1);
    S.v.alloc(S.padded > 0 ? S.padded : 1);
    k_sell_fill<<<grid_for((size_t)S.nslices * 32, 256), 256, 0, s>>>(A.n, A.rp.get(), A.ci.get(), vals, S.ptr.get(),
                                                                      S.ci.get(), S.v.get());
    CU_LAUNCH("k_sell_fill"); count_launch();
    CU(cudaStreamSynchronize(s));
}

// ------------------------------------------------------------------ casts
__global__ void k_cast32(const double *in, float *out, size_t n) {
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
        out[i] = __double2float_rn(in[i]);
}
__global__ void k_cast16(const double *in, __nv_bfloat16 *out, size_t n) {
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
        out[i] = __double2bfloat16(in[i]);
}
void cast_f64_f32(const double *in, float *out, size_t n, cudaStream_t s) {
    if (!n) return;
    k_cast32<<<grid_for(n, 256), 256, 0, s>>>(in, out, n);
    CU_LAUNCH("k_cast32"); count_launch();
}
void cast_f64_bf16(const double *in, __nv_bfloat16 *out, size_t n, cudaStream_t s) {
    if (!n) return;
    k_cast16<<<grid_for(n, 256), 256, 0, s>>>(in, out, n);
    CU_LAUNCH("k_cast16"); count_launch();
}

// ------------------------------------------------------------------ FV assembly (eq. (2))
struct FvGrid {
    int dim, nx, ny, nz;
    double hd2, hd;
};

// Face q in W, E, S, N, B, T order: neighbour, kind (0 interior, 1
// Dirichlet, 2 Neumann), conductivities, outward flux.
__device__ __forceinline__ void fv_face(const FvGrid &g, int i, int j, int k, long P, int q,
                                        const double *kx, const double *ky, const double *kz,
                                        const double *fx, const double *fy, const double *fz,
                                        long &nb, int &kind, double &kP, double &kN, double &F) {
    const long sxy = (long)g.nx * g.ny;
    switch (q) {
    case 0: nb = P - 1; kind = (i == 0) ? 2 : 0; kP = kx[P]; kN = (i == 0) ? 0.0 : kx[P - 1];
        F = -fx[i + (long)(g.nx + 1) * (j + (long)g.ny * k)]; break;
    case 1: nb = P + 1; kind = (i == g.nx - 1) ? 2 : 0; kP = kx[P]; kN = (i == g.nx - 1) ? 0.0 : kx[P + 1];
        F = fx[(i + 1) + (long)(g.nx + 1) * (j + (long)g.ny * k)]; break;
    case 2: nb = P - g.nx; kind = (j == 0) ? 1 : 0; kP = ky[P]; kN = (j == 0) ? 0.0 : ky[P - g.nx];
        F = -fy[i + (long)g.nx * (j + (long)(g.ny + 1) * k)]; break;
    case 3: nb = P + g.nx; kind = (j == g.ny - 1) ? 1 : 0; kP = ky[P]; kN = (j == g.ny - 1) ? 0.0 : ky[P + g.nx];
        F = fy[i + (long)g.nx * ((j + 1) + (long)(g.ny + 1) * k)]; break;
    case 4: nb = P - sxy; kind = (k == 0) ? 2 : 0; kP = kz[P]; kN = (k == 0) ? 0.0 : kz[P - sxy];
        F = -fz[i + (long)g.nx * (j + (long)g.ny * k)]; break;
    default: nb = P + sxy; kind = (k == g.nz - 1) ? 2 : 0; kP = kz[P]; kN = (k == g.nz - 1) ? 0.0 : kz[P + sxy];
        F = fz[i + (long)g.nx * (j + (long)g.ny * (k + 1))]; break;
    }
}

__device__ __forceinline__ double harmonic_T(double hd2, double kP, double kN) {
    return __dmul_rn(hd2, __ddiv_rn(__dmul_rn(__dmul_rn(2.0, kP), kN), __dadd_rn(kP, kN)));
}

__global__ void k_fv_count(FvGrid g, int *cnt) {
    const long N = (long)g.nx * g.ny * g.nz;
    for (long P = blockIdx.x * (long)blockDim.x + threadIdx.x; P < N; P += (long)gridDim.x * blockDim.x) {
        int i = (int)(P % g.nx), j = (int)((P / g.nx) % g.ny), k = (int)(P / ((long)g.nx * g.ny));
        int m = 1;
        m += (i > 0) + (i < g.nx - 1) + (j > 0) + (j < g.ny - 1);
        if (g.dim == 3) m += (k > 0) + (k < g.nz - 1);
        cnt[P] = m;
    }
}

__global__ void k_fv_fill(FvGrid g, const double *kx, const double *ky, const double *kz, const double *fx,
                          const double *fy, const double *fz, const double *f, const int *rp32, int64_t *rp,
                          int *ci, double *v, double *b) {
    const long N = (long)g.nx * g.ny * g.nz;
    for (long P = blockIdx.x * (long)blockDim.x + threadIdx.x; P < N; P += (long)gridDim.x * blockDim.x) {
        int i = (int)(P % g.nx), j = (int)((P / g.nx) % g.ny), k = (int)(P / ((long)g.nx * g.ny));
        const int nf = g.dim == 3 ? 6 : 4;
        long nbv[6];
        int kind[6];
        double off[6];
        double diag = 0.0;
        for (int q = 0; q < nf; ++q) {
            double kP, kN, F;
            fv_face(g, i, j, k, P, q, kx, ky, kz, fx, fy, fz, nbv[q], kind[q], kP, kN, F);
            off[q] = 0.0;
            if (kind[q] == 0) {
                double T = harmonic_T(g.hd2, kP, kN);
                diag = __dadd_rn(diag, T);
                if (F > 0.0) diag = __dadd_rn(diag, F);
                off[q] = -T;
                if (F < 0.0) off[q] = __dadd_rn(off[q], F);
            } else if (kind[q] == 1) {
                double T = __dmul_rn(g.hd2, __dmul_rn(2.0, kP));
                diag = __dadd_rn(diag, T);
                if (F > 0.0) diag = __dadd_rn(diag, F);
            } else {
                diag = __dadd_rn(diag, F);
            }
        }
        const int ord3[7] = {4, 2, 0, -1, 1, 3, 5};
        const int ord2[5] = {2, 0, -1, 1, 3};
        const int *ord = g.dim == 3 ? ord3 : ord2;
        const int nord = g.dim == 3 ? 7 : 5;
        int m = rp32[P];
        for (int t = 0; t < nord; ++t) {
            int q = ord[t];
            if (q < 0) { ci[m] = (int)P; v[m] = diag; ++m; }
            else if (kind[q] == 0) { ci[m] = (int)nbv[q]; v[m] = off[q]; ++m; }
        }
        rp[P] = rp32[P];
        if (P == N - 1) rp[N] = rp32[N];
        b[P] = __dmul_rn(f[P], g.hd);
    }
}

int64_t fv_assemble(int dim, int nx, int ny, int nz, const double *kx, const double *ky, const double *kz,
                    const double *fx, const double *fy, const double *fz, const double *f, int64_t *rp, int *ci,
                    double *v, double *b, cudaStream_t s) {
    FvGrid g;
    g.dim = dim; g.nx = nx; g.ny = ny; g.nz = nz;
    const double h = 1.0 / (double)nx;
    g.hd2 = dim == 2 ? 1.0 : h;
    g.hd = dim == 2 ? h * h : h * h * h;
    const long N = (long)nx * ny * nz;
    DBuf<int> cnt(N + 1), rp32(N + 1);
    fill_int(cnt.get(), 0, (int)(N + 1), s);
    k_fv_count<<<grid_for(N, 256), 256, 0, s>>>(g, cnt.get());
    CU_LAUNCH("k_fv_count"); count_launch();
    int nnz = 0;
    exclusive_scan_int(cnt.get(), rp32.get(), (int)(N + 1), &nnz, s);
    k_fv_fill<<<grid_for(N, 256), 256, 0, s>>>(g, kx, ky, kz, fx, fy, fz, f, rp32.get(), rp, ci, v, b);
    CU_LAUNCH("k_fv_fill"); count_launch();
    CU(cudaStreamSynchronize(s));
    return nnz;
}

// ISO: kx = ky = kz = kappa (one conductivity per cell), and the derivative
// with respect to log kappa is the sum of the per-axis ones, added in axis
// order (x + y) + z into gx; gy, gz are not written.
template <bool ISO>
__global__ void k_fv_grad(FvGrid g, const double *kx, const double *ky, const double *kz, const double *lam,
                          const double *x, double *gx, double *gy, double *gz) {
    const long N = (long)g.nx * g.ny * g.nz;
    const long sxy = (long)g.nx * g.ny;
    for (long P = blockIdx.x * (long)blockDim.x + threadIdx.x; P < N; P += (long)gridDim.x * blockDim.x) {
        int c[3] = {(int)(P % g.nx), (int)((P / g.nx) % g.ny), (int)(P / sxy)};
        int dims[3] = {g.nx, g.ny, g.nz};
        long stride[3] = {1, g.nx, sxy};
        double iso = 0.0;
        for (int axis = 0; axis < g.dim; ++axis) {
            const double *kk = axis == 0 ? kx : (axis == 1 ? ky : kz);
            double acc = 0.0;
            for (int side = 0; side < 2; ++side) {
                bool bnd = side == 0 ? (c[axis] == 0) : (c[axis] == dims[axis] - 1);
                if (bnd) {
                    if (axis == 1) {
                        double T = __dmul_rn(g.hd2, __dmul_rn(2.0, kk[P]));
                        double dLdT = -lam[P] * x[P];
                        acc = __dadd_rn(acc, __dmul_rn(dLdT, T));
                    }
                    continue;
                }
                long Q = side == 0 ? P - stride[axis] : P + stride[axis];
                double kP = kk[P], kN = kk[Q];
                double T = harmonic_T(g.hd2, kP, kN);
                double dLdT = __dmul_rn(-__dsub_rn(lam[P], lam[Q]), __dsub_rn(x[P], x[Q]));
                acc = __dadd_rn(acc, __dmul_rn(dLdT, __ddiv_rn(__dmul_rn(T, kN), __dadd_rn(kP, kN))));
            }
            if (ISO) {
                iso = axis == 0 ? acc : __dadd_rn(iso, acc);
            } else {
                double *gg = axis == 0 ? gx : (axis == 1 ? gy : gz);
                gg[P] = acc;
            }
        }
        if (ISO) gx[P] = iso;
    }
}

__global__ void k_exp(long n, const double *in, double *out) {
    for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x)
        out[i] = exp(in[i]);
}

void exp_f64(long n, const double *in, double *out, cudaStream_t s) {
    k_exp<<<grid_for(n, 256), 256, 0, s>>>(n, in, out);
    CU_LAUNCH("k_exp"); count_launch();
}

void fv_grad_logk(int dim, int nx, int ny, int nz, const double *kx, const double *ky, const double *kz,
                  const double *lam, const double *x, double *gx, double *gy, double *gz, cudaStream_t s) {
    FvGrid g;
    g.dim = dim; g.nx = nx; g.ny = ny; g.nz = nz;
    const double h = 1.0 / (double)nx;
    g.hd2 = dim == 2 ? 1.0 : h;
    g.hd = dim == 2 ? h * h : h * h * h;
    const long N = (long)nx * ny * nz;
    if (gy)
        k_fv_grad<false><<<grid_for(N, 256), 256, 0, s>>>(g, kx, ky, kz, lam, x, gx, gy, gz);
    else
        k_fv_grad<true><<<grid_for(N, 256), 256, 0, s>>>(g, kx, kx, kx, lam, x, gx, nullptr, nullptr);
    CU_LAUNCH("k_fv_grad"); count_launch();
}

}  // namespace amg
