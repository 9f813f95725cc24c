// tiles.cu -- the finest level's ILU(0) triangular solves for a matrix whose
// pattern is a 5-point (2D) or 7-point (3D) stencil on an nx x ny (x nz) grid
// numbered in natural order (x fastest).
//
// Natural-order ILU(0) is the smoother of the finest level (Section 3,
// GMG-NO; the SOLVE S t = z step of Algorithm 1).  Row (x, y, z) of the lower
// factor reads rows (x-1, y, z), (x, y-1, z) and (x, y, z-1), so the rows of
// one anti-diagonal x + y + z = d are independent and the forward solve is
// nx + ny + nz - 2 dependent wavefronts; the backward solve is the same with
// every axis reversed.  The grid is cut into tiles of 16^3 rows (64^2 in 2D).
// One thread block solves a tile.  Its right-hand side is staged in shared
// memory and its factor values arrive there by one bulk copy of the
// tensor-memory-access engine.  Compute thread (j, k) owns the tile's grid
// line (., j, k) and solves row i = d - j - k at step d: its x neighbour is
// the value it computed one step earlier (a register), its y and z
// neighbours were written to shared memory by threads (j-1, k) and (j, k-1)
// one step earlier, and a barrier of the compute warps separates the steps.
// Only the faces between tiles go through global memory: a row on a tile's
// last plane (x = 15, ...) is also stored in a mailbox of its tile, which
// holds a sentinel until written.  A halo warp of the consuming block polls
// those mailboxes a window of wavefronts ahead of its compute warps, moves
// the values that have arrived to shared memory and publishes how many
// wavefronts have their halo complete.  A tile therefore starts when the
// first rows of its neighbours' last planes are solved, and the tiles along
// a dependence chain run as a pipeline: the critical path is about
// nx + ny + nz steps plus one mailbox hop per tile boundary crossed.
//
// Every row is computed as in the sequential definition: acc = right-hand
// side, minus each factor entry times its solved neighbour in stored
// (ascending column) order by fused multiply-add, divided by the diagonal
// where the factor has one; the results are bit-identical to the other sweep
// kernels.
//
// Progress: all blocks are resident (cooperative launch) and block b takes
// the tiles b, b + G, b + 2G, ... of a topological order (by tile
// anti-diagonal), so the lowest unfinished tile has all its producers
// finished and an owner working on it.  Every wait is bounded; on expiry
// *err is set, the waits of the block end and the kernel returns.
// Mailbox upkeep: the forward phase's mailboxes are reset to the sentinel
// during the backward phase and the backward phase's during the forward
// phase; the grid barrier between the phases orders each reset against the
// uses of that array.
#include "amg.h"
#include "solve.cuh"
#include "devsync.cuh"

#include <algorithm>
#include <climits>
#include <vector>

namespace amg {

namespace {

constexpr unsigned int TILE_SPIN_LIMIT = 1u << 22;   // polls of one wait
constexpr int TILE_MAX_THREADS = 288;                // 16 x 16 line threads + the halo warp
#ifndef AMG_TILE_HALO_PER_LANE
#define AMG_TILE_HALO_PER_LANE 8
#endif
constexpr int HALO_PER_LANE = AMG_TILE_HALO_PER_LANE;   // mailbox loads per lane and poll round
// Sleep between polls that found nothing new (halo warp; compute threads
// waiting for a halo sleep a quarter of it), and a cap on resident blocks
// per SM (0: as many as fit): compile-time tunables.
#ifndef AMG_TILE_SLEEP_NS
#define AMG_TILE_SLEEP_NS 0
#endif
#ifndef AMG_TILE_BLOCKS_PER_SM
#define AMG_TILE_BLOCKS_PER_SM 0
#endif
constexpr unsigned int TILE_SLEEP_NS = AMG_TILE_SLEEP_NS;
constexpr int TILE_BLOCKS_PER_SM = AMG_TILE_BLOCKS_PER_SM;
// Right-hand-side values a thread loads before storing any (loads in flight)
constexpr int STAGE_BATCH = 8;

// Shared-memory layout of the tile kernel (host and device agree on it).
struct TileSmem {
    unsigned int ys, cs, ds, hs, hent, hwoff, mbar, flags, total;
    __host__ __device__ static unsigned int take(unsigned int &o, unsigned int bytes) {
        const unsigned int r = o;
        o = (o + bytes + 127u) & ~127u;
        return r;
    }
    __host__ __device__ TileSmem(const TileGeom &g, unsigned int tsz, unsigned int vsz) {
        unsigned int o = 0;
        ys = take(o, g.tv * tsz);
        cs = take(o, g.nq * g.tv * vsz);
        ds = take(o, g.tv * tsz);
        hs = take(o, 3u * g.fs * tsz);
        hent = take(o, g.ne * 4u);
        hwoff = take(o, (g.nd + 1) * 4u);
        mbar = take(o, 8u);
        flags = take(o, 16u);
        total = o;
    }
};

__device__ __forceinline__ unsigned int smem_addr(const void *p) {
    return static_cast<unsigned int>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ int ld_acquire_cta(const int *p) {
    int v;
    asm volatile("ld.acquire.cta.shared.u32 %0, [%1];" : "=r"(v) : "r"(smem_addr(p)) : "memory");
    return v;
}
__device__ __forceinline__ void st_release_cta(int *p, int v) {
    asm volatile("st.release.cta.shared.u32 [%0], %1;" ::"r"(smem_addr(p)), "r"(v) : "memory");
}
__device__ __forceinline__ void compute_barrier(int nc) {
    asm volatile("bar.sync 1, %0;" ::"r"(nc) : "memory");
}
__device__ __forceinline__ void mbar_init(unsigned int mbar) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(mbar) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
// One-dimensional bulk copy global -> shared through the tensor-memory-access
// engine, completing `bytes` transactions on the mbarrier.  Both addresses
// 16-byte aligned, bytes a multiple of 16.
__device__ __forceinline__ void bulk_g2s(unsigned int dst, const void *src, unsigned int bytes, unsigned int mbar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
                 ::"r"(dst), "l"(src), "r"(bytes), "r"(mbar) : "memory");
}
__device__ __forceinline__ bool mbar_wait(unsigned int mbar, unsigned int parity) {
    for (unsigned int spins = 0; spins < TILE_SPIN_LIMIT; ++spins) {
        unsigned int ok;
        asm volatile("{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
                     "selp.u32 %0, 1, 0, p;\n\t}"
                     : "=r"(ok) : "r"(mbar), "r"(parity) : "memory");
        if (ok) return true;
    }
    return false;
}

template <typename T, typename V>
struct TilePhaseD {
    const V *c;          // [ntiles][nq][tv] factor values, slot q = q-th consumed neighbour kind
    const T *d;          // [ntiles][tv] diagonal, or nullptr
    T *mb;               // this phase's mailboxes [ntiles][3][fs]
    T *mb_reset;         // the other phase's mailboxes, reset to the sentinel here
    const T *src;        // right-hand side (natural order)
    T *dst;              // solution (natural order)
    int src_coherent;    // src was written earlier in this launch: read it past L1
};

template <typename T, typename V>
struct TileArgs {
    TileGeom g;
    const unsigned int *hent;
    const int *hwoff;
    const int *torder;
    TilePhaseD<T, V> ph[2];
    unsigned int *bar;
    int *err;
};

// Shared-memory pointers of one block.
template <typename T, typename V>
struct TileShm {
    T *ys;                       // [tv] right-hand side, then solution, by local index
    V *cs;                       // [nq][tv] factor values by local index
    T *ds;                       // [tv] diagonal
    T *hs;                       // [3][fs] halo values (x, y, z faces)
    const unsigned int *hent;    // [ne]
    const int *hwoff;            // [nd + 1]
    int *hready;                 // wavefronts whose halo is complete
    int *abort;                  // a wait of this block gave up
    unsigned int mbar;           // completion of the factor-value copy
};

// Global row of step coordinates (i, j, k) in tile (I, J, K).
template <bool MIRROR>
__device__ __forceinline__ long long tile_row(const TileGeom &g, int I, int J, int K, int i, int j, int k) {
    const int gi = I * g.tx + (MIRROR ? g.tx - 1 - i : i);
    const int gj = J * g.ty + (MIRROR ? g.ty - 1 - j : j);
    const int gk = K * g.tz + (MIRROR ? g.tz - 1 - k : k);
    if (gi >= g.nx || gj >= g.ny || gk >= g.nz) return -1;
    return ((long long)gk * g.ny + gj) * g.nx + gi;
}

// The halo warp of one tile: polls the predecessors' mailboxes a window of
// entries ahead of the compute warps and publishes, in *hready, the number of
// wavefronts whose halo values are all in shared memory.  Returns false when
// its wait gave up or another block reported one.
template <typename T, typename V>
__device__ __forceinline__ bool halo_poll(const TileGeom &g, const TileShm<T, V> &S, const T *mbx, const T *mby,
                                          const T *mbz, int lox, int loy, int loz, int ex, int ey, int ez,
                                          int *err) {
    const int lane = threadIdx.x & 31;
    const int tx = g.tx, ty = g.ty, fs = g.fs, nd = g.nd, ne = g.ne;
    int lo = 0;
    unsigned int rounds = 0;
    while (lo < nd) {
        const int e0 = S.hwoff[lo];
        const int e1 = min(e0 + 32 * HALO_PER_LANE, ne);
        T v[HALO_PER_LANE];
        int slot[HALO_PER_LANE], wv[HALO_PER_LANE];
#pragma unroll
        for (int q = 0; q < HALO_PER_LANE; ++q) {
            const int e = e0 + lane + 32 * q;
            slot[q] = -1;
            wv[q] = 0;
            v[q] = T(0);
            if (e >= e1) continue;
            const unsigned int h = S.hent[e];
            const int f = (int)(h & 3u), w = (int)((h >> 2) & 1023u);
            const int a = (int)((h >> 12) & 1023u), b = (int)(h >> 22);
            const T *src;
            bool need;
            int fi;
            if (f == 0) {        // x face: row (0, a, b)
                need = mbx && a >= loy && a < loy + ey && b >= loz && b < loz + ez;
                fi = b * ty + a;
                src = mbx;
            } else if (f == 1) { // y face: row (a, 0, b)
                need = mby && a >= lox && a < lox + ex && b >= loz && b < loz + ez;
                fi = b * tx + a;
                src = mby;
            } else {             // z face: row (a, b, 0)
                need = mbz && a >= lox && a < lox + ex && b >= loy && b < loy + ey;
                fi = b * tx + a;
                src = mbz;
            }
            if (need) {
                v[q] = Sentinel<T>::ld(src + fi);
                slot[q] = f * fs + fi;
                wv[q] = w;
            }
        }
        int miss = INT_MAX;
#pragma unroll
        for (int q = 0; q < HALO_PER_LANE; ++q) {
            if (slot[q] < 0) continue;
            if (Sentinel<T>::is(v[q])) miss = min(miss, wv[q]);
            else S.hs[slot[q]] = v[q];
        }
        miss = __reduce_min_sync(0xffffffffu, miss);
        int nlo = e1 < ne ? (int)((S.hent[e1] >> 2) & 1023u) : nd;
        nlo = min(nlo, miss);
        if (nlo > lo) {
            __threadfence_block();
            __syncwarp();
            if (lane == 0) st_release_cta(S.hready, nlo);
            lo = nlo;
            rounds = 0;
        } else {
            ++rounds;
            if (TILE_SLEEP_NS > 0) __nanosleep(TILE_SLEEP_NS);
            bool quit = rounds > TILE_SPIN_LIMIT;
            if (quit && lane == 0) atomicExch(err, 1);
            if ((rounds & 255u) == 0 && *(volatile int *)err) quit = true;
            if (__any_sync(0xffffffffu, quit)) {
                if (lane == 0) { *S.abort = 1; st_release_cta(S.hready, INT_MAX); }
                return false;
            }
        }
    }
    return true;
}

// Compile-time tile shape of a 2D or 3D plan.
template <int DIM> struct TileShape {
    static constexpr int TX = DIM == 3 ? 16 : 64, TY = TX, TZ = DIM == 3 ? 16 : 1;
    static constexpr int LX = DIM == 3 ? 4 : 6, LY = LX;
    static constexpr int TV = TX * TY * TZ;                 // rows per tile
    static constexpr int ND = TX + TY + TZ - 2;             // steps per tile
    static constexpr int NC = TY * TZ;                      // compute threads: one per grid line
    static constexpr int FS = DIM == 3 ? TX * TY : TX;      // mailbox face stride
};

// One phase (MIRROR false: forward solve, lower neighbours consumed z, y, x;
// true: backward solve in reversed step coordinates, upper neighbours
// consumed x, y, z).  Step coordinates (i, j, k) of a row: its local
// coordinates in the tile, each reversed when MIRROR.  HAS_D: the factor
// has a diagonal to divide by.  Returns false when a wait gave up.
template <typename T, typename V, int DIM, bool MIRROR, bool HAS_D>
__device__ __forceinline__ bool tile_phase(const TileGeom &g, const TilePhaseD<T, V> &P, const int *torder,
                                           int *err, const TileShm<T, V> &S, unsigned int &parity) {
    using Sh = TileShape<DIM>;
    constexpr int TX = Sh::TX, TY = Sh::TY, TZ = Sh::TZ, TV = Sh::TV, ND = Sh::ND, NC = Sh::NC, FS = Sh::FS;
    constexpr int LX = Sh::LX, LXY = Sh::LX + Sh::LY;
    const bool halo = (int)threadIdx.x >= NC;
    const V *const pc = P.c;
    const T *const pd = P.d;
    T *const pmb = P.mb;
    const T *const src = P.src;
    T *const dst = P.dst;
    const bool coherent = P.src_coherent != 0;
    T *const ys = S.ys;
    const V *const cs = S.cs;
    const T *const ds = S.ds;
    const T *const hs = S.hs;
    {   // the other phase's mailboxes back to the sentinel
        T *const reset = P.mb_reset;
        const size_t nmb = (size_t)g.ntiles * 3 * FS;
        for (size_t q = (size_t)blockIdx.x * blockDim.x + threadIdx.x; q < nmb; q += (size_t)gridDim.x * blockDim.x)
            reset[q] = Sentinel<T>::value();
    }
    // this thread's grid line
    const int j = threadIdx.x % TY, k = threadIdx.x / TY;
    for (int u = blockIdx.x; u < g.ntiles; u += gridDim.x) {
        const int tile = torder[MIRROR ? g.ntiles - 1 - u : u];
        const int I = tile % g.ntx, J = (tile / g.ntx) % g.nty, K = tile / (g.ntx * g.nty);
        const int ex = min(TX, g.nx - I * TX), ey = min(TY, g.ny - J * TY), ez = min(TZ, g.nz - K * TZ);
        // rows exist at step coordinates [lo, lo + e) per axis
        const int lox = MIRROR ? TX - ex : 0, loy = MIRROR ? TY - ey : 0, loz = MIRROR ? TZ - ez : 0;
        // the tile before (predecessor) and after (successor) along each axis in step order
        const bool px = MIRROR ? I < g.ntx - 1 : I > 0, sx = MIRROR ? I > 0 : I < g.ntx - 1;
        const bool py = MIRROR ? J < g.nty - 1 : J > 0, sy = MIRROR ? J > 0 : J < g.nty - 1;
        const bool pz = MIRROR ? K < g.ntz - 1 : K > 0, sz = MIRROR ? K > 0 : K < g.ntz - 1;
        const int step = MIRROR ? 1 : -1;

        __syncthreads();   // the previous tile's shared data is no longer read
        if (threadIdx.x == 0) {
            constexpr unsigned int cb = (unsigned int)(DIM * TV * sizeof(V));
            constexpr unsigned int db = HAS_D ? (unsigned int)(TV * sizeof(T)) : 0u;
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(S.mbar), "r"(cb + db)
                         : "memory");
            bulk_g2s(smem_addr(cs), pc + (size_t)tile * DIM * TV, cb, S.mbar);
            if (HAS_D) bulk_g2s(smem_addr(ds), pd + (size_t)tile * TV, db, S.mbar);
            *S.hready = 0;
        }
        if (!halo) {   // stage the right-hand side, STAGE_BATCH loads in flight per thread
#pragma unroll 1
            for (int base = threadIdx.x; base < TV; base += NC * STAGE_BATCH) {
                T v[STAGE_BATCH];
#pragma unroll
                for (int q = 0; q < STAGE_BATCH; ++q) {
                    const int lex = base + q * NC;
                    const long long r = lex < TV ? tile_row<MIRROR>(g, I, J, K, lex & (TX - 1),
                                                                   (lex >> LX) & (TY - 1), lex >> LXY) : -1;
                    v[q] = r >= 0 ? (coherent ? __ldcg(src + r) : src[r]) : T(0);
                }
#pragma unroll
                for (int q = 0; q < STAGE_BATCH; ++q)
                    if (base + q * NC < TV) ys[base + q * NC] = v[q];
            }
        }
        __syncthreads();

        if (halo) {
            const T *mbx = px ? pmb + ((size_t)(tile + step) * 3 + 0) * FS : nullptr;
            const T *mby = py ? pmb + ((size_t)(tile + step * g.ntx) * 3 + 1) * FS : nullptr;
            const T *mbz = pz ? pmb + ((size_t)(tile + step * g.ntx * g.nty) * 3 + 2) * FS : nullptr;
            halo_poll<T, V>(g, S, mbx, mby, mbz, lox, loy, loz, ex, ey, ez, err);
        } else {
            if (!mbar_wait(S.mbar, parity)) { atomicExch(err, 1); *S.abort = 1; }
            // the line's rows: steps [dlo, dlo + len), row i = d - d0
            const bool line = j >= loy && j < loy + ey && k >= loz && k < loz + ez;
            const int d0 = j + k, dlo = d0 + lox, len = line ? ex : 0;
            const int base = (k * TY + j) * TX;               // local index of row (0, j, k)
            // neighbours in the tile or in the halo (y, z: the same for all the line's rows)
            const bool yin = j > loy, zin = DIM == 3 && k > loz;
            const bool uy = yin || py, uz = DIM == 3 && (zin || pz);
            const bool hy = !yin && py, hz = DIM == 3 && !zin && pz;
            // this tile's mailboxes the line writes to
            T *const mbt = pmb + (size_t)tile * 3 * FS;
            T *const mbx_out = sx ? mbt + k * TY + j : nullptr;                         // at i == TX - 1
            T *const mby_out = (sy && j == TY - 1) ? mbt + FS + k * TX : nullptr;        // + i
            T *const mbz_out = (DIM == 3 && sz && k == TZ - 1) ? mbt + 2 * FS + j * TX : nullptr;   // + i
            // the first row's right-hand side and factor values
            T rhs = T(0), c0 = T(0), c1 = T(0), c2 = T(0), dg = T(1);
            if (len > 0) {
                const int lex = base + lox;
                rhs = ys[lex];
                c0 = val_as<T, V>(cs[lex]);
                c1 = val_as<T, V>(cs[TV + lex]);
                if (DIM == 3) c2 = val_as<T, V>(cs[2 * TV + lex]);
                if (HAS_D) dg = ds[lex];
            }
            T prev = T(0);
            int hr = 0;
#pragma unroll 1
            for (int d = 0; d < ND; ++d) {
                if ((unsigned int)(d - dlo) < (unsigned int)len) {
                    const int i = d - d0;
                    const int lex = base + i;
                    const bool first = i == lox;
                    const bool hx = first && px, ux = !first || px;
                    T nbx = prev;
                    T nby = yin ? ys[lex - TX] : T(0);
                    T nbz = zin ? ys[lex - TX * TY] : T(0);
                    if (hx || hy || hz) {
                        if (hr <= d) {
                            unsigned int spins = 0;
                            while ((hr = ld_acquire_cta(S.hready)) <= d) {
                                if (++spins > TILE_SPIN_LIMIT) { atomicExch(err, 1); hr = INT_MAX; break; }
                                if (TILE_SLEEP_NS > 0) __nanosleep(TILE_SLEEP_NS / 4);
                            }
                        }
                        if (hx) nbx = hs[k * TY + j];
                        if (hy) nby = hs[FS + k * TX + i];
                        if (hz) nbz = hs[2 * FS + j * TX + i];
                    }
                    T acc = rhs;
                    if (MIRROR) {                 // stored order x, y, z
                        if (ux) acc = msub(acc, c0, nbx);
                        if (uy) acc = msub(acc, c1, nby);
                        if (uz) acc = msub(acc, c2, nbz);
                    } else if (DIM == 3) {        // stored order z, y, x
                        if (uz) acc = msub(acc, c0, nbz);
                        if (uy) acc = msub(acc, c1, nby);
                        if (ux) acc = msub(acc, c2, nbx);
                    } else {                      // 2D: y, x
                        if (uy) acc = msub(acc, c0, nby);
                        if (ux) acc = msub(acc, c1, nbx);
                    }
                    if (HAS_D) acc = acc / dg;
                    ys[lex] = acc;
                    prev = acc;
                    if (mbx_out && i == TX - 1) Sentinel<T>::st(mbx_out, acc);
                    if (mby_out) Sentinel<T>::st(mby_out + i, acc);
                    if (mbz_out) Sentinel<T>::st(mbz_out + i, acc);
                    // the next row's right-hand side and factor values (not
                    // written by this or the next step)
                    if (d + 1 - dlo < len) {
                        rhs = ys[lex + 1];
                        c0 = val_as<T, V>(cs[lex + 1]);
                        c1 = val_as<T, V>(cs[TV + lex + 1]);
                        if (DIM == 3) c2 = val_as<T, V>(cs[2 * TV + lex + 1]);
                        if (HAS_D) dg = ds[lex + 1];
                    }
                }
                compute_barrier(NC);
            }
        }
        parity ^= 1u;
        __syncthreads();
        if (!halo) {   // the tile's solution
#pragma unroll 4
            for (int lex = threadIdx.x; lex < TV; lex += NC) {
                const long long r = tile_row<MIRROR>(g, I, J, K, lex & (TX - 1), (lex >> LX) & (TY - 1), lex >> LXY);
                if (r >= 0) dst[r] = ys[lex];
            }
        }
        if (threadIdx.x == 0 && *(volatile int *)err) *S.abort = 1;
        __syncthreads();
        if (*(volatile int *)S.abort) return false;
    }
    return true;
}

template <typename T, typename V, int DIM, bool MIRROR>
__device__ __forceinline__ bool tile_phase_d(const TileGeom &g, const TilePhaseD<T, V> &P, const int *torder,
                                             int *err, const TileShm<T, V> &S, unsigned int &parity) {
    if (P.d) return tile_phase<T, V, DIM, MIRROR, true>(g, P, torder, err, S, parity);
    return tile_phase<T, V, DIM, MIRROR, false>(g, P, torder, err, S, parity);
}

template <typename T, typename V, int DIM>
__global__ void __launch_bounds__(TILE_MAX_THREADS) k_sweep_tiles(const __grid_constant__ TileArgs<T, V> A) {
    extern __shared__ __align__(128) unsigned char sm[];
    const TileGeom g = A.g;
    const TileSmem L(g, sizeof(T), sizeof(V));
    TileShm<T, V> S;
    S.ys = reinterpret_cast<T *>(sm + L.ys);
    S.cs = reinterpret_cast<V *>(sm + L.cs);
    S.ds = reinterpret_cast<T *>(sm + L.ds);
    S.hs = reinterpret_cast<T *>(sm + L.hs);
    unsigned int *he = reinterpret_cast<unsigned int *>(sm + L.hent);
    int *hw = reinterpret_cast<int *>(sm + L.hwoff);
    S.hent = he;
    S.hwoff = hw;
    S.hready = reinterpret_cast<int *>(sm + L.flags);
    S.abort = S.hready + 1;
    S.mbar = smem_addr(sm + L.mbar);
    for (int q = threadIdx.x; q <= g.nd; q += blockDim.x) hw[q] = A.hwoff[q];
    for (int q = threadIdx.x; q < g.ne; q += blockDim.x) he[q] = A.hent[q];
    if (threadIdx.x == 0) {
        mbar_init(S.mbar);
        *S.abort = 0;
    }
    __syncthreads();
    unsigned int parity = 0;
    if (!tile_phase_d<T, V, DIM, false>(g, A.ph[0], A.torder, A.err, S, parity)) return;   // *err set
    grid_barrier(A.bar, A.err);
    if (threadIdx.x == 0 && *(volatile int *)A.err) *S.abort = 1;
    __syncthreads();
    if (*(volatile int *)S.abort) return;
    tile_phase_d<T, V, DIM, true>(g, A.ph[1], A.torder, A.err, S, parity);
}

// ---------------------------------------------------------------- setup
// Offsets r - c of the lower entries: the smallest one above 1 and the
// largest, per block then one atomic each.
__global__ void k_grid_offsets(int n, const int *rp, const int *ci, int *mn, int *mx) {
    __shared__ int bmn, bmx;
    if (threadIdx.x == 0) { bmn = INT_MAX; bmx = 0; }
    __syncthreads();
    int lmn = INT_MAX, lmx = 0;
    for (int r = blockIdx.x * blockDim.x + threadIdx.x; r < n; r += gridDim.x * blockDim.x)
        for (int e = rp[r]; e < rp[r + 1]; ++e) {
            const int off = r - ci[e];
            if (off > 1) { lmn = min(lmn, off); lmx = max(lmx, off); }
        }
    lmn = __reduce_min_sync(0xffffffffu, lmn);
    lmx = __reduce_max_sync(0xffffffffu, lmx);
    if ((threadIdx.x & 31) == 0) { atomicMin(&bmn, lmn); atomicMax(&bmx, lmx); }
    __syncthreads();
    if (threadIdx.x == 0) { atomicMin(mn, bmn); atomicMax(mx, bmx); }
}

// Factor values of one triangular solve into tile layout (by local index in
// step coordinates); every row's stored entries must be exactly its stencil
// neighbours in ascending column order, else *bad is set.
template <typename T, typename V>
__global__ void k_tile_factor(TileGeom g, int mirror, int n, const int *rows, const int *rp, const int *ci,
                              const V *v, const T *d, V *c, T *dg, int *bad) {
    const int nx = g.nx, ny = g.ny, nz = g.nz;
    const long long nxy = (long long)nx * ny;
    for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < n; p += gridDim.x * blockDim.x) {
        const int r = rows[p];
        const int gi = r % nx, gj = (r / nx) % ny, gk = (int)(r / nxy);
        const int I = gi / g.tx, J = gj / g.ty, K = gk / g.tz;
        int i = gi - I * g.tx, j = gj - J * g.ty, k = gk - K * g.tz;
        if (mirror) { i = g.tx - 1 - i; j = g.ty - 1 - j; k = g.tz - 1 - k; }
        const long long tile = ((long long)K * g.nty + J) * g.ntx + I;
        const int lex = (k * g.ty + j) * g.tx + i;
        int e = rp[p];
        const int e1 = rp[p + 1];
        bool ok = true;
        for (int q = 0; q < g.nq && ok; ++q) {
            const int kind = mirror ? q : g.nq - 1 - q;
            bool has;
            long long col;
            if (kind == 0) { has = mirror ? gi < nx - 1 : gi > 0; col = mirror ? r + 1LL : r - 1LL; }
            else if (kind == 1) { has = mirror ? gj < ny - 1 : gj > 0; col = mirror ? r + (long long)nx : r - (long long)nx; }
            else { has = mirror ? gk < nz - 1 : gk > 0; col = mirror ? r + nxy : r - nxy; }
            if (!has) continue;
            if (e >= e1 || ci[e] != col) { ok = false; break; }
            c[(tile * g.nq + q) * g.tv + lex] = v[e];
            ++e;
        }
        if (!ok || e != e1) atomicExch(bad, 1);
        if (d) dg[tile * g.tv + lex] = d[p];
    }
}

template <typename T>
void fill_sentinel_bytes(DBuf<char> &b, cudaStream_t s) {
    fill_sentinel<T>(reinterpret_cast<T *>(b.get()), b.n / sizeof(T), s);
}

int tile_threads(const TileGeom &g) { return g.ty * g.tz + 32; }

template <typename T, typename V>
const void *tile_kernel(int dim) {
    return dim == 3 ? (const void *)k_sweep_tiles<T, V, 3> : (const void *)k_sweep_tiles<T, V, 2>;
}

}  // namespace

bool tile_plan_build(const DCsr &A, TilePlan &P, size_t tsz, size_t vsz, cudaStream_t s) {
    const int n = A.n;
    if (n < 4) return false;
    DBuf<int> mm(2);
    const int init[2] = {INT_MAX, 0};
    CU(cudaMemcpyAsync(mm.get(), init, sizeof(init), cudaMemcpyHostToDevice, s));
    k_grid_offsets<<<grid_for((size_t)n, 256), 256, 0, s>>>(n, A.rp.get(), A.ci.get(), mm.get(), mm.get() + 1);
    CU_LAUNCH("k_grid_offsets"); count_launch();
    int hm[2];
    CU(cudaMemcpyAsync(hm, mm.get(), sizeof(hm), cudaMemcpyDeviceToHost, s));
    CU(cudaStreamSynchronize(s));
    if (hm[0] == INT_MAX) return false;
    TileGeom g{};
    g.nx = hm[0];
    if (hm[1] == hm[0]) {
        if (n % g.nx) return false;
        g.dim = 2; g.ny = n / g.nx; g.nz = 1;
        g.tx = 64; g.ty = 64; g.tz = 1; g.lx = 6; g.ly = 6; g.nq = 2;
    } else {
        const int nxy = hm[1];
        if (nxy % g.nx || n % nxy) return false;
        g.dim = 3; g.ny = nxy / g.nx; g.nz = n / nxy;
        g.tx = 16; g.ty = 16; g.tz = 16; g.lx = 4; g.ly = 4; g.nq = 3;
        if (g.nz < 2) return false;
    }
    if (g.nx < 2 || g.ny < 2) return false;
    g.ntx = (g.nx + g.tx - 1) / g.tx;
    g.nty = (g.ny + g.ty - 1) / g.ty;
    g.ntz = (g.nz + g.tz - 1) / g.tz;
    g.ntiles = g.ntx * g.nty * g.ntz;
    g.tv = g.tx * g.ty * g.tz;
    g.nd = g.tx + g.ty + g.tz - 2;
    g.fs = std::max(g.ty * g.tz, std::max(g.tx * g.tz, g.dim == 3 ? g.tx * g.ty : 0));
    // halo entries (face, step of the consuming row, face coordinates) by step
    std::vector<std::pair<int, unsigned int>> he;
    auto add = [&](int f, int w, int a, int b) {
        he.push_back({w, (unsigned int)f | ((unsigned int)w << 2) | ((unsigned int)a << 12) | ((unsigned int)b << 22)});
    };
    for (int k = 0; k < g.tz; ++k)
        for (int j = 0; j < g.ty; ++j) add(0, j + k, j, k);
    for (int k = 0; k < g.tz; ++k)
        for (int i = 0; i < g.tx; ++i) add(1, i + k, i, k);
    if (g.dim == 3)
        for (int j = 0; j < g.ty; ++j)
            for (int i = 0; i < g.tx; ++i) add(2, i + j, i, j);
    std::stable_sort(he.begin(), he.end(), [](const auto &a, const auto &b) { return a.first < b.first; });
    g.ne = (int)he.size();
    std::vector<unsigned int> hent(g.ne);
    std::vector<int> hwoff(g.nd + 1, g.ne);
    for (int e = g.ne - 1; e >= 0; --e) {
        hent[e] = he[e].second;
        hwoff[he[e].first] = e;
    }
    for (int w = g.nd - 1; w >= 0; --w) hwoff[w] = std::min(hwoff[w], hwoff[w + 1]);
    // tiles by anti-diagonal
    std::vector<int> torder(g.ntiles);
    for (int t = 0; t < g.ntiles; ++t) torder[t] = t;
    auto diag = [&](int t) { return t % g.ntx + (t / g.ntx) % g.nty + t / (g.ntx * g.nty); };
    std::stable_sort(torder.begin(), torder.end(), [&](int a, int b) { return diag(a) < diag(b); });
    const TileSmem L(g, (unsigned int)tsz, (unsigned int)vsz);
    if (L.total > 227u * 1024u) return false;
    // the kernel's compile-time shapes
    if (g.dim == 3 && (g.fs != TileShape<3>::FS || g.tv != TileShape<3>::TV || g.nd != TileShape<3>::ND)) return false;
    if (g.dim == 2 && (g.fs != TileShape<2>::FS || g.tv != TileShape<2>::TV || g.nd != TileShape<2>::ND)) return false;

    P.g = g;
    P.tsz = tsz;
    P.vsz = vsz;
    P.hent.alloc(g.ne); P.hwoff.alloc(g.nd + 1); P.torder.alloc(g.ntiles);
    CU(cudaMemcpyAsync(P.hent.get(), hent.data(), hent.size() * 4, cudaMemcpyHostToDevice, s));
    CU(cudaMemcpyAsync(P.hwoff.get(), hwoff.data(), hwoff.size() * 4, cudaMemcpyHostToDevice, s));
    CU(cudaMemcpyAsync(P.torder.get(), torder.data(), torder.size() * 4, cudaMemcpyHostToDevice, s));
    for (int q = 0; q < 2; ++q) P.mb[q].alloc((size_t)g.ntiles * 3 * g.fs * tsz);
    tile_mailbox_reset(P, s);
    CU(cudaStreamSynchronize(s));   // the host tables above are freed on return
    return true;
}

void tile_mailbox_reset(TilePlan &P, cudaStream_t s) {
    for (int q = 0; q < 2; ++q) {
        if (P.tsz == sizeof(double)) fill_sentinel_bytes<double>(P.mb[q], s);
        else fill_sentinel_bytes<float>(P.mb[q], s);
    }
}

template <typename T, typename V>
bool tile_factor_build(const TilePlan &P, const SweepView<T, V> &S, bool mirror, TileFactor &F, cudaStream_t s) {
    const TileGeom &g = P.g;
    const int n = g.nx * g.ny * g.nz;
    if (S.lev_ptr[S.nlev] != n) return false;
    const size_t nv = (size_t)g.ntiles * g.nq * g.tv;
    F.c.alloc(nv * sizeof(V));
    CU(cudaMemsetAsync(F.c.get(), 0, F.c.bytes(), s));
    if (S.d) {
        F.d.alloc((size_t)g.ntiles * g.tv * sizeof(T));
        CU(cudaMemsetAsync(F.d.get(), 0, F.d.bytes(), s));
    } else {
        F.d.release();
    }
    DBuf<int> bad(1);
    CU(cudaMemsetAsync(bad.get(), 0, sizeof(int), s));
    k_tile_factor<T, V><<<grid_for((size_t)n, 256), 256, 0, s>>>(
        g, mirror ? 1 : 0, n, S.rows, S.rp, S.ci, S.v, S.d, reinterpret_cast<V *>(F.c.get()),
        S.d ? reinterpret_cast<T *>(F.d.get()) : nullptr, bad.get());
    CU_LAUNCH("k_tile_factor"); count_launch();
    int hbad = 0;
    CU(cudaMemcpyAsync(&hbad, bad.get(), sizeof(int), cudaMemcpyDeviceToHost, s));
    CU(cudaStreamSynchronize(s));
    return hbad == 0;
}

template <typename T, typename V>
void tile_prepare(TilePlan &P) {
    const TileGeom &g = P.g;
    const TileSmem L(g, sizeof(T), sizeof(V));
    static const int smem_max = [] {   // once per instantiation: allow the largest layout
        int dev = 0, optin = 0;
        CU(cudaGetDevice(&dev));
        CU(cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
        for (int dim = 2; dim <= 3; ++dim)
            CU(cudaFuncSetAttribute(tile_kernel<T, V>(dim), cudaFuncAttributeMaxDynamicSharedMemorySize, optin));
        return optin;
    }();
    if ((int)L.total > smem_max) fail(AMG_ERR_NOT_SUPPORTED, "tile sweep: shared memory layout too large");
    int occ = 0;
    CU(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, tile_kernel<T, V>(g.dim), tile_threads(g), L.total));
    if (occ < 1) fail(AMG_ERR_NOT_SUPPORTED, "tile sweep: no block fits an SM");
    if (TILE_BLOCKS_PER_SM > 0) occ = std::min(occ, TILE_BLOCKS_PER_SM);
    P.blocks = std::min(g.ntiles, sm_count() * occ);
}

template <typename T, typename V>
void sweep_pair_tiles(const TilePlan &P, const TileFactor &F, const TileFactor &B, const T *in, T *y, T *out,
                      unsigned int *bar, int *err, cudaStream_t s) {
    const TileGeom &g = P.g;
    const TileSmem L(g, sizeof(T), sizeof(V));
    TileArgs<T, V> A;
    A.g = g;
    A.hent = P.hent.get();
    A.hwoff = P.hwoff.get();
    A.torder = P.torder.get();
    T *mb0 = reinterpret_cast<T *>(P.mb[0].get()), *mb1 = reinterpret_cast<T *>(P.mb[1].get());
    A.ph[0] = TilePhaseD<T, V>{reinterpret_cast<const V *>(F.c.get()),
                               F.d.n ? reinterpret_cast<const T *>(F.d.get()) : nullptr, mb0, mb1, in, y, 0};
    A.ph[1] = TilePhaseD<T, V>{reinterpret_cast<const V *>(B.c.get()),
                               B.d.n ? reinterpret_cast<const T *>(B.d.get()) : nullptr, mb1, mb0, y, out, 1};
    A.bar = bar;
    A.err = err;
    void *args[] = {&A};
    CU(cudaLaunchCooperativeKernel(tile_kernel<T, V>(g.dim), dim3(P.blocks), dim3(tile_threads(g)), args, L.total, s));
    count_launch();
}

template void tile_prepare<double, double>(TilePlan &);
template void tile_prepare<float, float>(TilePlan &);
template void tile_prepare<float, __nv_bfloat16>(TilePlan &);
template bool tile_factor_build<double, double>(const TilePlan &, const SweepView<double, double> &, bool,
                                                TileFactor &, cudaStream_t);
template bool tile_factor_build<float, float>(const TilePlan &, const SweepView<float, float> &, bool, TileFactor &,
                                              cudaStream_t);
template bool tile_factor_build<float, __nv_bfloat16>(const TilePlan &, const SweepView<float, __nv_bfloat16> &,
                                                      bool, TileFactor &, cudaStream_t);
template void sweep_pair_tiles<double, double>(const TilePlan &, const TileFactor &, const TileFactor &,
                                               const double *, double *, double *, unsigned int *, int *,
                                               cudaStream_t);
template void sweep_pair_tiles<float, float>(const TilePlan &, const TileFactor &, const TileFactor &, const float *,
                                             float *, float *, unsigned int *, int *, cudaStream_t);
template void sweep_pair_tiles<float, __nv_bfloat16>(const TilePlan &, const TileFactor &, const TileFactor &,
                                                     const float *, float *, float *, unsigned int *, int *,
                                                     cudaStream_t);

}  // namespace amg
