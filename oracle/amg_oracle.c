/*
 * amg_oracle.c -- plain, slow, single-threaded FP64 reference of the
 * matching-aggregation two-grid AMG preconditioner inside FGMRES.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite, the package's smoke check
 * and the benchmark's CPU-baseline leg may load this library.  It shares no
 * source with the CUDA implementation: every formula below is restated here
 * from the paper (P. Kumar, "Aggregation based on graph matching and inexact
 * coarse grid solve for algebraic multigrid", arXiv:1105.3468) and from the
 * readings listed with each function.
 *
 * Compiled with -O2 -ffp-contract=off, so an expression a*b+c rounds twice,
 * as written.  Rounding of multiply-accumulate (the paper does not fix it):
 * the setup (assembly, gradient, ILU(0) factorisation, the pivot-row
 * division of the dense inverse) rounds each product and each sum, except
 * the elimination update of the dense inverse, one fused multiply-add;
 * the solve phase (matrix-vector
 * products, triangular solves, the dense product, dot products, vector
 * updates, Givens rotations, back substitution) accumulates with fma(),
 * IEEE 754 fused multiply-add with a single rounding.
 *
 * Status codes (same numeric meaning as the library's public header, defined
 * independently here):
 *   0 ok, 1 invalid argument, 5 breakdown (zero/non-finite pivot),
 *   6 numeric (NaN/Inf residual), 7 not converged, 8 limit reached.
 *
 * Parity pins: every function here is pinned by tests under tests/ against
 * closed forms, brute force or the paper's worked example (see the test
 * module docstrings).  Nothing here is "parity unpinned".
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define OR_OK 0
#define OR_EINVAL 1
#define OR_EBREAKDOWN 5
#define OR_ENUMERIC 6
#define OR_ENOTCONV 7
#define OR_ELIMIT 8

/* ------------------------------------------------------------------ */
/* SplitMix64 output finaliser (Steele, Lea, Flood, OOPSLA 2014).       */
/* A bijection on 64-bit words; used only as a deterministic tie-break  */
/* key, which the paper does not specify (reading: hashed tie-break).   */
/* ------------------------------------------------------------------ */
uint64_t or_mix64(uint64_t z)
{
    z = (z ^ (z >> 30)) * UINT64_C(0xbf58476d1ce4e5b9);
    z = (z ^ (z >> 27)) * UINT64_C(0x94d049bb133111eb);
    return z ^ (z >> 31);
}

#define OR_COLOR_SALT UINT64_C(0x9e3779b97f4a7c15)

/* ------------------------------------------------------------------ */
/* O1. Cell-centred finite-volume discretisation of eq. (2):            */
/*   div(a u) - div(kappa grad u) = f,  u = 0 on y = 0, 1 (Dirichlet),  */
/*   du/dn = 0 elsewhere (Neumann).  Section 1 of the paper names the    */
/*   scheme only ("cell centered finite volume"); the reading used:      */
/*   two-point diffusive flux with the harmonic mean of the face-normal  */
/*   conductivities, first-order upwind convection, Dirichlet value at   */
/*   the face (half-cell distance), zero-gradient ghost on Neumann       */
/*   faces.  Faces are visited W, E, S, N, B, T; the diagonal adds the   */
/*   diffusive then the convective part of each face in that order.      */
/* Returns nnz (>= 0) or -OR_EINVAL.  Output arrays: row_ptr[n+1],      */
/* col/val with room for (2*dim+1)*n entries, b[n].                     */
/* ------------------------------------------------------------------ */
int64_t or_fv_assemble(int dim, int nx, int ny, int nz,
                       const double *kx, const double *ky, const double *kz,
                       const double *fx, const double *fy, const double *fz,
                       const double *f,
                       int64_t *row_ptr, int32_t *col, double *val, double *b)
{
    if ((dim != 2 && dim != 3) || nx <= 0 || ny <= 0 || nz <= 0) return -OR_EINVAL;
    if (dim == 2 && nz != 1) return -OR_EINVAL;
    const double h = 1.0 / (double)nx;
    const double hd2 = (dim == 2) ? 1.0 : h;            /* h^(d-2) */
    const double hd = (dim == 2) ? h * h : h * h * h;   /* h^d */
    const int64_t sxy = (int64_t)nx * ny;
    int64_t nnz = 0;
    row_ptr[0] = 0;
    for (int k = 0; k < nz; ++k)
        for (int j = 0; j < ny; ++j)
            for (int i = 0; i < nx; ++i) {
                const int64_t P = i + (int64_t)nx * (j + (int64_t)ny * k);
                /* face data in W, E, S, N, B, T order */
                int nfaces = (dim == 2) ? 4 : 6;
                int64_t nb[6];
                int kind[6];        /* 0 interior, 1 Dirichlet, 2 Neumann */
                double kP[6], kN[6], F[6];
                /* W */
                nb[0] = P - 1; kind[0] = (i == 0) ? 2 : 0;
                kP[0] = kx[P]; kN[0] = (i == 0) ? 0.0 : kx[P - 1];
                F[0] = -fx[i + (int64_t)(nx + 1) * (j + (int64_t)ny * k)];
                /* E */
                nb[1] = P + 1; kind[1] = (i == nx - 1) ? 2 : 0;
                kP[1] = kx[P]; kN[1] = (i == nx - 1) ? 0.0 : kx[P + 1];
                F[1] = fx[(i + 1) + (int64_t)(nx + 1) * (j + (int64_t)ny * k)];
                /* S */
                nb[2] = P - nx; kind[2] = (j == 0) ? 1 : 0;
                kP[2] = ky[P]; kN[2] = (j == 0) ? 0.0 : ky[P - nx];
                F[2] = -fy[i + (int64_t)nx * (j + (int64_t)(ny + 1) * k)];
                /* N */
                nb[3] = P + nx; kind[3] = (j == ny - 1) ? 1 : 0;
                kP[3] = ky[P]; kN[3] = (j == ny - 1) ? 0.0 : ky[P + nx];
                F[3] = fy[i + (int64_t)nx * ((j + 1) + (int64_t)(ny + 1) * k)];
                if (dim == 3) {
                    /* B */
                    nb[4] = P - sxy; kind[4] = (k == 0) ? 2 : 0;
                    kP[4] = kz[P]; kN[4] = (k == 0) ? 0.0 : kz[P - sxy];
                    F[4] = -fz[i + (int64_t)nx * (j + (int64_t)ny * k)];
                    /* T */
                    nb[5] = P + sxy; kind[5] = (k == nz - 1) ? 2 : 0;
                    kP[5] = kz[P]; kN[5] = (k == nz - 1) ? 0.0 : kz[P + sxy];
                    F[5] = fz[i + (int64_t)nx * (j + (int64_t)ny * (k + 1))];
                }
                double diag = 0.0;
                double off[6];
                for (int q = 0; q < nfaces; ++q) {
                    off[q] = 0.0;
                    if (kind[q] == 0) {
                        double T = hd2 * ((2.0 * kP[q] * kN[q]) / (kP[q] + kN[q]));
                        diag += T;
                        if (F[q] > 0.0) diag += F[q];
                        off[q] = -T;
                        if (F[q] < 0.0) off[q] = off[q] + F[q];
                    } else if (kind[q] == 1) {
                        double T = hd2 * (2.0 * kP[q]);
                        diag += T;
                        if (F[q] > 0.0) diag += F[q];
                    } else {
                        diag += F[q];
                    }
                }
                /* emit in ascending column order: B, S, W, P, E, N, T */
                static const int order3[7] = {4, 2, 0, -1, 1, 3, 5};
                static const int order2[5] = {2, 0, -1, 1, 3};
                const int *ord = (dim == 3) ? order3 : order2;
                int nord = (dim == 3) ? 7 : 5;
                for (int t = 0; t < nord; ++t) {
                    int q = ord[t];
                    if (q < 0) {
                        col[nnz] = (int32_t)P; val[nnz] = diag; ++nnz;
                    } else if (kind[q] == 0) {
                        col[nnz] = (int32_t)nb[q]; val[nnz] = off[q]; ++nnz;
                    }
                }
                row_ptr[P + 1] = nnz;
                b[P] = f[P] * hd;
            }
    return nnz;
}

/* Gradient of a scalar loss with respect to per-cell log-conductivities,
 * given the adjoint lambda (A^T lambda = dL/dx) and the solution x.
 * dL/dA_ij = -lambda_i x_j on the pattern (implicit function theorem on
 * A x = b).  Only the diffusive transmissibilities depend on kappa:
 *   interior face P|N, T = hd2*2 kP kN/(kP+kN):
 *       dL/dT = -(lambda_P - lambda_N)(x_P - x_N),
 *       dT/dlog kP = T kN/(kP+kN);
 *   Dirichlet face, T = hd2*2 kP: dL/dT = -lambda_P x_P, dT/dlog kP = T.
 * Outputs gx, gy, gz: derivative with respect to log of kx, ky, kz. */
int or_fv_grad_logk(int dim, int nx, int ny, int nz,
                    const double *kx, const double *ky, const double *kz,
                    const double *lam, const double *x,
                    double *gx, double *gy, double *gz)
{
    if ((dim != 2 && dim != 3) || nx <= 0) return OR_EINVAL;
    const double h = 1.0 / (double)nx;
    const double hd2 = (dim == 2) ? 1.0 : h;
    const int64_t sxy = (int64_t)nx * ny;
    const int64_t N = sxy * nz;
    for (int64_t P = 0; P < N; ++P) { gx[P] = 0.0; gy[P] = 0.0; if (dim == 3) gz[P] = 0.0; }
    for (int k = 0; k < nz; ++k)
        for (int j = 0; j < ny; ++j)
            for (int i = 0; i < nx; ++i) {
                const int64_t P = i + (int64_t)nx * (j + (int64_t)ny * k);
                for (int axis = 0; axis < dim; ++axis) {
                    const double *kk = axis == 0 ? kx : (axis == 1 ? ky : kz);
                    double *g = axis == 0 ? gx : (axis == 1 ? gy : gz);
                    int lo = axis == 0 ? (i == 0) : (axis == 1 ? (j == 0) : (k == 0));
                    int hi = axis == 0 ? (i == nx - 1) : (axis == 1 ? (j == ny - 1) : (k == nz - 1));
                    int64_t stride = axis == 0 ? 1 : (axis == 1 ? nx : sxy);
                    for (int side = 0; side < 2; ++side) {
                        int at_bnd = side == 0 ? lo : hi;
                        if (at_bnd) {
                            if (axis == 1) { /* Dirichlet */
                                double T = hd2 * (2.0 * kk[P]);
                                double dLdT = -lam[P] * x[P];
                                g[P] += dLdT * T;
                            }
                            continue;
                        }
                        int64_t Q = side == 0 ? P - stride : P + stride;
                        double kP = kk[P], kN = kk[Q];
                        double T = hd2 * ((2.0 * kP * kN) / (kP + kN));
                        double dLdT = -(lam[P] - lam[Q]) * (x[P] - x[Q]);
                        g[P] += dLdT * (T * kN / (kP + kN));
                    }
                }
            }
    return OR_OK;
}

/* ------------------------------------------------------------------ */
/* Sparse basics                                                        */
/* ------------------------------------------------------------------ */

/* y = A x, each row summed in stored (ascending column) order. */
void or_spmv(int n, const int64_t *rp, const int32_t *ci, const double *v,
             const double *x, double *y)
{
    for (int i = 0; i < n; ++i) {
        double s = 0.0;
        for (int64_t e = rp[i]; e < rp[i + 1]; ++e) s = fma(v[e], x[ci[e]], s);
        y[i] = s;
    }
}

/* y = A^T x, accumulated row by row (i ascending). */
void or_spmv_t(int n, const int64_t *rp, const int32_t *ci, const double *v,
               const double *x, double *y)
{
    for (int i = 0; i < n; ++i) y[i] = 0.0;
    for (int i = 0; i < n; ++i)
        for (int64_t e = rp[i]; e < rp[i + 1]; ++e) y[ci[e]] = fma(v[e], x[i], y[ci[e]]);
}

static int64_t find_in_row(const int64_t *rp, const int32_t *ci, int row, int32_t c)
{
    int64_t lo = rp[row], hi = rp[row + 1] - 1;
    while (lo <= hi) {
        int64_t mid = lo + (hi - lo) / 2;
        if (ci[mid] == c) return mid;
        if (ci[mid] < c) lo = mid + 1; else hi = mid - 1;
    }
    return -1;
}

/* Validate a CSR: row pointers monotone from 0, columns in range and
 * strictly ascending per row, diagonal present.  Returns 0 or OR_EINVAL. */
int or_check_csr(int n, const int64_t *rp, const int32_t *ci)
{
    if (n < 0 || rp[0] != 0) return OR_EINVAL;
    for (int i = 0; i < n; ++i) {
        if (rp[i + 1] < rp[i]) return OR_EINVAL;
        int has_diag = 0;
        for (int64_t e = rp[i]; e < rp[i + 1]; ++e) {
            if (ci[e] < 0 || ci[e] >= n) return OR_EINVAL;
            if (e > rp[i] && ci[e] <= ci[e - 1]) return OR_EINVAL;
            if (ci[e] == i) has_diag = 1;
        }
        if (!has_diag) return OR_EINVAL;
    }
    return OR_OK;
}

/* Symmetrised off-diagonal adjacency: v in adj(u) iff u != v and a_uv or
 * a_vu is stored.  Lists ascending.  Caller frees *arp, *aci. */
static void sym_adjacency(int n, const int64_t *rp, const int32_t *ci,
                          int64_t **arp_out, int32_t **aci_out)
{
    int64_t nnz = rp[n];
    /* transpose pattern */
    int64_t *trp = calloc((size_t)n + 1, sizeof(int64_t));
    int32_t *tci = malloc(sizeof(int32_t) * (size_t)(nnz > 0 ? nnz : 1));
    for (int64_t e = 0; e < nnz; ++e) trp[ci[e] + 1]++;
    for (int i = 0; i < n; ++i) trp[i + 1] += trp[i];
    int64_t *fill = malloc(sizeof(int64_t) * (size_t)(n > 0 ? n : 1));
    for (int i = 0; i < n; ++i) fill[i] = trp[i];
    for (int i = 0; i < n; ++i)
        for (int64_t e = rp[i]; e < rp[i + 1]; ++e) tci[fill[ci[e]]++] = i;
    /* merge row i of A and row i of A^T, dropping the diagonal */
    int64_t *arp = calloc((size_t)n + 1, sizeof(int64_t));
    int32_t *aci = malloc(sizeof(int32_t) * (size_t)(2 * nnz > 0 ? 2 * nnz : 1));
    int64_t m = 0;
    for (int i = 0; i < n; ++i) {
        int64_t p = rp[i], q = trp[i];
        while (p < rp[i + 1] || q < trp[i + 1]) {
            int32_t c;
            if (q >= trp[i + 1] || (p < rp[i + 1] && ci[p] < tci[q])) c = ci[p++];
            else if (p >= rp[i + 1] || tci[q] < ci[p]) c = tci[q++];
            else { c = ci[p]; ++p; ++q; }
            if (c != i) aci[m++] = c;
        }
        arp[i + 1] = m;
    }
    free(trp); free(tci); free(fill);
    *arp_out = arp; *aci_out = aci;
}

/* ------------------------------------------------------------------ */
/* O2. Heavy-edge matching (one pass).  The paper forms aggregates from */
/* a graph partition of G(A) (Section 2, aggregation based on graph     */
/* matching); the deterministic variant used here pairs vertices by a   */
/* greedy maximal matching in decreasing edge-key order:                */
/*   edge {u,v}, u<v, exists iff a_uv or a_vu is stored, with weight    */
/*   w = (|a_uv| + |a_vu|) * 0.5 (missing entry = 0), kept iff w > 0;   */
/*   scaled weight (scaled = 1): w / sqrt(|a_uu| |a_vv|), the strength  */
/*   of connection of smoothed aggregation (Vanek, Mandel, Brezina,     */
/*   Computing 56, 1996) measured on the symmetrised coupling (reading: */
/*   the paper's partitioner keeps parts of equal size; unscaled        */
/*   weights grow with the aggregates, so a vertex left single on one   */
/*   level is outweighed by its neighbours on every later one and       */
/*   coarsening stalls);                                                */
/*   key = (w, mix64(((u<<32)|v) ^ seed), u, v), larger key first.      */
/* mate[u] = partner or -1.  Returns the number of pairs or -errno.     */
/* ------------------------------------------------------------------ */
typedef struct { double w; uint64_t hkey; int32_t u, v; } or_edge_t;

static int cmp_edge_desc(const void *a, const void *b)
{
    const or_edge_t *x = a, *y = b;
    if (x->w != y->w) return x->w > y->w ? -1 : 1;
    if (x->hkey != y->hkey) return x->hkey > y->hkey ? -1 : 1;
    if (x->u != y->u) return x->u > y->u ? -1 : 1;
    if (x->v != y->v) return x->v > y->v ? -1 : 1;
    return 0;
}

double or_edge_weight(const int64_t *rp, const int32_t *ci, const double *v, int u, int w)
{
    int lo = u < w ? u : w, hi = u < w ? w : u;
    int64_t e1 = find_in_row(rp, ci, lo, hi);
    int64_t e2 = find_in_row(rp, ci, hi, lo);
    double a1 = e1 >= 0 ? fabs(v[e1]) : 0.0;
    double a2 = e2 >= 0 ? fabs(v[e2]) : 0.0;
    return (a1 + a2) * 0.5;
}

static double diag_abs(const int64_t *rp, const int32_t *ci, const double *v, int u)
{
    int64_t e = find_in_row(rp, ci, u, u);
    return e >= 0 ? fabs(v[e]) : 0.0;
}

/* Weight of edge {u, w} in the matching key: plain, or divided by the  */
/* geometric mean of its endpoints' diagonal magnitudes, sqrt(|a_uu|    */
/* |a_ww|) with the product rounded first (a zero diagonal makes the    */
/* quotient +inf, an ordinary key value).                               */
double or_edge_key_weight(const int64_t *rp, const int32_t *ci, const double *v, int u, int w, int scaled)
{
    double x = or_edge_weight(rp, ci, v, u, w);
    if (scaled && x > 0.0) {
        double du = diag_abs(rp, ci, v, u), dw = diag_abs(rp, ci, v, w);
        x = x / sqrt(du * dw);
    }
    return x;
}

uint64_t or_edge_hash(int u, int v, uint64_t seed)
{
    uint64_t lo = (uint64_t)(uint32_t)(u < v ? u : v), hi = (uint64_t)(uint32_t)(u < v ? v : u);
    return or_mix64(((lo << 32) | hi) ^ seed);
}

int64_t or_match(int n, const int64_t *rp, const int32_t *ci, const double *v,
                 uint64_t seed, int scaled, int32_t *mate)
{
    int64_t *arp; int32_t *aci;
    sym_adjacency(n, rp, ci, &arp, &aci);
    int64_t ne = 0;
    or_edge_t *E = malloc(sizeof(or_edge_t) * (size_t)(arp[n] / 2 + 1));
    for (int u = 0; u < n; ++u)
        for (int64_t e = arp[u]; e < arp[u + 1]; ++e) {
            int w_ = aci[e];
            if (w_ <= u) continue;
            double w = or_edge_key_weight(rp, ci, v, u, w_, scaled);
            if (!(w > 0.0)) continue;
            E[ne].w = w; E[ne].hkey = or_edge_hash(u, w_, seed); E[ne].u = u; E[ne].v = w_;
            ++ne;
        }
    qsort(E, (size_t)ne, sizeof(or_edge_t), cmp_edge_desc);
    for (int u = 0; u < n; ++u) mate[u] = -1;
    int64_t pairs = 0;
    for (int64_t t = 0; t < ne; ++t)
        if (mate[E[t].u] < 0 && mate[E[t].v] < 0) {
            mate[E[t].u] = E[t].v; mate[E[t].v] = E[t].u; ++pairs;
        }
    free(E); free(arp); free(aci);
    return pairs;
}

/* ------------------------------------------------------------------ */
/* O3. Aggregates from a matching (eq. (4) partition; the "part" map of */
/* Section 2): each pair or singleton is one aggregate, numbered in     */
/* ascending order of its smallest member.  Returns N_c.                */
/* ------------------------------------------------------------------ */
int or_aggregate(int n, const int32_t *mate, int32_t *agg)
{
    int nc = 0;
    for (int u = 0; u < n; ++u)
        if (mate[u] < 0 || u < mate[u]) agg[u] = nc++;
    for (int u = 0; u < n; ++u)
        if (mate[u] >= 0 && mate[u] < u) agg[u] = agg[mate[u]];
    return nc;
}

/* ------------------------------------------------------------------ */
/* O4. Galerkin coarse matrix A_c = P^T A P (eq. (3)) in its entrywise  */
/* form (A_c)_IJ = sum_{k in G_I} sum_{l in G_J} a_kl (Section 2).       */
/* Entries of A in row-major, ascending-column order are stably sorted   */
/* by (agg[k], agg[l]); equal keys are summed sequentially in that       */
/* order, starting from the first value.  Every structurally present     */
/* coarse entry is kept.  Returns nnz_c (<= nnz).                        */
/* ------------------------------------------------------------------ */
typedef struct { uint64_t key; int64_t e; } or_kv_t;

static int cmp_kv(const void *a, const void *b)
{
    const or_kv_t *x = a, *y = b;
    if (x->key != y->key) return x->key < y->key ? -1 : 1;
    if (x->e != y->e) return x->e < y->e ? -1 : 1;
    return 0;
}

int64_t or_galerkin(int n, const int64_t *rp, const int32_t *ci, const double *v,
                    const int32_t *agg, int nc,
                    int64_t *crp, int32_t *cci, double *cv)
{
    int64_t nnz = rp[n];
    or_kv_t *kv = malloc(sizeof(or_kv_t) * (size_t)(nnz > 0 ? nnz : 1));
    for (int i = 0; i < n; ++i)
        for (int64_t e = rp[i]; e < rp[i + 1]; ++e) {
            kv[e].key = (uint64_t)(uint32_t)agg[i] * (uint64_t)nc + (uint64_t)(uint32_t)agg[ci[e]];
            kv[e].e = e;
        }
    qsort(kv, (size_t)nnz, sizeof(or_kv_t), cmp_kv);
    for (int I = 0; I <= nc; ++I) crp[I] = 0;
    int64_t m = 0;
    for (int64_t t = 0; t < nnz; ++t) {
        int I = (int)(kv[t].key / (uint64_t)nc), J = (int)(kv[t].key % (uint64_t)nc);
        if (t > 0 && kv[t].key == kv[t - 1].key) {
            cv[m - 1] += v[kv[t].e];
        } else {
            cci[m] = J; cv[m] = v[kv[t].e]; ++m;
            crp[I + 1] = m;
        }
    }
    for (int I = 0; I < nc; ++I) if (crp[I + 1] < crp[I]) crp[I + 1] = crp[I];
    free(kv);
    return m;
}

/* ------------------------------------------------------------------ */
/* O5a. Greedy colouring of the symmetrised graph in decreasing         */
/* priority; each vertex takes the smallest colour not used by its      */
/* already-coloured neighbours.  mode 0 (hash): priority               */
/* (mix64(i ^ (seed + SALT)), i); mode 1 (first fit): priority -i.      */
/* The paper orders ILU(0) naturally or by nested dissection (Section   */
/* 3, "Comments on numerical results"); a colour-major order is the     */
/* reading adopted for a parallel smoother.  Returns #colours.          */
/* ------------------------------------------------------------------ */
typedef struct { uint64_t h; int32_t i; } or_prio_t;

static int cmp_prio_desc(const void *a, const void *b)
{
    const or_prio_t *x = a, *y = b;
    if (x->h != y->h) return x->h > y->h ? -1 : 1;
    if (x->i != y->i) return x->i > y->i ? -1 : 1;
    return 0;
}

int or_color(int n, const int64_t *rp, const int32_t *ci, int mode, uint64_t seed,
             int32_t *color)
{
    int64_t *arp; int32_t *aci;
    sym_adjacency(n, rp, ci, &arp, &aci);
    or_prio_t *pr = malloc(sizeof(or_prio_t) * (size_t)(n > 0 ? n : 1));
    for (int i = 0; i < n; ++i) {
        pr[i].i = i;
        pr[i].h = (mode == 0) ? or_mix64((uint64_t)(uint32_t)i ^ (seed + OR_COLOR_SALT)) : 0;
    }
    if (mode == 0) qsort(pr, (size_t)n, sizeof(or_prio_t), cmp_prio_desc);
    for (int i = 0; i < n; ++i) color[i] = -1;
    int ncol = 0;
    int32_t *stamp = malloc(sizeof(int32_t) * (size_t)(n + 2));
    for (int i = 0; i < n + 2; ++i) stamp[i] = -1;
    for (int t = 0; t < n; ++t) {
        int u = pr[t].i;
        for (int64_t e = arp[u]; e < arp[u + 1]; ++e) {
            int c = color[aci[e]];
            if (c >= 0) stamp[c] = u;
        }
        int c = 0;
        while (stamp[c] == u) ++c;
        color[u] = c;
        if (c + 1 > ncol) ncol = c + 1;
    }
    free(stamp); free(pr); free(arp); free(aci);
    return ncol;
}

/* Elimination order: rows sorted by (colour, index).  pos[i] = rank. */
static void colour_order(int n, const int32_t *color, int32_t *perm, int32_t *pos)
{
    int ncol = 0;
    for (int i = 0; i < n; ++i) if (color[i] + 1 > ncol) ncol = color[i] + 1;
    int64_t *cnt = calloc((size_t)ncol + 1, sizeof(int64_t));
    for (int i = 0; i < n; ++i) cnt[color[i] + 1]++;
    for (int c = 0; c < ncol; ++c) cnt[c + 1] += cnt[c];
    for (int i = 0; i < n; ++i) { perm[cnt[color[i]]] = i; pos[i] = (int32_t)cnt[color[i]]; cnt[color[i]]++; }
    free(cnt);
}

/* ------------------------------------------------------------------ */
/* O5b. ILU(0) (Algorithm 1, smoother setup: zero-fill incomplete LU)     */
/* in the colour-major elimination order: the IKJ variant restricted    */
/* to the pattern of A.  For each row i in order, for each k with        */
/* pos(k) < pos(i) stored in row i, in increasing pos(k):                */
/*   a_ik <- a_ik / a_kk;  a_ij <- a_ij - a_ik * a_kj for every stored    */
/*   (k, j) with pos(j) > pos(k) whose (i, j) is stored.                  */
/* lu receives L (unit diagonal implied) and U on A's natural CSR        */
/* layout.  Returns 0, or OR_EBREAKDOWN on a zero / non-finite pivot.    */
/* ------------------------------------------------------------------ */
typedef struct { int32_t p; int64_t e; } or_pe_t;

int or_ilu0(int n, const int64_t *rp, const int32_t *ci, const double *v,
            const int32_t *color, double *lu)
{
    int64_t nnz = rp[n];
    memcpy(lu, v, sizeof(double) * (size_t)nnz);
    int32_t *perm = malloc(sizeof(int32_t) * (size_t)(n > 0 ? n : 1));
    int32_t *pos = malloc(sizeof(int32_t) * (size_t)(n > 0 ? n : 1));
    int64_t *dpos = malloc(sizeof(int64_t) * (size_t)(n > 0 ? n : 1));
    colour_order(n, color, perm, pos);
    for (int i = 0; i < n; ++i) dpos[i] = find_in_row(rp, ci, i, i);
    int maxlen = 0;
    for (int i = 0; i < n; ++i) if (rp[i + 1] - rp[i] > maxlen) maxlen = (int)(rp[i + 1] - rp[i]);
    or_pe_t *L = malloc(sizeof(or_pe_t) * (size_t)(maxlen + 1));
    int status = OR_OK;
    for (int t = 0; t < n && status == OR_OK; ++t) {
        int i = perm[t];
        int nl = 0;
        for (int64_t e = rp[i]; e < rp[i + 1]; ++e)
            if (pos[ci[e]] < pos[i]) { L[nl].p = pos[ci[e]]; L[nl].e = e; ++nl; }
        for (int a = 1; a < nl; ++a) {          /* insertion sort by pos */
            or_pe_t x = L[a]; int b = a - 1;
            while (b >= 0 && L[b].p > x.p) { L[b + 1] = L[b]; --b; }
            L[b + 1] = x;
        }
        for (int a = 0; a < nl; ++a) {
            int64_t eik = L[a].e;
            int k = ci[eik];
            lu[eik] = lu[eik] / lu[dpos[k]];
            for (int64_t ekj = rp[k]; ekj < rp[k + 1]; ++ekj) {
                int j = ci[ekj];
                if (pos[j] <= pos[k]) continue;
                int64_t eij = find_in_row(rp, ci, i, j);
                if (eij < 0) continue;
                lu[eij] = lu[eij] - lu[eik] * lu[ekj];
            }
        }
        double piv = lu[dpos[i]];
        if (piv == 0.0 || !isfinite(piv)) status = OR_EBREAKDOWN;
    }
    free(L); free(perm); free(pos); free(dpos);
    return status;
}

/* t = (L U)^{-1} z: forward L y = z then backward U t = y, rows in the
 * colour-major order, each row's terms in stored column order. */
void or_ilu_solve(int n, const int64_t *rp, const int32_t *ci, const double *lu,
                  const int32_t *color, const double *z, double *t)
{
    int32_t *perm = malloc(sizeof(int32_t) * (size_t)(n > 0 ? n : 1));
    int32_t *pos = malloc(sizeof(int32_t) * (size_t)(n > 0 ? n : 1));
    double *y = malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
    colour_order(n, color, perm, pos);
    for (int q = 0; q < n; ++q) {
        int i = perm[q];
        double s = z[i];
        for (int64_t e = rp[i]; e < rp[i + 1]; ++e)
            if (pos[ci[e]] < pos[i]) s = fma(-lu[e], y[ci[e]], s);
        y[i] = s;
    }
    for (int q = n - 1; q >= 0; --q) {
        int i = perm[q];
        double s = y[i], d = 0.0;
        for (int64_t e = rp[i]; e < rp[i + 1]; ++e) {
            if (pos[ci[e]] > pos[i]) s = fma(-lu[e], t[ci[e]], s);
            else if (ci[e] == i) d = lu[e];
        }
        t[i] = s / d;
    }
    free(perm); free(pos); free(y);
}

/* t = (L U)^{-T} z = L^{-T} U^{-T} z.  U^T w = z is lower triangular in
 * the elimination order (column sweep forward); L^T t = w is unit upper
 * triangular (column sweep backward). */
void or_ilu_solve_t(int n, const int64_t *rp, const int32_t *ci, const double *lu,
                    const int32_t *color, const double *z, double *t)
{
    int32_t *perm = malloc(sizeof(int32_t) * (size_t)(n > 0 ? n : 1));
    int32_t *pos = malloc(sizeof(int32_t) * (size_t)(n > 0 ? n : 1));
    double *w = malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
    colour_order(n, color, perm, pos);
    for (int i = 0; i < n; ++i) w[i] = z[i];
    for (int q = 0; q < n; ++q) {
        int i = perm[q];
        double d = 0.0;
        for (int64_t e = rp[i]; e < rp[i + 1]; ++e) if (ci[e] == i) d = lu[e];
        w[i] = w[i] / d;
        for (int64_t e = rp[i]; e < rp[i + 1]; ++e)
            if (pos[ci[e]] > pos[i]) w[ci[e]] = fma(-lu[e], w[i], w[ci[e]]);
    }
    for (int i = 0; i < n; ++i) t[i] = w[i];
    for (int q = n - 1; q >= 0; --q) {
        int i = perm[q];
        for (int64_t e = rp[i]; e < rp[i + 1]; ++e)
            if (pos[ci[e]] < pos[i]) t[ci[e]] = fma(-lu[e], t[i], t[ci[e]]);
    }
    free(perm); free(pos); free(w);
}

/* ------------------------------------------------------------------ */
/* O5c. ILUT(tau): the incomplete factorisation with a drop tolerance   */
/* that the paper applies to the coarse operator, A~_c = L~_c U~_c =     */
/* ILUT(A_c) (Section 2; Algorithm 1 setup), with the dropping rule of   */
/* Saad's ILUT and no limit on the entries per row, no pivoting (the     */
/* paper's operators are M-matrices, for which it notes pivoting is      */
/* rarely needed).  Natural order.  For each row i:                      */
/*   tau_i = tau * ||a_i||_2 (sum of squares in stored column order);    */
/*   w = a_i;                                                            */
/*   for k < i with w_k stored, in increasing k (fill included):         */
/*     w_k <- w_k / u_kk;  if w_k == 0 or |w_k| < tau_i drop it, else    */
/*     w_j <- w_j - w_k * u_kj for every stored u_kj, j > k;             */
/*   row i of L~ = the kept w_k (unit diagonal implied); row i of U~ =   */
/*   w_i and the w_j, j > i, with w_j != 0 and |w_j| >= tau_i.           */
/* Each product and each sum is rounded (setup arithmetic).  tau = 0     */
/* keeps every nonzero: the complete LU factorisation without pivoting.  */
/* Output: one CSR per row, L~ part then U~ part, ascending columns.     */
/* ------------------------------------------------------------------ */
typedef struct {
    int n;
    int64_t nnz, cap;
    int64_t *rp;        /* [n+1] */
    int32_t *ci;
    double *v;
    int64_t *dpos;      /* [n] index of u_ii */
} or_ilut_t;

static void ilut_push(or_ilut_t *F, int32_t c, double x)
{
    if (F->nnz == F->cap) {
        F->cap = F->cap ? 2 * F->cap : 1024;
        F->ci = realloc(F->ci, sizeof(int32_t) * (size_t)F->cap);
        F->v = realloc(F->v, sizeof(double) * (size_t)F->cap);
    }
    F->ci[F->nnz] = c;
    F->v[F->nnz] = x;
    F->nnz++;
}

static int cmp_i32(const void *a, const void *b)
{
    int32_t x = *(const int32_t *)a, y = *(const int32_t *)b;
    return (x > y) - (x < y);
}

or_ilut_t *or_ilut(int n, const int64_t *rp, const int32_t *ci, const double *v, double tau, int *status)
{
    *status = OR_OK;
    if (n < 0 || !(tau >= 0.0)) { *status = OR_EINVAL; return NULL; }
    or_ilut_t *F = calloc(1, sizeof(or_ilut_t));
    F->n = n;
    F->rp = malloc(sizeof(int64_t) * (size_t)(n + 1));
    F->dpos = malloc(sizeof(int64_t) * (size_t)(n > 0 ? n : 1));
    double *w = calloc((size_t)(n > 0 ? n : 1), sizeof(double));
    int32_t *mark = malloc(sizeof(int32_t) * (size_t)(n > 0 ? n : 1));
    int32_t *lst = malloc(sizeof(int32_t) * (size_t)(n > 0 ? n : 1));   /* stored positions of w */
    char *done = calloc((size_t)(n > 0 ? n : 1), 1);
    for (int j = 0; j < n; ++j) mark[j] = -1;
    F->rp[0] = 0;
    for (int i = 0; i < n; ++i) {
        double sq = 0.0;
        for (int64_t e = rp[i]; e < rp[i + 1]; ++e) sq = sq + v[e] * v[e];
        const double ti = tau * sqrt(sq);
        int len = 0;
        for (int64_t e = rp[i]; e < rp[i + 1]; ++e) {
            w[ci[e]] = v[e]; mark[ci[e]] = i; lst[len++] = ci[e];
        }
        if (mark[i] != i) { w[i] = 0.0; mark[i] = i; lst[len++] = i; }
        /* eliminate: the smallest unprocessed k < i each time */
        for (;;) {
            int k = -1;
            for (int a = 0; a < len; ++a)
                if (lst[a] < i && !done[lst[a]] && (k < 0 || lst[a] < k)) k = lst[a];
            if (k < 0) break;
            done[k] = 1;
            double wk = w[k] / F->v[F->dpos[k]];
            if (wk == 0.0 || fabs(wk) < ti) { w[k] = 0.0; continue; }
            w[k] = wk;
            for (int64_t e = F->dpos[k] + 1; e < F->rp[k + 1]; ++e) {
                int j = F->ci[e];
                if (mark[j] != i) { mark[j] = i; w[j] = 0.0; lst[len++] = j; }
                w[j] = w[j] - wk * F->v[e];
            }
        }
        qsort(lst, (size_t)len, sizeof(int32_t), cmp_i32);
        for (int a = 0; a < len; ++a) {
            int j = lst[a];
            double x = w[j];
            if (j < i) {
                if (done[j] && x != 0.0) ilut_push(F, j, x);
            } else if (j == i) {
                F->dpos[i] = F->nnz;
                ilut_push(F, j, x);
                if (x == 0.0 || !isfinite(x)) *status = OR_EBREAKDOWN;
            } else if (x != 0.0 && !(fabs(x) < ti)) {
                ilut_push(F, j, x);
            }
        }
        for (int a = 0; a < len; ++a) { done[lst[a]] = 0; w[lst[a]] = 0.0; }
        F->rp[i + 1] = F->nnz;
    }
    free(w); free(mark); free(lst); free(done);
    return F;
}

int64_t or_ilut_nnz(const or_ilut_t *F) { return F->nnz; }

void or_ilut_get(const or_ilut_t *F, int64_t *rp, int32_t *ci, double *v)
{
    memcpy(rp, F->rp, sizeof(int64_t) * (size_t)(F->n + 1));
    memcpy(ci, F->ci, sizeof(int32_t) * (size_t)F->nnz);
    memcpy(v, F->v, sizeof(double) * (size_t)F->nnz);
}

/* t = (L~ U~)^{-1} z: forward then backward substitution in natural
 * order, each row's terms accumulated in stored column order (solve
 * phase: fused multiply-add), the backward row divided by u_ii. */
void or_ilut_solve(const or_ilut_t *F, const double *z, double *t)
{
    const int n = F->n;
    double *y = malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
    for (int i = 0; i < n; ++i) {
        double s = z[i];
        for (int64_t e = F->rp[i]; e < F->dpos[i]; ++e) s = fma(-F->v[e], y[F->ci[e]], s);
        y[i] = s;
    }
    for (int i = n - 1; i >= 0; --i) {
        double s = y[i];
        for (int64_t e = F->dpos[i] + 1; e < F->rp[i + 1]; ++e) s = fma(-F->v[e], t[F->ci[e]], s);
        t[i] = s / F->v[F->dpos[i]];
    }
    free(y);
}

/* t = (L~ U~)^{-T} z = L~^{-T} U~^{-T} z: U~^T w = z column by column in
 * increasing i (divide by u_ii, then scatter -u_ij w_i to later rows),
 * then L~^T t = w in decreasing i (scatter -l_ij t_i to earlier rows). */
void or_ilut_solve_t(const or_ilut_t *F, const double *z, double *t)
{
    const int n = F->n;
    double *w = malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
    for (int i = 0; i < n; ++i) w[i] = z[i];
    for (int i = 0; i < n; ++i) {
        w[i] = w[i] / F->v[F->dpos[i]];
        for (int64_t e = F->dpos[i] + 1; e < F->rp[i + 1]; ++e) w[F->ci[e]] = fma(-F->v[e], w[i], w[F->ci[e]]);
    }
    for (int i = 0; i < n; ++i) t[i] = w[i];
    for (int i = n - 1; i >= 0; --i)
        for (int64_t e = F->rp[i]; e < F->dpos[i]; ++e) t[F->ci[e]] = fma(-F->v[e], t[i], t[F->ci[e]]);
    free(w);
}

void or_ilut_free(or_ilut_t *F)
{
    if (!F) return;
    free(F->rp); free(F->ci); free(F->v); free(F->dpos); free(F);
}

/* ------------------------------------------------------------------ */
/* Exact solve of the smallest level: the inverse by Gauss-Jordan        */
/* elimination with partial pivoting on [A | I] (pivot of column k: the  */
/* first row of largest magnitude at or below k; the pivot row is        */
/* divided by the pivot, then each other row i with f = m_ik != 0 gets   */
/* m_ij - f m_kj as one fused multiply-add), applied as a product with   */
/* the inverse.  a is n x n row-major (input); inv receives A^{-1}.      */
/* ------------------------------------------------------------------ */
static int dense_inverse(int n, const double *a, double *inv)
{
    size_t w = 2 * (size_t)n;
    double *m = calloc((size_t)n * w, sizeof(double));
    double *f = malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
    for (int i = 0; i < n; ++i) {
        for (int j = 0; j < n; ++j) m[(size_t)i * w + j] = a[(size_t)i * n + j];
        m[(size_t)i * w + n + i] = 1.0;
    }
    int status = OR_OK;
    for (int k = 0; k < n; ++k) {
        int p = k;
        double best = fabs(m[(size_t)k * w + k]);
        for (int i = k + 1; i < n; ++i)
            if (fabs(m[(size_t)i * w + k]) > best) { best = fabs(m[(size_t)i * w + k]); p = i; }
        if (!(best > 0.0) || !isfinite(best)) { status = OR_EBREAKDOWN; p = k; }
        if (p != k)
            for (size_t j = 0; j < w; ++j) {
                double t = m[(size_t)k * w + j]; m[(size_t)k * w + j] = m[(size_t)p * w + j]; m[(size_t)p * w + j] = t;
            }
        double d = m[(size_t)k * w + k];
        for (size_t j = 0; j < w; ++j) m[(size_t)k * w + j] = m[(size_t)k * w + j] / d;
        for (int i = 0; i < n; ++i) f[i] = (i == k) ? 0.0 : m[(size_t)i * w + k];
        for (int i = 0; i < n; ++i) {
            if (i == k || f[i] == 0.0) continue;
            for (size_t j = 0; j < w; ++j) m[(size_t)i * w + j] = fma(-f[i], m[(size_t)k * w + j], m[(size_t)i * w + j]);
        }
    }
    for (int i = 0; i < n; ++i)
        for (int j = 0; j < n; ++j) inv[(size_t)i * n + j] = m[(size_t)i * w + n + j];
    free(m); free(f);
    return status;
}

/* x = A^{-1} b (transpose = 0) or A^{-T} b (transpose = 1) from the     */
/* inverse: x_i = sum_j inv_ij b_j (inv_ji for the transpose), each row   */
/* an inner product evaluated as the Arnoldi inner products are (below):  */
/* as if in twice the working precision (Dot2), terms in ascending j.     */
static double dot2_strided(int n, const double *a, size_t stride, const double *b);

static void dense_solve(int n, const double *inv, const double *b, double *x, int transpose)
{
    for (int i = 0; i < n; ++i)
        x[i] = transpose ? dot2_strided(n, inv + i, (size_t)n, b) : dot2_strided(n, inv + (size_t)i * n, 1, b);
}

/* ------------------------------------------------------------------ */
/* Hierarchy.  Level 0 is A.  Level l+1 is the Galerkin product of level */
/* l through `passes` matching passes (Algorithm 1 setup: partition ->   */
/* P -> A_c), so each level's aggregates hold at most 2^passes points.   */
/* Every non-final level keeps its ILU(0) factors (the smoother S_l of   */
/* Algorithm 1) in its elimination order: natural (the paper's GMG-NO,   */
/* Section 3) or colour-major.  Coarsening stops when a level has at     */
/* most dense_max rows (it is then solved exactly, by its inverse), when */
/* matching no longer shrinks the level by 10%, or at max_levels; a      */
/* final level too large for the inverse keeps only its ILU(0) factors.  */
/*                                                                       */
/* Reading of the inexact coarse solve (Section 2 applies one ILUT(A_c)  */
/* solve; here a fixed small number of inner iterations is used): the    */
/* coarse system of level l+1 is solved by k_{l+1} Richardson steps      */
/*   g <- g + B_{l+1}^{-1} (h - A_{l+1} g),  g = 0 initially,            */
/* whose preconditioner B_{l+1} is the same two-grid construction built  */
/* on A_{l+1}; k_1 = coarse_inner (5), deeper levels deep_inner (1).     */
/* ------------------------------------------------------------------ */
typedef struct {
    int n; int64_t nnz; int64_t *rp; int32_t *ci; double *v;
} or_csr_t;

#define OR_MAX_LEVELS 24
#define OR_MAX_PASSES 8

typedef struct {
    or_csr_t A;
    int npass;                          /* matching passes run from this level */
    or_csr_t mid[OR_MAX_PASSES];        /* intermediate Galerkin products */
    int32_t *agg_pass[OR_MAX_PASSES];   /* per-pass maps */
    int n_pass[OR_MAX_PASSES + 1];
    int32_t *agg;                       /* composite map to the next level */
    int32_t *color;                     /* elimination-order labels */
    int ncol;
    double *lu;                         /* ILU(0) factors on A's layout */
    double *dense;                      /* final level: dense inverse, or NULL */
    or_ilut_t *ilut;                    /* level 1 of the ILUT two-grid, or NULL */
} or_level_t;

typedef struct {
    int nlev;
    or_level_t lev[OR_MAX_LEVELS];
    int passes, coarse_inner, deep_inner, dense_max, order_fine, order_coarse, coloring;
    int coarse_ilut;                    /* 1: two-grid, level 1 factored by ILUT(ilut_tau) */
    double ilut_tau;
    uint64_t seed;
    int status;
} or_hier_t;

static void csr_copy(or_csr_t *d, int n, const int64_t *rp, const int32_t *ci, const double *v)
{
    d->n = n; d->nnz = rp[n];
    d->rp = malloc(sizeof(int64_t) * ((size_t)n + 1));
    d->ci = malloc(sizeof(int32_t) * (size_t)(d->nnz > 0 ? d->nnz : 1));
    d->v = malloc(sizeof(double) * (size_t)(d->nnz > 0 ? d->nnz : 1));
    memcpy(d->rp, rp, sizeof(int64_t) * ((size_t)n + 1));
    memcpy(d->ci, ci, sizeof(int32_t) * (size_t)d->nnz);
    memcpy(d->v, v, sizeof(double) * (size_t)d->nnz);
}

static void csr_free(or_csr_t *d) { free(d->rp); free(d->ci); free(d->v); memset(d, 0, sizeof(*d)); }

void or_free(or_hier_t *H)
{
    if (!H) return;
    for (int l = 0; l < H->nlev; ++l) {
        or_level_t *L = &H->lev[l];
        csr_free(&L->A);
        for (int p = 0; p < OR_MAX_PASSES; ++p) { csr_free(&L->mid[p]); free(L->agg_pass[p]); }
        free(L->agg); free(L->color); free(L->lu); free(L->dense);
        or_ilut_free(L->ilut);
    }
    free(H);
}

/* Aggregate level L by `passes` matching passes; fills L->agg and returns
 * the next level's matrix in *next. */
static void coarsen_level(or_level_t *L, int passes, uint64_t seed, int scaled, or_csr_t *next)
{
    int n = L->A.n;
    or_csr_t cur = L->A;   /* borrowed */
    L->agg = malloc(sizeof(int32_t) * (size_t)n);
    for (int i = 0; i < n; ++i) L->agg[i] = i;
    L->n_pass[0] = n;
    L->npass = passes;
    for (int p = 0; p < passes; ++p) {
        int m = cur.n;
        int32_t *mate = malloc(sizeof(int32_t) * (size_t)(m > 0 ? m : 1));
        or_match(m, cur.rp, cur.ci, cur.v, seed, scaled, mate);
        L->agg_pass[p] = malloc(sizeof(int32_t) * (size_t)(m > 0 ? m : 1));
        int nc = or_aggregate(m, mate, L->agg_pass[p]);
        free(mate);
        or_csr_t c;
        c.n = nc;
        c.rp = malloc(sizeof(int64_t) * ((size_t)nc + 1));
        c.ci = malloc(sizeof(int32_t) * (size_t)(cur.nnz > 0 ? cur.nnz : 1));
        c.v = malloc(sizeof(double) * (size_t)(cur.nnz > 0 ? cur.nnz : 1));
        c.nnz = or_galerkin(m, cur.rp, cur.ci, cur.v, L->agg_pass[p], nc, c.rp, c.ci, c.v);
        for (int i = 0; i < n; ++i) L->agg[i] = L->agg_pass[p][L->agg[i]];
        L->n_pass[p + 1] = nc;
        if (p + 1 < passes) { L->mid[p] = c; cur = c; }
        else *next = c;
    }
}

or_hier_t *or_setup(int n, const int64_t *rp, const int32_t *ci, const double *v,
                    const int32_t *opt, double ilut_tau, uint64_t seed, int *status)
{
    /* opt: [passes, coarse_inner, deep_inner, dense_max, max_levels,
     *       order_fine, order_coarse, coloring, coarse_solver, match_weight]
     * match_weight: 0 = plain edge weights, 1 = scaled (see O2).
     * order: 0 = colour-major (hash or first-fit colouring), 1 = natural.
     * coarse_solver: 0 = the recursive Richardson coarse solve; 1 = the
     * paper's two-grid form (Section 2, Algorithm 1): level 1 is the last
     * one, factored once by ILUT(ilut_tau) and solved with its factors. */
    *status = OR_OK;
    int passes = opt[0], coarse_inner = opt[1], deep_inner = opt[2], dense_max = opt[3];
    int max_levels = opt[4], order_fine = opt[5], order_coarse = opt[6], coloring = opt[7];
    int coarse_ilut = opt[8], scaled = opt[9];
    if (coarse_ilut) max_levels = 2;
    if (n <= 0 || passes < 1 || passes > OR_MAX_PASSES || coarse_inner < 1 || deep_inner < 1 ||
        dense_max < 0 || max_levels < 2 || max_levels > OR_MAX_LEVELS || coarse_ilut < 0 || coarse_ilut > 1 ||
        (coarse_ilut && !(ilut_tau >= 0.0)) || scaled < 0 || scaled > 1) { *status = OR_EINVAL; return NULL; }
    if (or_check_csr(n, rp, ci) != OR_OK) { *status = OR_EINVAL; return NULL; }
    or_hier_t *H = calloc(1, sizeof(or_hier_t));
    H->passes = passes; H->coarse_inner = coarse_inner; H->deep_inner = deep_inner;
    H->dense_max = dense_max; H->order_fine = order_fine; H->order_coarse = order_coarse;
    H->coloring = coloring; H->seed = seed;
    H->coarse_ilut = coarse_ilut; H->ilut_tau = ilut_tau;
    csr_copy(&H->lev[0].A, n, rp, ci, v);
    H->nlev = 1;
    for (int l = 0; ; ++l) {
        or_level_t *L = &H->lev[l];
        int last = (l > 0 && L->A.n <= dense_max) || (l + 1 >= max_levels);
        if (!last) {
            or_csr_t next;
            coarsen_level(L, passes, seed, scaled, &next);
            if (l > 0 && (double)next.n > 0.9 * (double)L->A.n) {
                /* matching no longer coarsens: this level is the last one */
                csr_free(&next);
                for (int p = 0; p < OR_MAX_PASSES; ++p) { csr_free(&L->mid[p]); free(L->agg_pass[p]); L->agg_pass[p] = NULL; }
                free(L->agg); L->agg = NULL; L->npass = 0;
                last = 1;
            } else {
                H->lev[l + 1].A = next;
                H->nlev = l + 2;
            }
        }
        int m = L->A.n;
        if (coarse_ilut && l == 1) {
            int st = OR_OK;
            L->ilut = or_ilut(m, L->A.rp, L->A.ci, L->A.v, ilut_tau, &st);
            if (st != OR_OK) *status = st;
        } else if (last && m <= dense_max) {
            double *a = calloc((size_t)m * (size_t)m, sizeof(double));
            L->dense = malloc(sizeof(double) * (size_t)m * (size_t)m);
            for (int i = 0; i < m; ++i)
                for (int64_t e = L->A.rp[i]; e < L->A.rp[i + 1]; ++e)
                    a[(size_t)i * m + L->A.ci[e]] = L->A.v[e];
            if (dense_inverse(m, a, L->dense) != OR_OK) *status = OR_EBREAKDOWN;
            free(a);
        } else {
            int ord = (l == 0) ? order_fine : order_coarse;
            L->color = malloc(sizeof(int32_t) * (size_t)m);
            if (ord == 1) { for (int i = 0; i < m; ++i) L->color[i] = 0; L->ncol = 1; }
            else L->ncol = or_color(m, L->A.rp, L->A.ci, coloring, seed, L->color);
            L->lu = malloc(sizeof(double) * (size_t)(L->A.nnz > 0 ? L->A.nnz : 1));
            if (or_ilu0(m, L->A.rp, L->A.ci, L->A.v, L->color, L->lu) != OR_OK) *status = OR_EBREAKDOWN;
        }
        if (last) break;
    }
    H->status = *status;
    return H;
}

int or_hier_nlev(const or_hier_t *H) { return H->nlev; }

/* info[0..7] for level l: n, nnz (low 31 bits unsafe -> see or_hier_nnz),
 * ncol, has_dense, npass, n after pass 1, n of next level, has_lu */
void or_hier_level_info(const or_hier_t *H, int l, int32_t *info)
{
    const or_level_t *L = &H->lev[l];
    info[0] = L->A.n; info[1] = (int32_t)(L->A.nnz > 0x7fffffff ? -1 : L->A.nnz);
    info[2] = L->ncol; info[3] = L->dense != NULL; info[4] = L->npass;
    info[5] = L->npass > 0 ? L->n_pass[1] : -1;
    info[6] = (l + 1 < H->nlev) ? H->lev[l + 1].A.n : -1;
    info[7] = L->lu != NULL;
}

int64_t or_hier_nnz(const or_hier_t *H, int l) { return H->lev[l].A.nnz; }

void or_hier_matrix(const or_hier_t *H, int l, int64_t *rp, int32_t *ci, double *v)
{
    const or_csr_t *M = &H->lev[l].A;
    memcpy(rp, M->rp, sizeof(int64_t) * ((size_t)M->n + 1));
    memcpy(ci, M->ci, sizeof(int32_t) * (size_t)M->nnz);
    memcpy(v, M->v, sizeof(double) * (size_t)M->nnz);
}

/* pass 0: composite map of level l; pass p >= 1: map of pass p. */
int or_hier_agg(const or_hier_t *H, int l, int pass, int32_t *out)
{
    const or_level_t *L = &H->lev[l];
    if (!L->agg) return OR_EINVAL;
    if (pass == 0) { memcpy(out, L->agg, sizeof(int32_t) * (size_t)L->A.n); return OR_OK; }
    if (pass < 1 || pass > L->npass) return OR_EINVAL;
    memcpy(out, L->agg_pass[pass - 1], sizeof(int32_t) * (size_t)L->n_pass[pass - 1]);
    return OR_OK;
}

int or_hier_pass_n(const or_hier_t *H, int l, int p)
{
    const or_level_t *L = &H->lev[l];
    return (p >= 0 && p <= L->npass) ? L->n_pass[p] : -1;
}

int64_t or_hier_mid_nnz(const or_hier_t *H, int l, int p)
{
    const or_level_t *L = &H->lev[l];
    return (p >= 1 && p < L->npass) ? L->mid[p - 1].nnz : -1;
}

void or_hier_mid(const or_hier_t *H, int l, int p, int64_t *rp, int32_t *ci, double *v)
{
    const or_csr_t *M = &H->lev[l].mid[p - 1];
    memcpy(rp, M->rp, sizeof(int64_t) * ((size_t)M->n + 1));
    memcpy(ci, M->ci, sizeof(int32_t) * (size_t)M->nnz);
    memcpy(v, M->v, sizeof(double) * (size_t)M->nnz);
}

void or_hier_colors(const or_hier_t *H, int l, int32_t *out)
{
    memcpy(out, H->lev[l].color, sizeof(int32_t) * (size_t)H->lev[l].A.n);
}

void or_hier_lu(const or_hier_t *H, int l, double *out)
{
    memcpy(out, H->lev[l].lu, sizeof(double) * (size_t)H->lev[l].A.nnz);
}

/* ------------------------------------------------------------------ */
/* O6. Preconditioner.  Algorithm 1's preconditioner application does   */
/*   S t = z; M~ f = z; M~ q' = A t; q = t + f - q'                      */
/* with M~^{-1} = P A~_c^{-1} P^T linear, so q = t + M~^{-1}(z - A t):   */
/* one coarse solve of the restricted residual (eq. (5), inexact M~).    */
/* At level l:                                                           */
/*   t = S_l^{-1} z        ILU(0) forward/backward sweep                 */
/*   r = z - A_l t                                                       */
/*   h[I] = sum_{i in G_I} r_i        restriction P^T (i ascending)      */
/*   g = C_{l+1}(h)                   inexact coarse solve               */
/*   q_i = t_i + g[agg_i]             prolongation P and correction      */
/* C_m(h): product with the inverse on a dense final level; one solve    */
/* with the ILUT factors in the two-grid form; k_m                       */
/* Richardson steps with S_m^{-1} on a final level without it; else k_m  */
/* Richardson steps g <- g + B_m^{-1}(h - A_m g) from g = 0.             */
/* ------------------------------------------------------------------ */
void or_restrict(const or_hier_t *H, int l, const double *r, double *hc)
{
    const or_level_t *L = &H->lev[l];
    int nc = H->lev[l + 1].A.n;
    for (int I = 0; I < nc; ++I) hc[I] = 0.0;
    for (int i = 0; i < L->A.n; ++i) hc[L->agg[i]] += r[i];
}

void or_smooth(const or_hier_t *H, int l, const double *z, double *t, int transpose)
{
    const or_level_t *L = &H->lev[l];
    if (transpose) or_ilu_solve_t(L->A.n, L->A.rp, L->A.ci, L->lu, L->color, z, t);
    else or_ilu_solve(L->A.n, L->A.rp, L->A.ci, L->lu, L->color, z, t);
}

static void precond_level(const or_hier_t *H, int l, const double *z, double *q, int transpose);

void or_level_solve(const or_hier_t *H, int l, const double *h, double *g, int transpose)
{
    const or_level_t *L = &H->lev[l];
    int m = L->A.n;
    if (L->dense) { dense_solve(m, L->dense, h, g, transpose); return; }
    if (L->ilut) {                       /* A~_c^{-1} h with the ILUT factors */
        if (transpose) or_ilut_solve_t(L->ilut, h, g);
        else or_ilut_solve(L->ilut, h, g);
        return;
    }
    int k = (l == 1) ? H->coarse_inner : H->deep_inner;
    double *res = malloc(sizeof(double) * (size_t)(m > 0 ? m : 1));
    double *d = malloc(sizeof(double) * (size_t)(m > 0 ? m : 1));
    for (int i = 0; i < m; ++i) g[i] = 0.0;
    for (int it = 0; it < k; ++it) {
        if (it == 0) {
            for (int i = 0; i < m; ++i) res[i] = h[i];
        } else {
            if (transpose) or_spmv_t(m, L->A.rp, L->A.ci, L->A.v, g, res);
            else or_spmv(m, L->A.rp, L->A.ci, L->A.v, g, res);
            for (int i = 0; i < m; ++i) res[i] = h[i] - res[i];
        }
        if (L->agg) precond_level(H, l, res, d, transpose);
        else or_smooth(H, l, res, d, transpose);
        for (int i = 0; i < m; ++i) g[i] = g[i] + d[i];
    }
    free(res); free(d);
}

static void precond_level(const or_hier_t *H, int l, const double *z, double *q, int transpose)
{
    const or_level_t *L = &H->lev[l];
    int n = L->A.n, nc = H->lev[l + 1].A.n;
    double *t = malloc(sizeof(double) * (size_t)n);
    double *r = malloc(sizeof(double) * (size_t)n);
    double *hc = malloc(sizeof(double) * (size_t)(nc > 0 ? nc : 1));
    double *gc = malloc(sizeof(double) * (size_t)(nc > 0 ? nc : 1));
    if (!transpose) {
        or_smooth(H, l, z, t, 0);
        or_spmv(n, L->A.rp, L->A.ci, L->A.v, t, r);
        for (int i = 0; i < n; ++i) r[i] = z[i] - r[i];
        or_restrict(H, l, r, hc);
        or_level_solve(H, l + 1, hc, gc, 0);
        for (int i = 0; i < n; ++i) q[i] = t[i] + gc[L->agg[i]];
    } else {
        /* B^{-T} = S^{-T}(I - A^T P C^T P^T) + P C^T P^T */
        or_restrict(H, l, z, hc);
        or_level_solve(H, l + 1, hc, gc, 1);
        for (int i = 0; i < n; ++i) t[i] = gc[L->agg[i]];
        or_spmv_t(n, L->A.rp, L->A.ci, L->A.v, t, r);
        for (int i = 0; i < n; ++i) r[i] = z[i] - r[i];
        or_smooth(H, l, r, q, 1);
        for (int i = 0; i < n; ++i) q[i] = t[i] + q[i];
    }
    free(t); free(r); free(hc); free(gc);
}

/* q = B~^{-1} z at level l (transpose: B~^{-T} z). */
void or_precond_level(const or_hier_t *H, int l, const double *z, double *q, int transpose)
{
    precond_level(H, l, z, q, transpose);
}

void or_precond(const or_hier_t *H, const double *z, double *q) { precond_level(H, 0, z, q, 0); }
void or_precond_t(const or_hier_t *H, const double *z, double *q) { precond_level(H, 0, z, q, 1); }

/* ------------------------------------------------------------------ */
/* O7. Right-preconditioned flexible GMRES(m) with modified Gram-       */
/* Schmidt and Givens rotations: the Krylov loop of Algorithm 1 with    */
/* the preconditioner applied on the right and the preconditioned       */
/* vectors z_j kept (x = x0 + Z y).  The stopping test is the relative  */
/* residual of Section 3: |s_{j+1}|/||b|| <= tol ends a cycle; the true */
/* ||b - A x||/||b|| decides convergence after the update, otherwise    */
/* the method restarts from x.  hist[0] = ||r0||/||b||, then one entry  */
/* per inner iteration across restarts.                                  */
/*   H == NULL: identity preconditioner on the CSR (rp, ci, v).          */
/*   transpose: operator A^T with preconditioner B~^{-T} (adjoint).      */
/* out_i[0] = iterations, out_i[1] = restarts, out_i[2] = hist length.  */
/* out_d[0] = true final relative residual.                              */
/* ------------------------------------------------------------------ */
/* Inner products of the Arnoldi process (dot products and norms) are    */
/* evaluated as if in twice the working precision, by the Dot2 algorithm */
/* of Ogita, Rump and Oishi (SIAM J. Sci. Comput. 26(6), 2005): each     */
/* product is split exactly into p + e (TwoProduct, via fma), the p are  */
/* summed with the exact error of every addition kept (TwoSum, Knuth),   */
/* and the collected errors are added at the end.  Reading: the paper    */
/* does not fix how inner products are rounded; an accurately rounded    */
/* value does not depend on the summation order, which a parallel        */
/* reduction cannot follow.                                              */
static void two_sum(double a, double b, double *s, double *e)
{
    double t = a + b;
    double z = t - a;
    *e = (a - (t - z)) + (b - z);
    *s = t;
}

static double dot2_strided(int n, const double *a, size_t stride, const double *b)
{
    double p = 0.0, c = 0.0;
    for (int i = 0; i < n; ++i) {
        double ai = a[(size_t)i * stride];
        double h = ai * b[i];
        double r = fma(ai, b[i], -h);           /* a_i b_i = h + r exactly */
        double q;
        two_sum(p, h, &p, &q);
        c = c + (q + r);
    }
    return p + c;
}

double or_dot(int n, const double *a, const double *b) { return dot2_strided(n, a, 1, b); }

static double dot(int n, const double *a, const double *b) { return or_dot(n, a, b); }

int or_fgmres(const or_hier_t *H, int n, const int64_t *rp, const int32_t *ci, const double *v,
              const double *b, double *x, double tol, int restart, int maxit, int transpose,
              double *hist, int hist_cap, int32_t *out_i, double *out_d)
{
    if (H) { n = H->lev[0].A.n; rp = H->lev[0].A.rp; ci = H->lev[0].A.ci; v = H->lev[0].A.v; }
    if (n <= 0 || restart < 1 || maxit < 0) return OR_EINVAL;
    int m = restart;
    double *V = malloc(sizeof(double) * (size_t)n * (size_t)(m + 1));
    double *Z = malloc(sizeof(double) * (size_t)n * (size_t)m);
    double *w = malloc(sizeof(double) * (size_t)n);
    double *Hm = calloc((size_t)(m + 1) * (size_t)m, sizeof(double));   /* Hm[k*m + j] = h_{k,j} */
    double *cs = malloc(sizeof(double) * (size_t)m), *sn = malloc(sizeof(double) * (size_t)m);
    double *s = malloc(sizeof(double) * (size_t)(m + 1)), *y = malloc(sizeof(double) * (size_t)m);
    int total = 0, restarts = 0, hlen = 0, status = OR_OK;
    double relres = 0.0;

    double bnorm = sqrt(dot(n, b, b));
    if (!isfinite(bnorm)) { status = OR_ENUMERIC; goto done; }
    if (bnorm == 0.0) {
        for (int i = 0; i < n; ++i) x[i] = 0.0;
        if (hist_cap > 0) hist[hlen++] = 0.0;
        goto done;
    }
    /* r0 = b - op(A) x0 */
    if (transpose) or_spmv_t(n, rp, ci, v, x, w); else or_spmv(n, rp, ci, v, x, w);
    for (int i = 0; i < n; ++i) w[i] = b[i] - w[i];
    double beta = sqrt(dot(n, w, w));
    relres = beta / bnorm;
    if (hist_cap > hlen) hist[hlen++] = relres;
    if (!isfinite(relres)) { status = OR_ENUMERIC; goto done; }
    for (;;) {
        if (relres <= tol) break;
        if (total >= maxit) { status = OR_ENOTCONV; break; }
        for (int i = 0; i < n; ++i) V[i] = w[i] / beta;
        for (int k = 0; k <= m; ++k) s[k] = 0.0;
        s[0] = beta;
        int j = 0, stop = 0;
        for (; j < m; ) {
            double *vj = V + (size_t)j * n, *zj = Z + (size_t)j * n;
            if (!H) memcpy(zj, vj, sizeof(double) * (size_t)n);
            else if (transpose) or_precond_t(H, vj, zj);
            else or_precond(H, vj, zj);
            if (transpose) or_spmv_t(n, rp, ci, v, zj, w); else or_spmv(n, rp, ci, v, zj, w);
            for (int k = 0; k <= j; ++k) {
                double *vk = V + (size_t)k * n;
                double hk = dot(n, w, vk);
                Hm[k * m + j] = hk;
                for (int i = 0; i < n; ++i) w[i] = fma(-hk, vk[i], w[i]);
            }
            double hn = sqrt(dot(n, w, w));
            Hm[(j + 1) * m + j] = hn;
            if (hn != 0.0) {
                double *vn = V + (size_t)(j + 1) * n;
                for (int i = 0; i < n; ++i) vn[i] = w[i] / hn;
            }
            for (int k = 0; k < j; ++k) {
                double a = Hm[k * m + j], c = Hm[(k + 1) * m + j];
                Hm[k * m + j] = fma(cs[k], a, sn[k] * c);
                Hm[(k + 1) * m + j] = fma(-sn[k], a, cs[k] * c);
            }
            double a = Hm[j * m + j], c = Hm[(j + 1) * m + j];
            double rho = sqrt(fma(a, a, c * c));
            if (rho == 0.0 || !isfinite(rho)) { status = OR_ENUMERIC; stop = 2; break; }
            cs[j] = a / rho; sn[j] = c / rho;
            Hm[j * m + j] = rho; Hm[(j + 1) * m + j] = 0.0;
            s[j + 1] = -sn[j] * s[j];
            s[j] = cs[j] * s[j];
            ++j; ++total;
            double est = fabs(s[j]) / bnorm;
            if (hist_cap > hlen) hist[hlen++] = est;
            if (!isfinite(est)) { status = OR_ENUMERIC; stop = 2; break; }
            if (est <= tol || hn == 0.0 || total >= maxit) { stop = 1; break; }
        }
        if (stop == 2) break;
        /* UPDATE: back-solve the j x j triangle, x += Z y */
        for (int k = j - 1; k >= 0; --k) {
            double t = s[k];
            for (int l = k + 1; l < j; ++l) t = fma(-Hm[k * m + l], y[l], t);
            y[k] = t / Hm[k * m + k];
        }
        for (int k = 0; k < j; ++k) {
            double *zk = Z + (size_t)k * n;
            for (int i = 0; i < n; ++i) x[i] = fma(y[k], zk[i], x[i]);
        }
        if (transpose) or_spmv_t(n, rp, ci, v, x, w); else or_spmv(n, rp, ci, v, x, w);
        for (int i = 0; i < n; ++i) w[i] = b[i] - w[i];
        beta = sqrt(dot(n, w, w));
        relres = beta / bnorm;
        if (!isfinite(relres)) { status = OR_ENUMERIC; break; }
        if (relres <= tol) break;
        if (total >= maxit) { status = OR_ENOTCONV; break; }
        ++restarts;
    }
done:
    out_i[0] = total; out_i[1] = restarts; out_i[2] = hlen;
    out_d[0] = relres;
    free(V); free(Z); free(w); free(Hm); free(cs); free(sn); free(s); free(y);
    return status;
}
