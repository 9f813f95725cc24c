// ilut.cu -- ILUT(tau) of the coarse operator on the host (Section 2 of the
// paper: the inexact coarse factorisation A~_c = L~_c U~_c = ILUT(A_c), as in
// the setup phase of Algorithm 1).
//
// Dropping rule of Saad's ILUT with a threshold only (no cap on the entries
// per row) and no pivoting; natural order.  Row i, with tau_i = tau ||a_i||_2
// (squares summed in stored column order):
//   w = a_i; for each k < i stored in w, in increasing k (fill included):
//     w_k = w_k / u_kk; dropped when it is 0 or below tau_i, otherwise
//     w_j -= w_k u_kj for every stored u_kj, j > k;
//   L~ keeps the surviving w_k, U~ keeps w_i and every w_j (j > i) that is
//   nonzero and at least tau_i.
// Setup arithmetic: each product and each difference is rounded on its own
// (host code is compiled without floating-point contraction), so the
// factors do not depend on the machine the library runs on.
//
// The factorisation is sequential and data-dependent (which entries survive
// depends on the values), so it runs on the host; the triangular solves with
// its factors are the same sparse sweeps as ILU(0)'s.
#include "internal.cuh"
#include "../../include/amg.h"

#include <algorithm>
#include <cmath>
#include <functional>
#include <queue>
#include <vector>

namespace amg {

struct IlutHost {
    std::vector<int64_t> rp;   // [n+1]
    std::vector<int32_t> ci;
    std::vector<double> v;
    bool breakdown = false;
};

static void ilut_factor_host(int n, const int64_t *rp, const int32_t *ci, const double *val, double tau,
                             IlutHost &F) {
    F.rp.assign((size_t)n + 1, 0);
    F.ci.clear();
    F.v.clear();
    F.breakdown = false;
    std::vector<int64_t> diag((size_t)n, -1);   // index of u_kk in F
    std::vector<double> w((size_t)n, 0.0);
    std::vector<int> stamp((size_t)n, -1);
    std::vector<int32_t> touched;
    std::priority_queue<int32_t, std::vector<int32_t>, std::greater<int32_t>> pending;   // L columns
    for (int i = 0; i < n; ++i) {
        double sq = 0.0;
        for (int64_t e = rp[i]; e < rp[i + 1]; ++e) {
            const double p = val[e] * val[e];
            sq = sq + p;
        }
        const double ti = tau * std::sqrt(sq);
        touched.clear();
        for (int64_t e = rp[i]; e < rp[i + 1]; ++e) {
            const int32_t j = ci[e];
            stamp[j] = i;
            w[j] = val[e];
            touched.push_back(j);
            if (j < i) pending.push(j);
        }
        if (stamp[i] != i) {
            stamp[i] = i;
            w[i] = 0.0;
            touched.push_back(i);
        }
        while (!pending.empty()) {
            const int32_t k = pending.top();
            pending.pop();
            const double wk = w[k] / F.v[(size_t)diag[k]];
            if (wk == 0.0 || std::fabs(wk) < ti) {
                w[k] = 0.0;
                continue;
            }
            w[k] = wk;
            for (int64_t e = diag[k] + 1; e < F.rp[(size_t)k + 1]; ++e) {
                const int32_t j = F.ci[(size_t)e];
                if (stamp[j] != i) {
                    stamp[j] = i;
                    w[j] = 0.0;
                    touched.push_back(j);
                    if (j < i) pending.push(j);
                }
                const double p = wk * F.v[(size_t)e];
                w[j] = w[j] - p;
            }
        }
        std::sort(touched.begin(), touched.end());
        for (const int32_t j : touched) {
            const double x = w[j];
            bool keep;
            if (j < i) keep = x != 0.0;
            else if (j == i) keep = true;
            else keep = x != 0.0 && !(std::fabs(x) < ti);
            if (j == i) {
                diag[i] = (int64_t)F.ci.size();
                if (x == 0.0 || !std::isfinite(x)) F.breakdown = true;
            }
            if (keep) {
                F.ci.push_back(j);
                F.v.push_back(x);
            }
            w[j] = 0.0;
        }
        F.rp[(size_t)i + 1] = (int64_t)F.ci.size();
    }
}

bool ilut_factor_host(int n, const int64_t *rp, const int32_t *ci, const double *val, double tau,
                      std::vector<int64_t> &frp, std::vector<int32_t> &fci, std::vector<double> &fv) {
    IlutHost F;
    ilut_factor_host(n, rp, ci, val, tau, F);
    frp.swap(F.rp);
    fci.swap(F.ci);
    fv.swap(F.v);
    return !F.breakdown;
}

}  // namespace amg

extern "C" int amg_ilut_host(int32_t n, const int64_t *row_ptr, const int32_t *col, const double *val, double tau,
                             int64_t cap, int64_t *f_row_ptr, int32_t *f_col, double *f_val, int64_t *f_nnz) {
    if (n < 0 || !row_ptr || !f_row_ptr || !f_nnz || !(tau >= 0.0) || cap < 0 || (cap > 0 && (!f_col || !f_val)))
        return AMG_ERR_INVALID_ARG;
    if (n > 0 && (!col || !val)) return AMG_ERR_INVALID_ARG;
    if (row_ptr[0] != 0) return AMG_ERR_INVALID_ARG;
    for (int i = 0; i < n; ++i) {
        if (row_ptr[i + 1] < row_ptr[i]) return AMG_ERR_INVALID_ARG;
        bool has_diag = false;
        for (int64_t e = row_ptr[i]; e < row_ptr[i + 1]; ++e) {
            if (col[e] < 0 || col[e] >= n || (e > row_ptr[i] && col[e] <= col[e - 1])) return AMG_ERR_INVALID_ARG;
            has_diag = has_diag || col[e] == i;
        }
        if (!has_diag) return AMG_ERR_INVALID_ARG;
    }
    amg::IlutHost F;
    try {
        amg::ilut_factor_host(n, row_ptr, col, val, tau, F);
    } catch (const std::bad_alloc &) {
        return AMG_ERR_OOM;
    }
    const int64_t nnz = (int64_t)F.ci.size();
    *f_nnz = nnz;
    if (nnz > cap) return AMG_ERR_LIMIT;
    std::copy(F.rp.begin(), F.rp.end(), f_row_ptr);
    std::copy(F.ci.begin(), F.ci.end(), f_col);
    std::copy(F.v.begin(), F.v.end(), f_val);
    return F.breakdown ? AMG_ERR_BREAKDOWN : AMG_OK;
}
