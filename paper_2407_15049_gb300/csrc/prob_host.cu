// Host-side validation and layout of one problem instance (see prob_host.h).
#include <algorithm>
#include <cmath>
#include <thread>
#include <utility>

#include "common.cuh"
#include "prob_host.h"

namespace lorads {

namespace {

// Symmetry of C: every stored (i, j, v) has a stored (j, i, v).  The lookups jump
// across the whole column array (a cache miss each on large graphs), so the rows are
// checked in contiguous ranges by several threads; each range reports its first
// failure and the lowest failing row is returned (-1: symmetric), whatever the
// thread count.
int64_t first_asymmetric_row(int64_t n, const int64_t* rp, const int32_t* ci, const double* cv, int32_t* bad_col) {
    unsigned nt = std::thread::hardware_concurrency();
    nt = std::max(1u, std::min(nt, 32u));
    if (rp[n] < (int64_t(1) << 22)) nt = 1;
    std::vector<int64_t> first(nt, -1);
    std::vector<int32_t> col(nt, -1);
    auto check = [&](unsigned t) {
        const int64_t r0 = n * (int64_t)t / nt, r1 = n * (int64_t)(t + 1) / nt;
        for (int64_t i = r0; i < r1; ++i) {
            for (int64_t s = rp[i]; s < rp[i + 1]; ++s) {
                const int32_t j = ci[s];
                const int32_t* lo = ci + rp[j];
                const int32_t* hi = ci + rp[j + 1];
                const int32_t* f = std::lower_bound(lo, hi, (int32_t)i);
                if (f == hi || *f != i || cv[f - ci] != cv[s]) {
                    first[t] = i;
                    col[t] = j;
                    return;
                }
            }
        }
    };
    std::vector<std::thread> pool;
    for (unsigned t = 1; t < nt; ++t) pool.emplace_back(check, t);
    check(0);
    for (auto& th : pool) th.join();
    for (unsigned t = 0; t < nt; ++t)
        if (first[t] >= 0) {
            *bad_col = col[t];
            return first[t];
        }
    return -1;
}

}  // namespace

lorads_status build_host_prob(HostProb* hp, std::string* err, int64_t n, const int64_t* rp, const int32_t* ci,
                              const double* cv, int64_t m, int64_t nnz_a, const int32_t* acon, const int32_t* arow,
                              const int32_t* acol, const double* aval, const double* b) {
    auto set_err = [&](const std::string& msg) { *err = msg; return false; };
    if (n < 1 || n > INT32_MAX) return set_err("n must be in [1, 2^31)"), LORADS_ERR_INVALID_ARG;
    if (m < 1 || m > INT32_MAX) return set_err("m must be in [1, 2^31)"), LORADS_ERR_INVALID_ARG;
    if (!rp || !ci || !cv || !acon || !arow || !acol || !aval || !b)
        return set_err("null input pointer"), LORADS_ERR_INVALID_ARG;
    if (rp[0] != 0) return set_err("c_rowptr[0] must be 0"), LORADS_ERR_INVALID_ARG;
    for (int64_t i = 0; i < n; ++i)
        if (rp[i + 1] < rp[i]) return set_err("c_rowptr must be nondecreasing"), LORADS_ERR_INVALID_ARG;
    const int64_t nnz = rp[n];
    double sum_abs = 0.0;
    int64_t cnt_nz = 0;
    for (int64_t i = 0; i < n; ++i) {
        for (int64_t s = rp[i]; s < rp[i + 1]; ++s) {
            const int32_t j = ci[s];
            if (j < 0 || j >= n) return set_err("C column index out of range at row " + std::to_string(i)), LORADS_ERR_INVALID_ARG;
            if (s > rp[i] && ci[s - 1] >= j)
                return set_err("C column indices must be sorted and distinct within row " + std::to_string(i)),
                       LORADS_ERR_INVALID_ARG;
            if (!std::isfinite(cv[s])) return set_err("non-finite value in C"), LORADS_ERR_INVALID_ARG;
            if (cv[s] != 0.0) { sum_abs += std::fabs(cv[s]); ++cnt_nz; }
        }
    }
    // symmetry: (i, j, v) needs (j, i, v)
    {
        int32_t j = -1;
        const int64_t i = first_asymmetric_row(n, rp, ci, cv, &j);
        if (i >= 0)
            return set_err("C is not symmetric at (" + std::to_string(i) + "," + std::to_string(j) + ")"),
                   LORADS_ERR_NOT_SYMMETRIC;
    }
    hp->cnorm1 = sum_abs;
    hp->mean_abs_c = cnt_nz ? sum_abs / (double)cnt_nz : 1.0;
    // constraints: validate every triplet, then group the triplets by constraint
    if (nnz_a < m) return set_err("every constraint needs at least one triplet (nnz_a >= m)"), LORADS_ERR_INVALID_ARG;
    std::vector<int64_t> kstart(m + 1, 0);
    for (int64_t t = 0; t < nnz_a; ++t) {
        const int32_t k = acon[t], i = arow[t], j = acol[t];
        if (k < 0 || k >= m) return set_err("a_con out of range"), LORADS_ERR_INVALID_ARG;
        if (i < 0 || j < 0 || i >= n || j >= n || i > j)
            return set_err("constraint triplet needs 0 <= a_row <= a_col < n"), LORADS_ERR_INVALID_ARG;
        if (!std::isfinite(aval[t]) || aval[t] == 0.0)
            return set_err("constraint coefficient must be finite and nonzero"), LORADS_ERR_INVALID_ARG;
        kstart[k + 1]++;
    }
    for (int64_t k = 0; k < m; ++k) {
        if (kstart[k + 1] == 0) return set_err("constraint " + std::to_string(k) + " has no triplet"), LORADS_ERR_INVALID_ARG;
        kstart[k + 1] += kstart[k];
    }
    std::vector<int32_t> trip(nnz_a);           // triplet ids grouped by constraint, input order within
    {
        std::vector<int64_t> fill(kstart.begin(), kstart.end() - 1);
        for (int64_t t = 0; t < nnz_a; ++t) trip[fill[acon[t]]++] = (int32_t)t;
    }
    // two triplets of one constraint on the same entry are one entry with the summed coefficient
    for (int64_t k = 0; k < m; ++k) {
        if (kstart[k + 1] - kstart[k] < 2) continue;
        std::vector<int64_t> keys;
        for (int64_t q = kstart[k]; q < kstart[k + 1]; ++q) keys.push_back((int64_t)arow[trip[q]] * n + acol[trip[q]]);
        std::sort(keys.begin(), keys.end());
        if (std::adjacent_find(keys.begin(), keys.end()) != keys.end())
            return set_err("constraint " + std::to_string(k) + " lists one entry twice"), LORADS_ERR_INVALID_ARG;
    }
    double bmax = 0.0, b1 = 0.0;
    for (int64_t k = 0; k < m; ++k) {
        if (!std::isfinite(b[k])) return set_err("non-finite b"), LORADS_ERR_INVALID_ARG;
        bmax = std::max(bmax, std::fabs(b[k]));
        b1 += std::fabs(b[k]);
    }
    hp->bnorm_inf = bmax;
    hp->bnorm1 = b1;
    // General form (Sec. 4.5: constraints with several entries, or several constraints
    // on one entry): constraint list positions carry triplet ranges (k_ptr).  Otherwise
    // every constraint is one triplet and position = triplet.
    bool general = nnz_a > m;
    // diagonal constraints of one triplet, at most one per row: fused into the row passes
    std::vector<int32_t> dk(n, -1);
    std::vector<double> da(n, 0.0);
    std::vector<char> fused(m, 0);
    int64_t m_diag = 0;
    for (int64_t k = 0; k < m; ++k) {
        if (kstart[k + 1] - kstart[k] != 1) continue;
        const int32_t t = trip[kstart[k]];
        const int32_t i = arow[t];
        if (i != acol[t]) continue;
        if (dk[i] >= 0) {
            general = true;                     // a second one on this row stays in the list
            continue;
        }
        dk[i] = (int32_t)k;
        da[i] = aval[t];
        fused[k] = 1;
        ++m_diag;
    }
    const int64_t m_off = m - m_diag;
    // the other constraints, ordered by the entry of their first triplet
    std::vector<std::pair<int64_t, int32_t>> off;
    off.reserve(m_off);
    for (int64_t k = 0; k < m; ++k)
        if (!fused[k]) {
            const int32_t t = trip[kstart[k]];
            off.emplace_back((int64_t)arow[t] * n + acol[t], (int32_t)k);
        }
    std::sort(off.begin(), off.end());
    for (size_t q = 1; q < off.size() && !general; ++q)
        if (off[q].first == off[q - 1].first) general = true;     // several constraints on one entry
    // ordered constraint list: fused diagonal constraints by row, then the others
    std::vector<int32_t> order;
    order.reserve(m);
    for (int64_t i = 0; i < n; ++i)
        if (dk[i] >= 0) order.push_back(dk[i]);
    for (auto& pr : off) order.push_back(pr.second);
    // triplets in list order; k_ptr (general form) maps a list position to its range
    std::vector<int32_t> k_row, k_col, k_id(m);
    std::vector<double> k_a;
    std::vector<int64_t> k_ptr;
    if (general) k_ptr.assign(m + 1, 0);
    for (int64_t q = 0; q < m; ++q) {
        const int32_t k = order[q];
        k_id[q] = k;
        for (int64_t u = kstart[k]; u < kstart[k + 1]; ++u) {
            const int32_t t = trip[u];
            k_row.push_back(arow[t]);
            k_col.push_back(acol[t]);
            k_a.push_back(aval[t]);
        }
        if (general) k_ptr[q + 1] = (int64_t)k_row.size();
    }
    // pattern of the listed constraints (symmetric, sorted by column within a row):
    // slot (row i, column j) per entry of A_k, i.e. two per off-diagonal triplet and
    // one per diagonal triplet (general form only)
    std::vector<int64_t> a_rp(n + 1, 0);
    std::vector<int32_t> a_col, a_k;
    std::vector<double> a_a;
    if (m_off > 0) {
        const int64_t t0 = general ? k_ptr[m_diag] : m_diag;
        const int64_t t1 = (int64_t)k_row.size();
        for (int64_t t = t0; t < t1; ++t) {
            a_rp[k_row[t] + 1]++;
            if (k_row[t] != k_col[t]) a_rp[k_col[t] + 1]++;
        }
        for (int64_t i = 0; i < n; ++i) a_rp[i + 1] += a_rp[i];
        const int64_t nz = a_rp[n];
        a_col.resize(nz);
        a_k.resize(nz);
        a_a.resize(nz);
        std::vector<int64_t> fill(a_rp.begin(), a_rp.end() - 1);
        int64_t q = m_diag;
        for (int64_t t = t0; t < t1; ++t) {
            if (general) {
                while (k_ptr[q + 1] <= t) ++q;
            } else {
                q = t;
            }
            const int32_t i = k_row[t], j = k_col[t];
            int64_t s = fill[i]++;
            a_col[s] = j; a_k[s] = k_id[q]; a_a[s] = k_a[t];
            if (i != j) {
                s = fill[j]++;
                a_col[s] = i; a_k[s] = k_id[q]; a_a[s] = k_a[t];
            }
        }
        // sort each row by column
        std::vector<int64_t> idx;
        for (int64_t i = 0; i < n; ++i) {
            const int64_t s0 = a_rp[i], s1 = a_rp[i + 1];
            if (s1 - s0 < 2) continue;
            idx.resize(s1 - s0);
            for (int64_t u = 0; u < s1 - s0; ++u) idx[u] = s0 + u;
            std::sort(idx.begin(), idx.end(), [&](int64_t x, int64_t y) { return a_col[x] < a_col[y]; });
            std::vector<int32_t> tc(s1 - s0), tk(s1 - s0);
            std::vector<double> ta(s1 - s0);
            for (int64_t u = 0; u < s1 - s0; ++u) { tc[u] = a_col[idx[u]]; tk[u] = a_k[idx[u]]; ta[u] = a_a[idx[u]]; }
            for (int64_t u = 0; u < s1 - s0; ++u) { a_col[s0 + u] = tc[u]; a_k[s0 + u] = tk[u]; a_a[s0 + u] = ta[u]; }
        }
        hp->nnz_aoff = nz;
    }
    hp->k_ptr = std::move(k_ptr);
    hp->n = n; hp->m = m; hp->nnz_c = nnz; hp->m_diag = m_diag; hp->m_off = m_off;
    hp->rp = rp; hp->ci = ci; hp->cv = cv; hp->b = b;
    hp->cv32.assign(cv, cv + nnz);
    hp->cvdf.resize(nnz);
    for (int64_t q = 0; q < nnz; ++q) {
        const float h = (float)cv[q];
        hp->cvdf[q] = dfloat(h, (float)(cv[q] - (double)h));
    }
    if (m_diag > 0) {
        hp->da32.resize(n);
        hp->dadf.resize(n);
        for (int64_t i = 0; i < n; ++i) {
            hp->da32[i] = (float)da[i];
            hp->dadf[i] = dfloat(hp->da32[i], (float)(da[i] - (double)hp->da32[i]));
        }
        hp->dk = std::move(dk);
        hp->da = std::move(da);
    }
    hp->bdf.resize(m);
    for (int64_t k = 0; k < m; ++k) {
        const float h = (float)b[k];
        hp->bdf[k] = dfloat(h, (float)(b[k] - (double)h));
    }
    if (m_off > 0) {
        hp->a_rp = std::move(a_rp);
        hp->a_col = std::move(a_col);
        hp->a_k = std::move(a_k);
        hp->a_a = std::move(a_a);
    }
    hp->k_row = std::move(k_row);
    hp->k_col = std::move(k_col);
    hp->k_a = std::move(k_a);
    hp->k_id = std::move(k_id);
    auto split = [](double v) {
        const float h = (float)v;
        return dfloat(h, (float)(v - (double)h));
    };
    hp->k_adf.resize(hp->k_a.size());
    for (size_t q = 0; q < hp->k_a.size(); ++q) hp->k_adf[q] = split(hp->k_a[q]);
    hp->a_adf.resize(hp->a_a.size());
    for (size_t q = 0; q < hp->a_a.size(); ++q) hp->a_adf[q] = split(hp->a_a[q]);
    return LORADS_OK;
}

std::string solver_params_error(const lorads_params& p) {
    auto finite = [](double v) { return std::isfinite(v); };
    if (p.lbfgs_mem < 1 || p.lbfgs_mem > kMaxMem) return "lbfgs_mem must be in [1, 4]";
    if (!(p.tol > 0.0) || !finite(p.tol)) return "tol must be finite and > 0";
    if (!(p.time_limit > 0.0)) return "time_limit must be > 0";
    if (p.max_inner < 1 || p.max_outer < 1) return "max_inner and max_outer must be >= 1";
    if (p.rank_update_threshold < 1) return "rank_update_threshold must be >= 1";
    if (!finite(p.rho0)) return "rho0 must be finite (<= 0 selects the automatic value)";
    if (!(p.rho_growth >= 1.0) || !finite(p.rho_growth)) return "rho_growth must be finite and >= 1";
    if (!(p.rho_max > 0.0)) return "rho_max must be > 0";
    if (!(p.infeas_decrease >= 0.0) || !finite(p.infeas_decrease)) return "infeas_decrease must be finite and >= 0";
    if (!(p.inner_rel > 0.0) || !finite(p.inner_rel) || !(p.inner_progress > 0.0) || !finite(p.inner_progress))
        return "inner_rel and inner_progress must be finite and > 0";
    if (p.lanczos_steps < 1) return "lanczos_steps must be >= 1";
    if (p.lbfgs_scaling < 0 || p.lbfgs_scaling > 1) return "lbfgs_scaling must be 0 or 1";
    if (p.rho_policy < 0 || p.rho_policy > 2) return "rho_policy must be 0, 1 or 2";
    if (p.inner_scale < 0 || p.inner_scale > 2) return "inner_scale must be 0, 1 or 2";
    if (!(p.admm_switch >= 0.0) || !(p.cg_rel > 0.0 && p.cg_rel < 1.0) || p.cg_max < 1 || p.admm_max_iter < 0)
        return "need admm_switch >= 0, 0 < cg_rel < 1, cg_max >= 1 and admm_max_iter >= 0";
    if (p.reopt_level < 0 || p.reopt_level > 2 || p.max_reopt < 0 || !(p.reopt_factor > 0.0 && p.reopt_factor < 1.0))
        return "need reopt_level in [0, 2], max_reopt >= 0 and 0 < reopt_factor < 1";
    return std::string();
}

}  // namespace lorads
