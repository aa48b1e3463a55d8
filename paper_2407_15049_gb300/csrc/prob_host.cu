// Host-side validation and layout of one problem instance (see prob_host.h).
#include <algorithm>
#include <cmath>
#include <utility>

#include "prob_host.h"

namespace lorads {

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
    for (int64_t i = 0; i < n; ++i) {
        for (int64_t s = rp[i]; s < rp[i + 1]; ++s) {
            const int32_t j = ci[s];
            const int32_t* lo = ci + rp[j];
            const int32_t* hi = ci + rp[j + 1];
            const int32_t* f = std::lower_bound(lo, hi, (int32_t)i);
            if (f == hi || *f != i || cv[f - ci] != cv[s])
                return set_err("C is not symmetric at (" + std::to_string(i) + "," + std::to_string(j) + ")"),
                       LORADS_ERR_NOT_SYMMETRIC;
        }
    }
    hp->cnorm1 = sum_abs;
    hp->mean_abs_c = cnt_nz ? sum_abs / (double)cnt_nz : 1.0;
    // constraints
    if (nnz_a != m)
        return set_err("every constraint must be a single triplet (nnz_a == m); constraints with several "
                            "entries are not supported"),
               LORADS_ERR_UNSUPPORTED;
    std::vector<int32_t> seen(m, 0);
    std::vector<int32_t> trip_of(m, -1);
    for (int64_t t = 0; t < nnz_a; ++t) {
        const int32_t k = acon[t], i = arow[t], j = acol[t];
        if (k < 0 || k >= m) return set_err("a_con out of range"), LORADS_ERR_INVALID_ARG;
        if (i < 0 || j < 0 || i >= n || j >= n || i > j)
            return set_err("constraint triplet needs 0 <= a_row <= a_col < n"), LORADS_ERR_INVALID_ARG;
        if (!std::isfinite(aval[t]) || aval[t] == 0.0)
            return set_err("constraint coefficient must be finite and nonzero"), LORADS_ERR_INVALID_ARG;
        if (seen[k]++) return set_err("constraint with several triplets"), LORADS_ERR_UNSUPPORTED;
        trip_of[k] = (int32_t)t;
    }
    double bmax = 0.0, b1 = 0.0;
    for (int64_t k = 0; k < m; ++k) {
        if (!std::isfinite(b[k])) return set_err("non-finite b"), LORADS_ERR_INVALID_ARG;
        bmax = std::max(bmax, std::fabs(b[k]));
        b1 += std::fabs(b[k]);
    }
    hp->bnorm_inf = bmax;
    hp->bnorm1 = b1;
    // diagonal constraints by row
    std::vector<int32_t> dk(n, -1);
    std::vector<double> da(n, 0.0);
    int64_t m_diag = 0;
    std::vector<int64_t> offkeys;
    for (int64_t k = 0; k < m; ++k) {
        const int32_t t = trip_of[k];
        const int32_t i = arow[t], j = acol[t];
        if (i == j) {
            if (dk[i] >= 0) return set_err("two constraints on the same diagonal entry"), LORADS_ERR_UNSUPPORTED;
            dk[i] = (int32_t)k;
            da[i] = aval[t];
            ++m_diag;
        }
    }
    const int64_t m_off = m - m_diag;
    // ordered constraint list: diagonal constraints by row, then off-diagonal by (row, col)
    std::vector<int32_t> order;
    order.reserve(m);
    for (int64_t i = 0; i < n; ++i)
        if (dk[i] >= 0) order.push_back(dk[i]);
    {
        std::vector<std::pair<int64_t, int32_t>> off;
        off.reserve(m_off);
        for (int64_t k = 0; k < m; ++k) {
            const int32_t t = trip_of[k];
            if (arow[t] != acol[t]) off.emplace_back((int64_t)arow[t] * n + acol[t], (int32_t)k);
        }
        std::sort(off.begin(), off.end());
        for (size_t q = 1; q < off.size(); ++q)
            if (off[q].first == off[q - 1].first)
                return set_err("two constraints on the same off-diagonal entry"), LORADS_ERR_UNSUPPORTED;
        for (auto& pr : off) order.push_back(pr.second);
    }
    std::vector<int32_t> k_row(m), k_col(m), k_id(m);
    std::vector<double> k_a(m);
    for (int64_t q = 0; q < m; ++q) {
        const int32_t k = order[q];
        const int32_t t = trip_of[k];
        k_row[q] = arow[t];
        k_col[q] = acol[t];
        k_a[q] = aval[t];
        k_id[q] = k;
    }
    // off-diagonal constraint pattern (symmetric, sorted by column within a row)
    std::vector<int64_t> a_rp(n + 1, 0);
    std::vector<int32_t> a_col, a_k;
    std::vector<double> a_a;
    if (m_off > 0) {
        for (int64_t q = m_diag; q < m; ++q) {
            a_rp[k_row[q] + 1]++;
            a_rp[k_col[q] + 1]++;
        }
        for (int64_t i = 0; i < n; ++i) a_rp[i + 1] += a_rp[i];
        const int64_t nz = a_rp[n];
        a_col.resize(nz);
        a_k.resize(nz);
        a_a.resize(nz);
        std::vector<int64_t> fill(a_rp.begin(), a_rp.end() - 1);
        for (int64_t q = m_diag; q < m; ++q) {
            const int32_t i = k_row[q], j = k_col[q];
            int64_t s = fill[i]++;
            a_col[s] = j; a_k[s] = k_id[q]; a_a[s] = k_a[q];
            s = fill[j]++;
            a_col[s] = i; a_k[s] = k_id[q]; a_a[s] = k_a[q];
        }
        // sort each row by column
        std::vector<int64_t> idx;
        for (int64_t i = 0; i < n; ++i) {
            const int64_t s0 = a_rp[i], s1 = a_rp[i + 1];
            if (s1 - s0 < 2) continue;
            idx.resize(s1 - s0);
            for (int64_t q = 0; q < s1 - s0; ++q) idx[q] = s0 + q;
            std::sort(idx.begin(), idx.end(), [&](int64_t x, int64_t y) { return a_col[x] < a_col[y]; });
            std::vector<int32_t> tc(s1 - s0), tk(s1 - s0);
            std::vector<double> ta(s1 - s0);
            for (int64_t q = 0; q < s1 - s0; ++q) { tc[q] = a_col[idx[q]]; tk[q] = a_k[idx[q]]; ta[q] = a_a[idx[q]]; }
            for (int64_t q = 0; q < s1 - s0; ++q) { a_col[s0 + q] = tc[q]; a_k[s0 + q] = tk[q]; a_a[s0 + q] = ta[q]; }
        }
        hp->nnz_aoff = nz;
    }
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

}  // namespace lorads
