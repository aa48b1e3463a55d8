// Host-side validation and layout of one problem instance (the primal SDP
// min <C,X> s.t. <A_k,X> = b_k of Sec. 2, constraints given as triplets):
// the checks of lorads_create and the derived arrays every solver uploads.
#pragma once

#include <stdint.h>
#include <string>
#include <vector>

#include "../../include/lorads.h"
#include "dfloat.cuh"

namespace lorads {

struct HostProb {
    int64_t n = 0, m = 0, nnz_c = 0, m_diag = 0, m_off = 0, nnz_aoff = 0;
    double cnorm1 = 0, mean_abs_c = 1, bnorm_inf = 0, bnorm1 = 0;
    // C as given (caller's arrays, not copied) plus its FP32 and double-float mirrors
    const int64_t* rp = nullptr;
    const int32_t* ci = nullptr;
    const double* cv = nullptr;
    const double* b = nullptr;
    std::vector<float> cv32;
    std::vector<dfloat> cvdf;
    // diagonal constraints by row (empty when there are none)
    std::vector<int32_t> dk;
    std::vector<double> da;
    std::vector<float> da32;
    std::vector<dfloat> dadf;
    std::vector<dfloat> bdf;
    // off-diagonal constraint pattern, symmetric, columns sorted within a row
    std::vector<int64_t> a_rp;
    std::vector<int32_t> a_col, a_k;
    std::vector<double> a_a;
    // constraint list: fused diagonal constraints by row, then the others by the entry
    // of their first triplet.  k_id: constraint of each list position.  k_row, k_col,
    // k_a: the triplets in list order; with k_ptr (general form: a constraint with
    // several triplets, or several constraints on one entry) position q owns triplets
    // k_ptr[q] .. k_ptr[q+1]-1, otherwise position q is triplet q.
    std::vector<int32_t> k_row, k_col, k_id;
    std::vector<double> k_a;
    std::vector<int64_t> k_ptr;
    // double-float mirrors of k_a and a_a
    std::vector<dfloat> k_adf, a_adf;
};

// Validates the inputs of lorads_create and fills `hp`.  On failure returns the
// status and sets `*err`; no device call is made.
lorads_status build_host_prob(HostProb* hp, std::string* err, int64_t n, const int64_t* rp, const int32_t* ci,
                              const double* cv, int64_t m, int64_t nnz_a, const int32_t* acon, const int32_t* arow,
                              const int32_t* acol, const double* aval, const double* b);

// Checks the solver constants of `p` against their documented ranges.  Returns an
// empty string when every value is usable, else a message naming the first bad one.
std::string solver_params_error(const lorads_params& p);

}  // namespace lorads
