// Kernels of the splitting (ADMM) stage of Sec. 2.2.
//
// With X = U V^T and the Lagrangian of Eq. (1.3) (multiplier y = -lambda of
// the paper's body), each block step of Eq. (2.2) is the linear system of
// Eq. (2.3); for the U step (V fixed)
//     frakA_V(X) = rho A*(A(X V^T)) V + rho X,
//     frakb_V    = -C V + A*(y) V + rho A*(b) V + rho V,
// solved by the conjugate gradients of Algorithm 2 from the current iterate.
// The V step is the same system with U and V exchanged (C, A_k symmetric).
//
// The residual of Algorithm 2's start folds into one sparse pass:
//     frakb_V - frakA_V(X) = -(C - A*(w)) V + rho (V - X),
//     w = y - rho (A(X V^T) - b)                  (an m-vector, like y~),
// and <p, frakA_V(p)> = rho (||A(p V^T)||^2 + ||p||^2), because
// <p, A*(v) V> = <A(p V^T), v>: no pass over Q is needed for the CG step size.
//
// Types: TR stores the block iterates U, V (double, double-float or float),
// TW the CG vectors r, p, Q (double, float or double-float).  Per-constraint
// scalars are double on the all-FP64 path, double-float otherwise.
#pragma once

#include <type_traits>
#include "admm.h"
#include "kernels.cuh"

namespace lorads {

// partial-sum slots
enum { PA_RR = 0, PA_N = 1 };                       // ||r||^2
enum { PQ_PP = 0, PQ_WW = 1, PQ_N = 2 };            // ||p||^2, ||A(p V^T)||^2
enum { PY_ZZ = 0, PY_BY = 1, PY_N = 2 };            // ||A(U V^T) - b||^2, b^T y_new

template <typename TR>
using admm_cs_t = std::conditional_t<std::is_same_v<arith_t<TR>, double>, double, dfloat>;

// Lanes of the calling lane's row group (groups of L lanes, L a power of two).
__device__ __forceinline__ unsigned group_lanes(int L) {
    if (L >= 32) return 0xffffffffu;
    const int g = (threadIdx.x & 31) / L;
    return ((1u << L) - 1u) << (g * L);
}
__device__ __forceinline__ float shfl_xor_in(float v, int o, unsigned m) { return __shfl_xor_sync(m, v, o); }
__device__ __forceinline__ double shfl_xor_in(double v, int o, unsigned m) { return __shfl_xor_sync(m, v, o); }
__device__ __forceinline__ dfloat shfl_xor_in(dfloat v, int o, unsigned m) {
    return dfloat(__shfl_xor_sync(m, v.hi, o), __shfl_xor_sync(m, v.lo, o));
}

template <typename CS>
__device__ __forceinline__ CS ld_cs(const double* d, const dfloat* df, int64_t k) {
    if constexpr (std::is_same_v<CS, double>) return __ldg(d + k);
    else return df ? ld_scalar<dfloat>(d, df, k) : dfloat(__ldg(d + k));
}

// ------------------------------------------------------------------ control (one thread)
// Algorithm 2's start: ||r_0|| and the stop threshold eps = cg_rel ||r_0||.
__device__ inline void admm_cg_init_apply(AdmmCtrl* ac, double rr) {
    ac->cg_k = 0;
    ac->rr = rr;
    ac->eps = ac->cg_rel * sqrt(fmax(rr, 0.0));
    if (!isfinite(rr)) {
        ac->cg_active = 0;
        ac->status = 5;                     // LORADS_ERR_NUMERIC
        ac->done = 1;
        return;
    }
    // Algorithm 2 returns the start when its residual already meets the test
    ac->cg_active = (sqrt(fmax(rr, 0.0)) > ac->eps && rr > 0.0) ? 1 : 0;
}

// alpha = <r,r> / <p, frakA_V(p)>, <p, frakA_V(p)> = rho (||p||^2 + ||A(p V^T)||^2)
__device__ inline void admm_alpha_apply(AdmmCtrl* ac, double pp, double ww) {
    const double pq = ac->rho * (pp + ww);
    const double alpha = ac->rr / pq;
    if (!(pq > 0.0) || !isfinite(alpha)) {
        ac->cg_active = 0;                  // no positive curvature left: keep the iterate
        return;
    }
    ac->alpha = alpha;
}

// ||r_new||: the stop test, else beta = <r_new, r_new> / <r, r>
__device__ inline void admm_beta_apply(AdmmCtrl* ac, double rr_new) {
    ac->cg_k += 1;
    ac->cg_total += 1;
    if (!isfinite(rr_new)) {
        ac->cg_active = 0;
        ac->status = 5;
        ac->done = 1;
        return;
    }
    if (sqrt(fmax(rr_new, 0.0)) <= ac->eps || ac->cg_k >= ac->cg_max) {
        ac->cg_active = 0;
        return;
    }
    ac->beta = rr_new / ac->rr;
    ac->rr = rr_new;
}

// After the multiplier step and R = (U + V)/2: err1 and err3 of Sec. 4.2 at R
// (zz = ||A(RR^T) - b||^2, by = b^T y, obj = <C R, R>), the stop test and the cap.
__device__ inline void admm_outer_apply(AdmmCtrl* ac, double zz, double by, double obj) {
    if (ac->done) return;                   // a block step already failed
    const double err1 = sqrt(fmax(zz, 0.0)) / (1.0 + ac->bnorm_inf);
    const double err3 = (obj - by) / (1.0 + fabs(obj) + fabs(by));
    ac->err1 = err1;
    ac->err3 = err3;
    ac->primal_obj = obj;
    ac->dual_obj = by;
    ac->iters += 1;
    if (!isfinite(zz) || !isfinite(err3)) {
        ac->status = 5;
        ac->done = 1;
    } else if (err1 <= ac->tol && fabs(err3) <= ac->tol) {
        ac->status = 0;
        ac->done = 1;
    } else if (ac->iters >= ac->max_iter) {
        ac->status = 6;                     // LORADS_ERR_MAXITER
        ac->done = 1;
    }
}

// ------------------------------------------------------------------ constraint pass
// One group of L lanes per constraint t (list order):
//   s = <A_k, X V^T> = a x_i.v_i (i == j) or a (x_i.v_j + x_j.v_i),  z = s - b_k.
// MODE 0: w_k = y_k - rho z  (written to om, scalar type CS)
// MODE 1: y_k <- y_k - rho z (and the double-float mirror); partials z^2, b_k y_k.
template <typename TR, int CPL, int MODE>
__device__ __forceinline__ void
k_admm_cons_body(ProbDev p, const TR* __restrict__ X, const TR* __restrict__ V, int ld, int L, int Q,
            double* y, dfloat* ydf, void* __restrict__ om, const AdmmCtrl* __restrict__ ac,
            double* __restrict__ part, VGrid vg) {
    using AR = arith_t<TR>;
    using CS = admm_cs_t<TR>;
    using PA = part_t<TR, TR>;
    PA accq[PY_N] = {PA(0), PA(0)};
    const CS rho = CS(ac->rho);
    RowLoop rl(L, vg);
    for (int64_t base = rl.first; base < p.m; base += rl.stride) {
        const int64_t t = base + rl.gw;
        const bool act = t < p.m;
        int i = 0, j = 0;
        if (act) {
            i = __ldg(p.k_row + t);
            j = __ldg(p.k_col + t);
        }
        AR s = AR(0);
        if (act && p.k_ptr != nullptr) {
            // general form: list position t is one constraint, sum over its triplets
            // (the coefficient is applied per triplet; a = 1 below)
            const int64_t u0 = __ldg(p.k_ptr + t), u1 = __ldg(p.k_ptr + t + 1);
            for (int64_t u = u0; u < u1; ++u) {
                const int iu = __ldg(p.k_row + u), ju = __ldg(p.k_col + u);
                Unit<TR> xi[CPL], vj[CPL];
                load_row<TR, CPL>(xi, X, iu, ld, L, Q, rl.lig);
                load_row<TR, CPL>(vj, V, ju, ld, L, Q, rl.lig);
                AR d = dot_units<AR>(xi, vj);
                if (iu != ju) {
                    Unit<TR> xj[CPL], vi[CPL];
                    load_row<TR, CPL>(xj, X, ju, ld, L, Q, rl.lig);
                    load_row<TR, CPL>(vi, V, iu, ld, L, Q, rl.lig);
                    d = d + dot_units<AR>(xj, vi);
                }
                s = s + AR(ld_cs<CS>(p.k_a, p.k_adf, u)) * d;
            }
        } else if (act) {
            Unit<TR> xi[CPL], vj[CPL];
            load_row<TR, CPL>(xi, X, i, ld, L, Q, rl.lig);
            load_row<TR, CPL>(vj, V, j, ld, L, Q, rl.lig);
            s = dot_units<AR>(xi, vj);
            if (i != j) {
                Unit<TR> xj[CPL], vi[CPL];
                load_row<TR, CPL>(xj, X, j, ld, L, Q, rl.lig);
                load_row<TR, CPL>(vi, V, i, ld, L, Q, rl.lig);
                s = s + dot_units<AR>(xj, vi);
            }
        }
        s = group_sum(s, L);
        if (act && rl.lig == 0) {
            const int k = __ldg(p.k_id + t);
            const CS a = p.k_ptr != nullptr ? CS(1.0) : ld_cs<CS>(p.k_a, p.k_adf, t);
            const CS bk = ld_cs<CS>(p.b, p.b_df, k);
            const CS z = a * CS(s) - bk;
            const CS yk = ld_cs<CS>(y, ydf, k);
            const CS yn = yk - rho * z;
            if constexpr (MODE == 0) {
                static_cast<CS*>(om)[k] = yn;
            } else {
                y[k] = double(yn);
                if (ydf != nullptr) ydf[k] = dfloat(yn);
                accq[PY_ZZ] += PA(z * z);
                accq[PY_BY] += PA(bk * yn);
            }
        }
    }
    if constexpr (MODE == 1) block_partials<PY_N>(accq, part, vg.pslot);
}

// ------------------------------------------------------------------ residual pass
// r = p = -(C - A*(w)) V + rho (V - X) row by row (Algorithm 2's r_0 and p_0);
// partial ||r||^2 of the stored values.
template <typename TR, typename TW, int CPL>
__device__ __forceinline__ void
k_admm_resid_body(ProbDev p, const TR* __restrict__ X, const TR* __restrict__ V, int ld, int L, int Q,
             const void* __restrict__ om_v, TW* __restrict__ r, TW* __restrict__ pd,
             const AdmmCtrl* __restrict__ ac, double* __restrict__ part, VGrid vg) {
    using AR = arith_t<TR>;
    using AW = arith_t<TW>;
    using CS = admm_cs_t<TR>;
    using PA = part_t<TW, TR>;
    const CS* __restrict__ om = static_cast<const CS*>(om_v);
    const AR* __restrict__ cv = cvals<AR>(p);
    const AR rho = AR(ac->rho);
    PA acc_rr[PA_N] = {PA(0)};
    RowLoop rl(L, vg);
    for (int64_t base = rl.first; base < p.n; base += rl.stride) {
        const int64_t i = base + rl.gw;
        if (i >= p.n) continue;
        AR acc[CPL][4];
#pragma unroll
        for (int c = 0; c < CPL; ++c)
#pragma unroll
            for (int e = 0; e < 4; ++e) acc[c][e] = AR(0);
        // C V: gathered rows of V, two stored entries in flight per lane
        const int64_t s0 = __ldg(p.c_rowptr + i), s1 = __ldg(p.c_rowptr + i + 1);
        int64_t s = s0;
        for (; s + 2 <= s1; s += 2) {
            const int j0 = __ldg(p.c_col + s), j1 = __ldg(p.c_col + s + 1);
            const AR w0 = ldv(cv + s), w1 = ldv(cv + s + 1);
            Unit<TR> x0[CPL], x1[CPL];
            load_row<TR, CPL>(x0, V, j0, ld, L, Q, rl.lig);
            load_row<TR, CPL>(x1, V, j1, ld, L, Q, rl.lig);
#pragma unroll
            for (int c = 0; c < CPL; ++c)
#pragma unroll
                for (int e = 0; e < 4; ++e)
                    acc[c][e] = fma(w1, AR(x1[c].v[e]), fma(w0, AR(x0[c].v[e]), acc[c][e]));
        }
        if (s < s1) {
            const int j0 = __ldg(p.c_col + s);
            const AR w0 = ldv(cv + s);
            Unit<TR> x0[CPL];
            load_row<TR, CPL>(x0, V, j0, ld, L, Q, rl.lig);
#pragma unroll
            for (int c = 0; c < CPL; ++c)
#pragma unroll
                for (int e = 0; e < 4; ++e) acc[c][e] = fma(w0, AR(x0[c].v[e]), acc[c][e]);
        }
        Unit<TR> vi[CPL], xi[CPL];
        load_row<TR, CPL>(vi, V, i, ld, L, Q, rl.lig);
        load_row<TR, CPL>(xi, X, i, ld, L, Q, rl.lig);
        // - A*(w) V: the diagonal constraint of row i, then the off-diagonal pattern
        if (p.dk != nullptr) {
            const int k = __ldg(p.dk + i);
            if (k >= 0) {
                const AR wk = AR(-(ld_cs<CS>(p.da, p.da_df, i) * om[k]));
#pragma unroll
                for (int c = 0; c < CPL; ++c)
#pragma unroll
                    for (int e = 0; e < 4; ++e) acc[c][e] = fma(wk, AR(vi[c].v[e]), acc[c][e]);
            }
        }
        if (p.m_off > 0) {
            const int64_t a0 = __ldg(p.a_rowptr + i), a1 = __ldg(p.a_rowptr + i + 1);
            for (int64_t q = a0; q < a1; ++q) {
                const int j = __ldg(p.a_col + q);
                const int k = __ldg(p.a_k + q);
                const AR wk = AR(-(ld_cs<CS>(p.a_a, p.a_adf, q) * om[k]));
                Unit<TR> xj[CPL];
                load_row<TR, CPL>(xj, V, j, ld, L, Q, rl.lig);
#pragma unroll
                for (int c = 0; c < CPL; ++c)
#pragma unroll
                    for (int e = 0; e < 4; ++e) acc[c][e] = fma(wk, AR(xj[c].v[e]), acc[c][e]);
            }
        }
        Unit<TW> ro[CPL];
        AW rr = AW(0);
#pragma unroll
        for (int c = 0; c < CPL; ++c)
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                const AR val = rho * (AR(vi[c].v[e]) - AR(xi[c].v[e])) - acc[c][e];
                ro[c].v[e] = AW(val);
                const AW rv = AW(ro[c].v[e]);
                rr = fma(rv, rv, rr);
            }
        store_row<TW, CPL>(ro, r, i, ld, L, Q, rl.lig);
        store_row<TW, CPL>(ro, pd, i, ld, L, Q, rl.lig);
        acc_rr[PA_RR] += PA(rr);
    }
    block_partials<PA_N>(acc_rr, part, vg.pslot);
}

// ------------------------------------------------------------------ p update
// p = r + beta p (CG steps after the first), for the path with off-diagonal
// constraints whose operator pass gathers neighbouring rows of p.
template <typename TW>
__device__ __forceinline__ void
k_admm_pupd_body(int64_t nunits, const TW* __restrict__ r, TW* __restrict__ pd, const AdmmCtrl* __restrict__ ac, VGrid vg) {
    if (!ac->cg_active || ac->cg_k == 0) return;
    using AW = arith_t<TW>;
    const AW beta = AW(ac->beta);
    for (int64_t u = vg.bid * (int64_t)blockDim.x + threadIdx.x; u < nunits; u += (int64_t)vg.nblk * blockDim.x) {
        Unit<TW> ru, pu;
        ru.load_stream(r + 4 * u);
        pu.load(pd + 4 * u);
#pragma unroll
        for (int e = 0; e < 4; ++e) pu.v[e] = fma(beta, AW(pu.v[e]), AW(ru.v[e]));
        pu.store(pd + 4 * u);
    }
}

// ------------------------------------------------------------------ operator pass
// Q = frakA_V(p) = rho (A*(A(p V^T)) V + p) row by row; partials ||p||^2 and
// ||A(p V^T)||^2 (each off-diagonal constraint is met from both of its rows:
// half of its square from each).
// FUSE_P: first p = r + beta p (CG steps after the first; only without
// off-diagonal constraints, whose rows would read neighbours' p).
// With ac == nullptr (standalone operator) the pass runs with rho_arg and no update.
template <typename TR, typename TW, int CPL, bool FUSE_P>
__device__ __forceinline__ void
k_admm_op_body(ProbDev p, const TR* __restrict__ V, int ld, int L, int Q, const TW* __restrict__ r,
          TW* __restrict__ pd, TW* __restrict__ Qo, const AdmmCtrl* __restrict__ ac, double rho_arg,
          double* __restrict__ part, VGrid vg) {
    if (ac != nullptr && !ac->cg_active) return;
    using AW = arith_t<TW>;
    using CS = admm_cs_t<TR>;
    using PA = part_t<TW, TW>;
    const double rho_d = ac ? ac->rho : rho_arg;
    const AW rho = AW(rho_d);
    const bool upd = FUSE_P && ac != nullptr && ac->cg_k > 0;
    const AW beta = upd ? AW(ac->beta) : AW(0);
    PA accq[PQ_N] = {PA(0), PA(0)};
    RowLoop rl(L, vg);
    for (int64_t base = rl.first; base < p.n; base += rl.stride) {
        const int64_t i = base + rl.gw;
        const bool act = i < p.n;
        Unit<TW> pi[CPL];
        Unit<TR> vi[CPL];
        AW q[CPL][4];
        AW pp = AW(0), wv = AW(0);
        int k = -1;
        if (act) {
            load_row<TW, CPL>(pi, pd, i, ld, L, Q, rl.lig);
            if (upd) {
                Unit<TW> ri[CPL];
                load_row<TW, CPL>(ri, r, i, ld, L, Q, rl.lig);
#pragma unroll
                for (int c = 0; c < CPL; ++c)
#pragma unroll
                    for (int e = 0; e < 4; ++e) pi[c].v[e] = fma(beta, AW(pi[c].v[e]), AW(ri[c].v[e]));
                store_row<TW, CPL>(pi, pd, i, ld, L, Q, rl.lig);
            }
            load_row<TR, CPL>(vi, V, i, ld, L, Q, rl.lig);
#pragma unroll
            for (int c = 0; c < CPL; ++c)
#pragma unroll
                for (int e = 0; e < 4; ++e) {
                    const AW pe = AW(pi[c].v[e]);
                    q[c][e] = pe;
                    pp = fma(pe, pe, pp);
                }
            if (p.dk != nullptr) k = __ldg(p.dk + i);
            if (k >= 0) {
#pragma unroll
                for (int c = 0; c < CPL; ++c)
#pragma unroll
                    for (int e = 0; e < 4; ++e) wv = fma(AW(pi[c].v[e]), AW(vi[c].v[e]), wv);
            }
        }
        // diagonal constraint: w = a p_i.v_i, Q_i += a w v_i
        wv = group_sum(wv, L);
        if (k >= 0) {
            const AW a = AW(ld_cs<CS>(p.da, p.da_df, i));
            const AW w = a * wv;
            const AW aw = a * w;
#pragma unroll
            for (int c = 0; c < CPL; ++c)
#pragma unroll
                for (int e = 0; e < 4; ++e) q[c][e] = fma(aw, AW(vi[c].v[e]), q[c][e]);
            if (rl.lig == 0) accq[PQ_WW] += PA(w * w);
        }
        // off-diagonal constraints of row i: w = a (p_i.v_j + p_j.v_i), Q_i += a w v_j
        // (single-triplet form; the general form adds these terms in k_admm_opw/opq)
        if (act && p.m_off > 0 && p.k_ptr == nullptr) {
            const int64_t a0 = __ldg(p.a_rowptr + i), a1 = __ldg(p.a_rowptr + i + 1);
            for (int64_t s = a0; s < a1; ++s) {
                const int j = __ldg(p.a_col + s);
                const AW a = AW(ld_cs<CS>(p.a_a, p.a_adf, s));
                Unit<TW> pj[CPL];
                Unit<TR> vj[CPL];
                load_row<TW, CPL>(pj, pd, j, ld, L, Q, rl.lig);
                load_row<TR, CPL>(vj, V, j, ld, L, Q, rl.lig);
                AW d = AW(0);
#pragma unroll
                for (int c = 0; c < CPL; ++c)
#pragma unroll
                    for (int e = 0; e < 4; ++e)
                        d = fma(AW(pi[c].v[e]), AW(vj[c].v[e]), fma(AW(pj[c].v[e]), AW(vi[c].v[e]), d));
                // the group's lanes hold parts of the row: sum within the group only
                // (groups of one warp may run different numbers of entries)
                const unsigned gm = group_lanes(L);
                for (int o = L >> 1; o > 0; o >>= 1) d += shfl_xor_in(d, o, gm);
                const AW w = a * d;
                const AW aw = a * w;
#pragma unroll
                for (int c = 0; c < CPL; ++c)
#pragma unroll
                    for (int e = 0; e < 4; ++e) q[c][e] = fma(aw, AW(vj[c].v[e]), q[c][e]);
                if (rl.lig == 0) accq[PQ_WW] += PA(AW(0.5f) * w * w);
            }
        }
        if (act) {
            Unit<TW> qo[CPL];
#pragma unroll
            for (int c = 0; c < CPL; ++c)
#pragma unroll
                for (int e = 0; e < 4; ++e) qo[c].v[e] = rho * q[c][e];
            store_row<TW, CPL>(qo, Qo, i, ld, L, Q, rl.lig);
            accq[PQ_PP] += PA(pp);
        }
    }
    block_partials<PQ_N>(accq, part, vg.pslot);
}

// ------------------------------------------------------------------ general form
// w_k = <A_k, p V^T> for the listed constraints (positions m_diag..m-1; each a sum
// over its triplets), stored by constraint; partial sum of w_k^2.
template <typename TR, typename TW, int CPL>
__device__ __forceinline__ void
k_admm_opw_body(ProbDev p, const TR* __restrict__ V, int ld, int L, int Q, const TW* __restrict__ pd,
           void* __restrict__ w_v, const AdmmCtrl* __restrict__ ac, double* __restrict__ part, VGrid vg) {
    if (!ac->cg_active) return;
    using AW = arith_t<TW>;
    using CS = admm_cs_t<TR>;
    using PA = part_t<TW, TW>;
    CS* __restrict__ w = static_cast<CS*>(w_v);
    PA acc[1] = {PA(0)};
    RowLoop rl(L, vg);
    const int64_t cnt = p.m - p.m_diag;
    for (int64_t base = rl.first; base < cnt; base += rl.stride) {
        const int64_t q = p.m_diag + base + rl.gw;
        const bool act = q < p.m;
        AW s = AW(0);
        if (act) {
            const int64_t u0 = __ldg(p.k_ptr + q), u1 = __ldg(p.k_ptr + q + 1);
            for (int64_t u = u0; u < u1; ++u) {
                const int i = __ldg(p.k_row + u), j = __ldg(p.k_col + u);
                Unit<TW> pi[CPL];
                Unit<TR> vj[CPL];
                load_row<TW, CPL>(pi, pd, i, ld, L, Q, rl.lig);
                load_row<TR, CPL>(vj, V, j, ld, L, Q, rl.lig);
                AW d = AW(0);
#pragma unroll
                for (int c = 0; c < CPL; ++c)
#pragma unroll
                    for (int e = 0; e < 4; ++e) d = fma(AW(pi[c].v[e]), AW(vj[c].v[e]), d);
                if (i != j) {
                    Unit<TW> pj[CPL];
                    Unit<TR> vi[CPL];
                    load_row<TW, CPL>(pj, pd, j, ld, L, Q, rl.lig);
                    load_row<TR, CPL>(vi, V, i, ld, L, Q, rl.lig);
#pragma unroll
                    for (int c = 0; c < CPL; ++c)
#pragma unroll
                        for (int e = 0; e < 4; ++e) d = fma(AW(pj[c].v[e]), AW(vi[c].v[e]), d);
                }
                s = fma(AW(ld_cs<CS>(p.k_a, p.k_adf, u)), d, s);
            }
        }
        s = group_sum(s, L);
        if (act && rl.lig == 0) {
            w[__ldg(p.k_id + q)] = CS(s);
            acc[0] += PA(s * s);
        }
    }
    block_partials<1>(acc, part, vg.pslot);
}

// Q_i += rho sum over the slots (j, k, a) of row i of a w_k v_j (A*(w) V of the listed
// constraints).
template <typename TR, typename TW, int CPL>
__device__ __forceinline__ void
k_admm_opq_body(ProbDev p, const TR* __restrict__ V, int ld, int L, int Q, const void* __restrict__ w_v,
           TW* __restrict__ Qo, const AdmmCtrl* __restrict__ ac, VGrid vg) {
    if (!ac->cg_active) return;
    using AW = arith_t<TW>;
    using CS = admm_cs_t<TR>;
    const CS* __restrict__ w = static_cast<const CS*>(w_v);
    const AW rho = AW(ac->rho);
    RowLoop rl(L, vg);
    for (int64_t base = rl.first; base < p.n; base += rl.stride) {
        const int64_t i = base + rl.gw;
        if (i >= p.n) continue;
        AW acc[CPL][4];
#pragma unroll
        for (int c = 0; c < CPL; ++c)
#pragma unroll
            for (int e = 0; e < 4; ++e) acc[c][e] = AW(0);
        const int64_t s0 = __ldg(p.a_rowptr + i), s1 = __ldg(p.a_rowptr + i + 1);
        for (int64_t s = s0; s < s1; ++s) {
            const int j = __ldg(p.a_col + s);
            const AW c_w = AW(ld_cs<CS>(p.a_a, p.a_adf, s) * w[__ldg(p.a_k + s)]);
            Unit<TR> vj[CPL];
            load_row<TR, CPL>(vj, V, j, ld, L, Q, rl.lig);
#pragma unroll
            for (int c = 0; c < CPL; ++c)
#pragma unroll
                for (int e = 0; e < 4; ++e) acc[c][e] = fma(c_w, AW(vj[c].v[e]), acc[c][e]);
        }
        Unit<TW> q[CPL];
        load_row<TW, CPL>(q, Qo, i, ld, L, Q, rl.lig);
#pragma unroll
        for (int c = 0; c < CPL; ++c)
#pragma unroll
            for (int e = 0; e < 4; ++e) q[c].v[e] = fma(rho, acc[c][e], AW(q[c].v[e]));
        store_row<TW, CPL>(q, Qo, i, ld, L, Q, rl.lig);
    }
}

// ------------------------------------------------------------------ update pass
// X += alpha p, r -= alpha Q; partial ||r||^2 (flat over units of 4 elements).
template <typename TR, typename TW>
__device__ __forceinline__ void
k_admm_upd_body(int64_t nunits, TR* __restrict__ X, const TW* __restrict__ pd, TW* __restrict__ r,
           const TW* __restrict__ Qo, const AdmmCtrl* __restrict__ ac, double* __restrict__ part, VGrid vg) {
    if (!ac->cg_active) return;
    using AR = arith_t<TR>;
    using AW = arith_t<TW>;
    using PA = part_t<TW, TW>;
    const AR alpha_r = AR(ac->alpha);
    const AW alpha_w = AW(ac->alpha);
    PA acc[PA_N] = {PA(0)};
    AW rr = AW(0);
    for (int64_t u = vg.bid * (int64_t)blockDim.x + threadIdx.x; u < nunits; u += (int64_t)vg.nblk * blockDim.x) {
        Unit<TR> xu;
        Unit<TW> pu, ru, qu;
        xu.load_stream(X + 4 * u);
        pu.load_stream(pd + 4 * u);
        ru.load_stream(r + 4 * u);
        qu.load_stream(Qo + 4 * u);
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            xu.v[e] = fma(alpha_r, AR(pu.v[e]), AR(xu.v[e]));
            ru.v[e] = fma(-alpha_w, AW(qu.v[e]), AW(ru.v[e]));
            const AW rv = AW(ru.v[e]);
            rr = fma(rv, rv, rr);
        }
        xu.store_stream(X + 4 * u);
        ru.store_stream(r + 4 * u);
    }
    acc[PA_RR] += PA(rr);
    block_partials<PA_N>(acc, part, vg.pslot);
}

// R = (U + V) / 2 (flat), the factor whose X = R R^T the stage reports.
template <typename TR>
__device__ __forceinline__ void
k_admm_avg_body(int64_t nunits, const TR* __restrict__ U, const TR* __restrict__ V, TR* __restrict__ R, VGrid vg) {
    using AR = arith_t<TR>;
    for (int64_t u = vg.bid * (int64_t)blockDim.x + threadIdx.x; u < nunits; u += (int64_t)vg.nblk * blockDim.x) {
        Unit<TR> a, b;
        a.load_stream(U + 4 * u);
        b.load_stream(V + 4 * u);
#pragma unroll
        for (int e = 0; e < 4; ++e) a.v[e] = AR(0.5f) * (AR(a.v[e]) + AR(b.v[e]));
        a.store(R + 4 * u);
    }
}


// ------------------------------------------------------------------ kernels
// One launch per body over the hardware grid (the batched solve runs the bodies
// over the blocks of one instance).
template <typename TR, int CPL, int MODE>
__global__ void __launch_bounds__(kThreads)
k_admm_cons(ProbDev p, const TR* __restrict__ X, const TR* __restrict__ V, int ld, int L, int Q,
            double* y, dfloat* ydf, void* __restrict__ om, const AdmmCtrl* __restrict__ ac,
            double* __restrict__ part) {
    k_admm_cons_body<TR, CPL, MODE>(p, X, V, ld, L, Q, y, ydf, om, ac, part, hw_grid());
}

template <typename TR, typename TW, int CPL>
__global__ void __launch_bounds__(kThreads)
k_admm_resid(ProbDev p, const TR* __restrict__ X, const TR* __restrict__ V, int ld, int L, int Q,
             const void* __restrict__ om_v, TW* __restrict__ r, TW* __restrict__ pd,
             const AdmmCtrl* __restrict__ ac, double* __restrict__ part) {
    k_admm_resid_body<TR, TW, CPL>(p, X, V, ld, L, Q, om_v, r, pd, ac, part, hw_grid());
}

template <typename TW>
__global__ void __launch_bounds__(kThreads)
k_admm_pupd(int64_t nunits, const TW* __restrict__ r, TW* __restrict__ pd, const AdmmCtrl* __restrict__ ac) {
    k_admm_pupd_body<TW>(nunits, r, pd, ac, hw_grid());
}

template <typename TR, typename TW, int CPL, bool FUSE_P>
__global__ void __launch_bounds__(kThreads)
k_admm_op(ProbDev p, const TR* __restrict__ V, int ld, int L, int Q, const TW* __restrict__ r,
          TW* __restrict__ pd, TW* __restrict__ Qo, const AdmmCtrl* __restrict__ ac, double rho_arg,
          double* __restrict__ part) {
    k_admm_op_body<TR, TW, CPL, FUSE_P>(p, V, ld, L, Q, r, pd, Qo, ac, rho_arg, part, hw_grid());
}

template <typename TR, typename TW, int CPL>
__global__ void __launch_bounds__(kThreads)
k_admm_opw(ProbDev p, const TR* __restrict__ V, int ld, int L, int Q, const TW* __restrict__ pd,
           void* __restrict__ w_v, const AdmmCtrl* __restrict__ ac, double* __restrict__ part) {
    k_admm_opw_body<TR, TW, CPL>(p, V, ld, L, Q, pd, w_v, ac, part, hw_grid());
}

template <typename TR, typename TW, int CPL>
__global__ void __launch_bounds__(kThreads)
k_admm_opq(ProbDev p, const TR* __restrict__ V, int ld, int L, int Q, const void* __restrict__ w_v,
           TW* __restrict__ Qo, const AdmmCtrl* __restrict__ ac) {
    k_admm_opq_body<TR, TW, CPL>(p, V, ld, L, Q, w_v, Qo, ac, hw_grid());
}

template <typename TR, typename TW>
__global__ void __launch_bounds__(kThreads)
k_admm_upd(int64_t nunits, TR* __restrict__ X, const TW* __restrict__ pd, TW* __restrict__ r,
           const TW* __restrict__ Qo, const AdmmCtrl* __restrict__ ac, double* __restrict__ part) {
    k_admm_upd_body<TR, TW>(nunits, X, pd, r, Qo, ac, part, hw_grid());
}

template <typename TR>
__global__ void __launch_bounds__(kThreads)
k_admm_avg(int64_t nunits, const TR* __restrict__ U, const TR* __restrict__ V, TR* __restrict__ R) {
    k_admm_avg_body<TR>(nunits, U, V, R, hw_grid());
}

}  // namespace lorads
