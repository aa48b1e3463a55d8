// Scalar decisions of the solve loop, shared by the single-block control
// kernels of the single-instance solve and by the batched persistent solve:
// the cubic root of the exact line search (App. A.2), the L-BFGS memory and
// two-loop recursion of Algorithm 1 on Gram data, and the multiplier/penalty
// step of Sec. 2.1.  Every function here is executed by one thread on folded
// (already reduced) sums, so both solvers take identical decisions from
// identical sums.
#pragma once

#include <math.h>
#include "common.cuh"

namespace lorads {

// ---------------------------------------------------------------- random draws
// SplitMix64 output function (Steele, Lea, Flood 2014) applied to a counter state.
__device__ __forceinline__ uint64_t splitmix_out(uint64_t state) {
    uint64_t z = state;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

// Standard normal number e of the stream started at `base`: outputs 2e+1 and
// 2e+2 of SplitMix64 (u1 in (0,1], u2 in [0,1)), Box-Muller cosine branch.
__device__ __forceinline__ double normal_at(uint64_t base, int64_t e) {
    const uint64_t golden = 0x9E3779B97F4A7C15ull;
    const uint64_t x1 = splitmix_out(base + (uint64_t)(2 * e + 1) * golden);
    const uint64_t x2 = splitmix_out(base + (uint64_t)(2 * e + 2) * golden);
    const double u1 = (double)((x1 >> 11) + 1) * (1.0 / 9007199254740992.0);
    const double u2 = (double)(x2 >> 11) * (1.0 / 9007199254740992.0);
    return sqrt(-2.0 * log(u1)) * cos(2.0 * 3.141592653589793 * u2);
}

// ---------------------------------------------------------------- cubic root
__device__ __forceinline__ double qval(const double* a, double t) {
    return ((a[0] * t + a[1]) * t + a[2]) * t * t + a[3] * t;
}
__device__ __forceinline__ double qd1(const double* a, double t) {
    return ((4.0 * a[0] * t + 3.0 * a[1]) * t + 2.0 * a[2]) * t + a[3];
}
__device__ __forceinline__ double qd2(const double* a, double t) {
    return (12.0 * a[0] * t + 6.0 * a[1]) * t + 2.0 * a[2];
}

// Root of f' in [lo, hi] where f'(lo), f'(hi) have opposite signs and f' is
// monotone: Newton steps kept inside the bracket, bisection otherwise.
__device__ inline double bracketed_root(const double* a, double lo, double hi) {
    double flo = qd1(a, lo);
    double t = 0.5 * (lo + hi);
    for (int it = 0; it < 200; ++it) {
        const double f = qd1(a, t);
        if (f == 0.0) return t;
        if ((f < 0.0) == (flo < 0.0)) { lo = t; flo = f; } else { hi = t; }
        const double d = qd2(a, t);
        double tn = (d != 0.0) ? t - f / d : 0.5 * (lo + hi);
        if (!(tn > lo && tn < hi)) tn = 0.5 * (lo + hi);
        if (tn == t || hi - lo <= 4.0 * 2.220446049250313e-16 * fabs(t)) { t = tn; break; }
        t = tn;
    }
    return t;
}

// Smallest t > 0 with f'(t) of the sign `positive` beyond `from`, by doubling.
__device__ inline double grow_until(const double* a, double from, bool positive) {
    double h = fmax(1.0, fabs(from));
    for (int it = 0; it < 2100; ++it) {
        const double t = from + h;
        const double f = qd1(a, t);
        if (positive ? (f > 0.0) : (f < 0.0)) return t;
        h *= 2.0;
        if (!isfinite(t)) break;
    }
    return from + h;
}

// Step of the exact line search (App. A.2): among the positive real roots of
// 4a1 t^3 + 3a2 t^2 + 2a3 t + a4 the one with the lowest quartic value
// f(t) = a1 t^4 + a2 t^3 + a3 t^2 + a4 t; 0 when no positive root lowers f.
__device__ inline double quartic_step(const double* a) {
    double cand[3];
    int nc = 0;
    if (a[0] != 0.0) {
        // monotone pieces of f' split at the roots of f'' = 12a1 t^2 + 6a2 t + 2a3
        double cuts[2];
        int ncut = 0;
        const double A = 12.0 * a[0], B = 6.0 * a[1], C = 2.0 * a[2];
        const double disc = B * B - 4.0 * A * C;
        if (disc > 0.0) {
            const double sq = sqrt(disc);
            const double qq = -0.5 * (B + copysign(sq, B));
            double c1 = qq / A, c2 = (qq != 0.0) ? C / qq : -c1;
            if (c1 > c2) { const double t = c1; c1 = c2; c2 = t; }
            cuts[ncut++] = c1;
            cuts[ncut++] = c2;
        }
        // pieces [edge_k, edge_{k+1}] clipped to t > 0
        double edges[4];
        int ne = 0;
        edges[ne++] = 0.0;
        for (int k = 0; k < ncut; ++k)
            if (cuts[k] > 0.0) edges[ne++] = cuts[k];
        for (int k = 0; k < ne; ++k) {
            const double lo = edges[k];
            const double flo = qd1(a, lo);
            double hi;
            bool last = (k == ne - 1);
            if (!last) {
                hi = edges[k + 1];
            } else {
                // f' -> +inf: find a finite right end with f' > 0
                if (flo >= 0.0) continue;
                hi = grow_until(a, lo, true);
            }
            const double fhi = qd1(a, hi);
            if (flo == 0.0) {
                if (lo > 0.0 && nc < 3) cand[nc++] = lo;
                continue;
            }
            if ((flo < 0.0 && fhi > 0.0) || (flo > 0.0 && fhi < 0.0)) {
                if (nc < 3) cand[nc++] = bracketed_root(a, lo, hi);
            } else if (fhi == 0.0 && hi > 0.0 && last == false) {
                if (nc < 3) cand[nc++] = hi;
            }
        }
    } else if (a[1] != 0.0) {
        // f' = 3a2 t^2 + 2a3 t + a4
        const double A = 3.0 * a[1], B = 2.0 * a[2], C = a[3];
        const double disc = B * B - 4.0 * A * C;
        if (disc >= 0.0) {
            const double sq = sqrt(disc);
            const double qq = -0.5 * (B + copysign(sq, B));
            if (qq != 0.0) {
                cand[nc++] = qq / A;
                cand[nc++] = C / qq;
            } else {
                cand[nc++] = 0.0;
            }
        }
    } else if (a[2] != 0.0) {
        cand[nc++] = -a[3] / (2.0 * a[2]);
    }
    // sort candidates ascending (ties keep the smaller)
    for (int i = 1; i < nc; ++i)
        for (int j = i; j > 0 && cand[j] < cand[j - 1]; --j) {
            const double t = cand[j]; cand[j] = cand[j - 1]; cand[j - 1] = t;
        }
    double best = 0.0, best_f = 0.0;
    for (int i = 0; i < nc; ++i) {
        const double t = cand[i];
        if (!(t > 0.0) || !isfinite(t)) continue;
        const double f = qval(a, t);
        if (f < best_f) { best = t; best_f = f; }
    }
    return best;
}

// ---------------------------------------------------------------- memory helpers
__device__ inline void mem_clear(Ctrl* c) {
    c->mem_count = 0;
    for (int s = 0; s < kMaxMem; ++s) {
        c->order[s] = s;
        c->cS[s] = 0.0;
        c->cY[s] = 0.0;
        c->g_s[s] = 0.0;
        c->g_y[s] = 0.0;
    }
}

// Two-loop recursion of Algorithm 1 (initial matrix I) carried out on
// coefficients: D = cG G + sum cS_u S_u + sum cY_u Y_u, using only the dot
// products <G,S_u>, <G,Y_u>, <S_u,Y_v>, <Y_u,Y_v> of the stored pairs.
__device__ inline void two_loop_coeffs(Ctrl* c) {
    const int mem = c->mem_count;
    double alpha[kMaxMem];
    c->cG = -1.0;
    for (int s = 0; s < kMaxMem; ++s) { c->cS[s] = 0.0; c->cY[s] = 0.0; }
    for (int t = mem - 1; t >= 0; --t) {                 // newest to oldest
        const int st = c->order[t];
        double sD = c->cG * c->g_s[st];
        for (int u = 0; u < mem; ++u) {
            const int su = c->order[u];
            sD += c->cY[su] * c->SY[st][su];
        }
        alpha[t] = sD / c->SY[st][st];
        c->cY[st] -= alpha[t];
    }
    if (c->lbfgs_scaling && mem > 0) {                   // r = gamma q
        const int sn = c->order[mem - 1];
        const double gamma = c->SY[sn][sn] / c->YY[sn][sn];
        c->cG *= gamma;
        for (int u = 0; u < mem; ++u) c->cY[c->order[u]] *= gamma;
    }
    for (int t = 0; t < mem; ++t) {                      // oldest to newest
        const int st = c->order[t];
        double yD = c->cG * c->g_y[st];
        for (int u = 0; u < mem; ++u) {
            const int su = c->order[u];
            yD += c->cY[su] * c->YY[st][su] + c->cS[su] * c->SY[su][st];
        }
        c->cS[st] += alpha[t] - yD / c->SY[st][st];
    }
}

// Physical slot of the next pair and the pairs it keeps.
__device__ inline void plan_next_slot(Ctrl* c, int T) {
    const int mem = c->mem_count;
    if (mem < T) {
        int used = 0;
        for (int t = 0; t < mem; ++t) used |= 1 << c->order[t];
        int ns = 0;
        while (used & (1 << ns)) ++ns;
        c->new_slot = ns;
        c->old_count = mem;
        for (int t = 0; t < mem; ++t) c->old_slots[t] = c->order[t];
    } else {
        c->new_slot = c->order[0];
        c->old_count = mem - 1;
        for (int t = 1; t < mem; ++t) c->old_slots[t - 1] = c->order[t];
    }
}

__device__ inline void finish_inner_test(Ctrl* c) {
    if (c->dev_error) {
        c->status = 7;                          // LORADS_ERR_TIMEOUT: a device wait expired
        c->solve_done = 1;
        return;
    }
    const double zn = sqrt(fmax(c->znorm2, 0.0));
    const double floor_ = c->tol * (1.0 + c->bnorm_inf);
    double thr;
    if (c->inner_scale == 0) thr = c->inner_rel * fmax(zn, floor_);
    else if (c->inner_scale == 1) thr = c->inner_rel * fmax(c->rho * zn, floor_);
    else thr = fmax(floor_, fmin(c->inner_rel * c->rho * zn, c->inner_progress * c->gnorm0));
    const double gn = sqrt(fmax(c->gnorm2, 0.0));
    // tested on the sums themselves: fmax(NaN, 0) is 0
    if (!isfinite(c->gnorm2) || !isfinite(c->znorm2)) {
        c->status = 5;                          // LORADS_ERR_NUMERIC
        c->solve_done = 1;
        return;
    }
    if (c->total_limit > 0 && c->total_inner >= c->total_limit) {
        c->status = 6;                          // LORADS_ERR_MAXITER
        c->solve_done = 1;
        return;
    }
    if (gn <= thr || c->inner_k >= c->max_inner) {
        c->inner_done = 1;
        c->phase = PHASE_OUTER;
        return;
    }
    two_loop_coeffs(c);
    plan_next_slot(c, c->lbfgs_mem);
}

// ---------------------------------------------------------------- decisions
// After the line-search sums of one iteration: a1..a4 and tau (App. A.2).
// a4 = <G, D> (the directional derivative; equal to p1 - y~^T q1).
// sd: PD_* sums; sl, sc: PL_* sums of the C pass and the constraint pass.
__device__ inline void ctrl_root_apply(Ctrl* c, const double* sd, const double* sl, const double* sc) {
    const double rho = c->rho;
    const double yq2 = sl[PL_YQ2] + sc[PL_YQ2];
    const double q1q1 = sl[PL_Q1Q1] + sc[PL_Q1Q1];
    const double q1q2 = sl[PL_Q1Q2] + sc[PL_Q1Q2];
    const double q2q2 = sl[PL_Q2Q2] + sc[PL_Q2Q2];
    c->gD = sd[PD_GD];
    c->DD = sd[PD_DD];
    c->a[0] = 0.5 * rho * q2q2;
    c->a[1] = rho * q1q2;
    c->a[2] = sl[PL_P2] - yq2 + 0.5 * rho * q1q1;
    c->a[3] = sd[PD_GD];
    c->inner_k += 1;
    c->total_inner += 1;
    const double tau = quartic_step(c->a);
    bool finite = isfinite(c->a[0]) && isfinite(c->a[1]) && isfinite(c->a[2]) && isfinite(c->a[3]);
    if (!finite) {
        c->status = 5;
        c->solve_done = 1;
        c->step_ok = 0;
        return;
    }
    if (tau > 0.0) {
        c->tau = tau;
        c->step_ok = 1;
    } else {
        c->tau = 0.0;
        c->step_ok = 0;
        if (c->mem_count > 0) {
            mem_clear(c);               // next direction is -G
        } else {
            c->inner_done = 1;          // no descent along -G: leave the inner loop
            c->phase = PHASE_OUTER;
        }
    }
}

// After the row update (or the gradient at a fresh point when `reset`):
// store the new pair if its curvature is positive enough, test the inner stop
// and prepare the next direction.  su: PU_* sums, sy: PC_* sums of y~.
__device__ inline void ctrl_hist_apply(Ctrl* c, bool reset, bool fresh, const double* su, const double* sy) {
    if (fresh) {
        c->gnorm2 = su[PU_GG];
        c->znorm2 = su[PU_ZZ] + sy[PC_ZZ];
    }
    if (reset) {
        mem_clear(c);
        c->gnorm0 = sqrt(fmax(c->gnorm2, 0.0));
        c->inner_k = 0;
        c->inner_done = 0;
        c->step_ok = 0;
        c->phase = PHASE_INNER;
    } else if (c->step_ok) {
        const double tau = c->tau;
        const double ys = su[PU_SYN], yy = su[PU_YYN];
        const double ss = tau * tau * c->DD;                      // ||tau D||^2
        if (ys > 1e-16 * sqrt(fmax(yy, 0.0) * fmax(ss, 0.0)) && ys > 0.0) {
            const int ns = c->new_slot;
            for (int t = 0; t < c->old_count; ++t) {
                const int v = c->old_slots[t];
                const double* q = su + PU_FIXED + PU_PER_OLD * t;
                // G' = G + Y_new: dots with the new gradient from the previous ones
                c->g_s[v] += q[1];
                c->g_y[v] += q[2];
                c->SY[ns][v] = q[0];
                c->SY[v][ns] = q[1];
                c->YY[ns][v] = q[2];
                c->YY[v][ns] = q[2];
            }
            c->SY[ns][ns] = ys;
            c->YY[ns][ns] = yy;
            c->g_s[ns] = tau * c->gD + ys;                          // <G,S_new> + <Y_new,S_new>
            c->g_y[ns] = su[PU_GYN];
            // order: keep old slots (oldest first), append the new one
            for (int t = 0; t < c->old_count; ++t) c->order[t] = c->old_slots[t];
            c->order[c->old_count] = ns;
            c->mem_count = c->old_count + 1;
        } else {
            mem_clear(c);
        }
    }
    finish_inner_test(c);
}

// After the multiplier step: err1, err3, stop test, penalty and rank request.
// sc: PC_* sums at the new multiplier, so: PO_* sums.
__device__ inline void ctrl_outer_apply(Ctrl* c, const double* sc, const double* so) {
    const double err1 = sqrt(fmax(sc[PC_ZZ], 0.0)) / (1.0 + c->bnorm_inf);
    const double obj = so[PO_CRR];
    const double dual = sc[PC_BY];
    const double err3 = (obj - dual) / (1.0 + fabs(obj) + fabs(dual));
    c->err1 = err1;
    c->err3 = err3;
    c->primal_obj = obj;
    c->dual_obj = dual;
    c->outer += 1;
    c->last_iter_rho = c->rho;
    if (!isfinite(sc[PC_ZZ]) || !isfinite(err3)) {
        c->status = 5;
        c->solve_done = 1;
        return;
    }
    if (err1 <= c->tol && (c->stop_rule == 1 || fabs(err3) <= c->tol)) {
        c->status = 0;
        c->solve_done = 1;
        return;
    }
    const bool capped = c->inner_k >= c->max_inner;
    bool grow = err1 > c->infeas_decrease * c->err1_prev;
    if (c->rho_policy == 1) grow = grow && !capped;
    else if (c->rho_policy == 2) grow = grow && (!capped || err1 > c->err1_prev);
    if (grow) c->rho = fmin(c->rho * c->rho_growth, c->rho_max);
    c->err1_prev = err1;
    if (c->outer >= c->max_outer) {
        c->status = 6;                          // LORADS_ERR_MAXITER
        c->solve_done = 1;
        return;
    }
    c->hit_cap_streak = capped ? c->hit_cap_streak + 1 : 0;
    if (c->hit_cap_streak >= c->rank_threshold) {
        c->hit_cap_streak = 0;
        c->pause = 1;                           // host grows the rank
    }
}

// Start of a solve: err1 at R0 and the outer phase for the first gradient.
__device__ inline void ctrl_init_apply(Ctrl* c, const double* sc, const double* so) {
    c->err1_prev = sqrt(fmax(sc[PC_ZZ], 0.0)) / (1.0 + c->bnorm_inf);
    c->err1 = c->err1_prev;
    c->primal_obj = so[PO_CRR];
    c->phase = PHASE_OUTER;
    c->solve_done = 0;
    c->pause = 0;
}

}  // namespace lorads
