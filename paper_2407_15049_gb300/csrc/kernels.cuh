// Streaming kernels of the LoRADS hot path (templates; instantiated per
// precision in kern_*.cu).  Every kernel is memory-bound by design: rows of the
// n x ld factors are read with 16-byte vector loads by groups of L lanes,
// sparse rows are gathered through L2, and all reductions end in per-block FP64
// partial sums that a single-block control kernel folds in a fixed order.
#pragma once

#include <type_traits>
#include "common.cuh"

namespace lorads {

// ------------------------------------------------------------------ problem arrays
struct ProbDev {
    int64_t n, m;
    // C: full symmetric CSR
    const int64_t* c_rowptr;
    const int32_t* c_col;
    const double* c_val;
    const float* c_val32;
    const dfloat* c_valdf;
    // diagonal constraints by row: constraint index (-1: none) and coefficient
    const int32_t* dk;
    const double* da;
    const float* da32;          // float and double-float mirrors of da and b for the
    const dfloat* da_df;        // FP32-unit paths (no per-row FP64 there)
    const dfloat* b_df;
    // off-diagonal constraints as a symmetric pattern: slot -> (column, constraint, coef)
    const int64_t* a_rowptr;
    const int32_t* a_col;
    const int32_t* a_k;
    const double* a_a;
    // constraint list, fused diagonal constraints first: triplets (row <= col, coef) in
    // list order and the constraint of each list position.  k_ptr (general form,
    // constraints with several triplets): position q owns triplets k_ptr[q]..k_ptr[q+1]-1;
    // null: position q is triplet q.
    const int32_t* k_row;
    const int32_t* k_col;
    const double* k_a;
    const int32_t* k_id;
    const int64_t* k_ptr;
    int64_t m_diag, m_off;
    const double* b;
    // double-float mirrors of the constraint coefficients (list order and pattern
    // order) for the FP32-unit paths; may be null for FP64 callers
    const dfloat* k_adf;
    const dfloat* a_adf;
};

// ------------------------------------------------------------------ gating
// Kernels of the captured iteration graph check the control block first and
// return at once when the current phase does not need them.
enum { PH_ALWAYS = 0, PH_INNER = 1, PH_STEP = 2, PH_OUTER = 3 };

__device__ __forceinline__ bool gated_off(const Ctrl* g, int ph) {
    if (g == nullptr || ph == PH_ALWAYS) return false;
    if (g->solve_done | g->pause) return true;
    if (ph == PH_OUTER) return g->phase != PHASE_OUTER;
    if (g->phase != PHASE_INNER) return true;
    if (ph == PH_STEP) return g->step_ok == 0;
    return false;
}

template <typename T>
using arith_t = typename Arith<T>::type;
template <typename T>
using A_of_t = arith_t<T>;

// precision rank of an arithmetic type: float < double-float < double
template <typename T> struct PrecRank;
template <> struct PrecRank<float> { static constexpr int v = 0; };
template <> struct PrecRank<dfloat> { static constexpr int v = 1; };
template <> struct PrecRank<double> { static constexpr int v = 2; };

template <int R> struct RankType;
template <> struct RankType<0> { using type = float; };
template <> struct RankType<1> { using type = dfloat; };
template <> struct RankType<2> { using type = double; };

// wider of the arithmetic types of two storage types
template <typename A, typename B>
using wide_t = typename RankType<(PrecRank<arith_t<A>>::v > PrecRank<arith_t<B>>::v ? PrecRank<arith_t<A>>::v
                                                                                   : PrecRank<arith_t<B>>::v)>::type;

// partial-sum type: double on the all-FP64 path, double-float otherwise (no FP64 pipe)
template <typename A, typename B>
using part_t = std::conditional_t<std::is_same_v<arith_t<A>, double> && std::is_same_v<arith_t<B>, double>,
                                  double, dfloat>;

// value type of C entries multiplied against rows of type TX
template <typename TX>
using cval_t = arith_t<TX>;

template <typename TV> __device__ __forceinline__ const TV* cvals(const ProbDev& p);
template <> __device__ __forceinline__ const double* cvals<double>(const ProbDev& p) { return p.c_val; }
template <> __device__ __forceinline__ const float* cvals<float>(const ProbDev& p) { return p.c_val32; }
template <> __device__ __forceinline__ const dfloat* cvals<dfloat>(const ProbDev& p) { return p.c_valdf; }

// per-row scalar type of the row-update math: double on the FP64 path,
// otherwise the arithmetic type of R (double-float or float)
template <typename TR, typename TD>
using rowscalar_t = std::conditional_t<std::is_same_v<arith_t<TR>, double> && std::is_same_v<arith_t<TD>, double>,
                                       double, arith_t<TR>>;

template <typename S> __device__ __forceinline__ S ld_scalar(const double* d, const dfloat* df, int64_t k);
template <> __device__ __forceinline__ double ld_scalar<double>(const double* d, const dfloat*, int64_t k) {
    return __ldg(d + k);
}
template <> __device__ __forceinline__ dfloat ld_scalar<dfloat>(const double*, const dfloat* df, int64_t k) {
    const float2 v = __ldg(reinterpret_cast<const float2*>(df + k));
    return dfloat(v.x, v.y);
}
template <> __device__ __forceinline__ float ld_scalar<float>(const double*, const dfloat* df, int64_t k) {
    return __ldg(reinterpret_cast<const float*>(df + k));     // hi part
}

// type of the per-row z cache (and of the line-search row terms): double on the
// FP64 path, otherwise the arithmetic type of the direction D
template <typename TD, typename TR>
using zrow_t = std::conditional_t<std::is_same_v<part_t<TD, TR>, double>, double, arith_t<TD>>;

// read-only scalar loads
__device__ __forceinline__ double ldv(const double* p) { return __ldg(p); }
__device__ __forceinline__ float ldv(const float* p) { return __ldg(p); }
__device__ __forceinline__ dfloat ldv(const dfloat* p) {
    const float2 v = __ldg(reinterpret_cast<const float2*>(p));
    return dfloat(v.x, v.y);
}

// Warp-uniform row loop: each warp owns 32/L consecutive rows per trip, so the
// group shuffles below always see the full warp.  Packed groups (`dense`): L may
// be any width up to 32 (one unit per lane, L = units per row); the warp holds
// floor(32/L) rows and its last 32 mod L lanes take no row (`live` false), e.g.
// ld = 24: 5 rows of 6 lanes instead of 4 rows of 8 lanes with 2 idle each.
struct RowLoop {
    int L, lig, gw, rows_per_warp, base_lane;
    bool live;
    int64_t first, stride;
    __device__ __forceinline__ RowLoop(int L_, VGrid vg, bool dense = false) : L(L_) {
        const int lane = threadIdx.x & 31;
        if (dense) {
            gw = lane / L;
            lig = lane - gw * L;
            rows_per_warp = 32 / L;
            live = gw < rows_per_warp;
        } else {
            lig = threadIdx.x & (L - 1);
            gw = lane / L;
            rows_per_warp = 32 / L;
            live = true;
        }
        base_lane = live ? gw * L : 0;
        const int64_t warp = (vg.bid * (int64_t)blockDim.x + threadIdx.x) >> 5;
        const int64_t nwarps = ((int64_t)vg.nblk * blockDim.x) >> 5;
        first = warp * rows_per_warp;
        stride = nwarps * rows_per_warp;
    }
};

// Sum over the L lanes of a packed group, taken in lane order by every lane (the
// same bits in each lane of the group); all 32 lanes take part in the shuffles.
__device__ __forceinline__ float shfl_idx(float v, int src) { return __shfl_sync(0xffffffffu, v, src); }
__device__ __forceinline__ double shfl_idx(double v, int src) { return __shfl_sync(0xffffffffu, v, src); }
__device__ __forceinline__ dfloat shfl_idx(dfloat v, int src) {
    return dfloat(__shfl_sync(0xffffffffu, v.hi, src), __shfl_sync(0xffffffffu, v.lo, src));
}
template <typename V>
__device__ __forceinline__ V group_sum_packed(V v, int L, int base_lane) {
    V t = shfl_idx(v, base_lane);
    for (int k = 1; k < L; ++k) t += shfl_idx(v, base_lane + k);
    return t;
}

// Row helpers: lane `lig` of a group of L handles units c*L + lig < Q.
// Units past Q are zero on load and skipped on store.
template <typename T, int CPL>
__device__ __forceinline__ void load_row(Unit<T> (&u)[CPL], const T* base, int64_t row, int ld, int L, int Q, int lig) {
    const T* p = base + row * (int64_t)ld + lig * 4;
#pragma unroll
    for (int c = 0; c < CPL; ++c) {
        if (c * L + lig < Q) u[c].load(p + c * L * 4);
        else
#pragma unroll
            for (int e = 0; e < 4; ++e) u[c].v[e] = 0;
    }
}

template <typename T, int CPL>
__device__ __forceinline__ void load_row_stream(Unit<T> (&u)[CPL], const T* base, int64_t row, int ld, int L, int Q,
                                                int lig) {
    const T* p = base + row * (int64_t)ld + lig * 4;
#pragma unroll
    for (int c = 0; c < CPL; ++c) {
        if (c * L + lig < Q) u[c].load_stream(p + c * L * 4);
        else
#pragma unroll
            for (int e = 0; e < 4; ++e) u[c].v[e] = 0;
    }
}

// L2 prefetch (no register, no wait) of one address of global memory.
__device__ __forceinline__ void prefetch_l2(const void* a) {
    asm volatile("prefetch.global.L2 [%0];" ::"l"(a));
}

// L2 prefetch of the units of `row` that lane `lig` loads: issued one row
// iteration ahead, it turns the dependent loads of that iteration into L2 hits.
template <typename T, int CPL>
__device__ __forceinline__ void prefetch_row(const T* base, int64_t row, int ld, int L, int Q, int lig) {
    const T* p = base + row * (int64_t)ld + lig * 4;
#pragma unroll
    for (int c = 0; c < CPL; ++c)
        if (c * L + lig < Q) prefetch_l2(p + c * L * 4);
}

template <typename T, int CPL>
__device__ __forceinline__ void store_row(const Unit<T> (&u)[CPL], T* base, int64_t row, int ld, int L, int Q, int lig) {
    T* p = base + row * (int64_t)ld + lig * 4;
#pragma unroll
    for (int c = 0; c < CPL; ++c)
        if (c * L + lig < Q) u[c].store_stream(p + c * L * 4);
}

template <typename A, typename T1, typename T2, int CPL>
__device__ __forceinline__ A dot_units(const Unit<T1> (&x)[CPL], const Unit<T2> (&y)[CPL]) {
    A s = A(0);
#pragma unroll
    for (int c = 0; c < CPL; ++c)
#pragma unroll
        for (int e = 0; e < 4; ++e) s = fma(A(x[c].v[e]), A(y[c].v[e]), s);
    return s;
}

// Value an element has once stored as T (bf16 rounds; every other type keeps it).
template <typename T, typename A>
__device__ __forceinline__ A as_stored(A v) {
    if constexpr (std::is_same_v<T, __nv_bfloat16>) return A(__bfloat162float(__float2bfloat16_rn(float(v))));
    else return v;
}

// ================================================================== SpMM over C
// out = C X  (+ the diagonal-constraint part -A*(v) X when v != nullptr),
// optional epilogues:
//   EPI_LS : line-search partials at R (= argument R) along D (= X):
//            p1 = 2<CD, R>, p2 = <CD, D>, and for diagonal constraints
//            sum y~ q1, sum y~ q2, sum q1^2, sum q1 q2, sum q2^2
//   EPI_OBJ: <C X, X> (objective with X = R)
enum { EPI_NONE = 0, EPI_LS = 1, EPI_OBJ = 2 };

// PF (compile-time, so that the default form carries none of the others' code):
// 0 none, 1 the next row's bounds and L2 prefetches, 2 also two rows ahead.
template <typename TX, typename TO, typename TR, int CPL, int EPI, bool DENSE = false, int PF = 0>
__device__ __forceinline__ void
k_spmm_c_body(ProbDev p, const TX* __restrict__ X, TO* __restrict__ out, int ld, int L, int Q,
         const double* __restrict__ v, int write_out,
         const TR* __restrict__ R, const double* __restrict__ y, const void* __restrict__ zrow_v,
         const dfloat* __restrict__ ydf, const Ctrl* ctrl, double rho_arg, double* __restrict__ part, VGrid vg) {
    using A = arith_t<TO>;
    using TV = cval_t<TX>;
    using PA = part_t<TO, TR>;
    // scalar type of the per-row line-search terms: double on the FP64 path, otherwise
    // the arithmetic type of the direction (float, or double-float on the DF64 path)
    using LS = zrow_t<TX, TR>;
    const LS* __restrict__ zrow = static_cast<const LS*>(zrow_v);
    constexpr int NQ = EPI == EPI_LS ? PL_N : (EPI == EPI_OBJ ? PO_N : 1);
    PA accq[NQ];
#pragma unroll
    for (int q = 0; q < NQ; ++q) accq[q] = PA(0);
    const double rho = ctrl ? ctrl->rho : rho_arg;
    const LS rho_s = LS(rho);
    const TV* __restrict__ cv = cvals<TV>(p);
    static_assert(!DENSE || CPL == 1, "packed row groups hold one unit per lane");
    RowLoop rl(L, vg, DENSE);
    // With pf: the bounds (and constraint index) of this group's next row are loaded one
    // iteration ahead, and that row's entries, own-row streams and scalars are prefetched
    // into L2, so of its dependent load phases only the neighbour gathers wait on HBM.
    const bool own_row = EPI == EPI_LS || EPI == EPI_OBJ || (v != nullptr && p.dk != nullptr);
    // With pf == 2 the bounds run two rows ahead: the stored entries of the row after
    // next are prefetched, so that the next row's column indices are L2 hits one
    // iteration early and each lane can prefetch one neighbour row of D for it.
    int64_t s_nx = -1, e_nx = -1;
    int64_t s_n2 = -1, e_n2 = -1;
    for (int64_t base = rl.first; base < p.n; base += rl.stride) {
        const int64_t i = base + rl.gw;
        const bool act = rl.live && i < p.n;
        const int64_t s_cur = s_nx, e_cur = e_nx;
        s_nx = -1;
        int k_nx = -1;
        int jn = -1;
        if (PF != 0 && rl.live) {
            const int64_t nx = i + rl.stride;
            if (nx < p.n) {
                if (PF == 2 && s_n2 >= 0) {
                    s_nx = s_n2;
                    e_nx = e_n2;
                } else {
                    s_nx = __ldg(p.c_rowptr + nx);
                    e_nx = __ldg(p.c_rowptr + nx + 1);
                }
                if (own_row) prefetch_row<TX, CPL>(X, nx, ld, L, Q, rl.lig);
                if constexpr (EPI == EPI_LS) prefetch_row<TR, CPL>(R, nx, ld, L, Q, rl.lig);
                if (p.dk != nullptr && rl.lig == 0) {
                    k_nx = __ldg(p.dk + nx);
                    prefetch_l2(p.da + nx);
                    if (p.da_df != nullptr) prefetch_l2(p.da_df + nx);
                    if constexpr (EPI == EPI_LS)
                        if (zrow != nullptr) prefetch_l2(zrow + nx);
                }
            }
            if constexpr (PF == 2) {
                const int64_t n2 = nx + rl.stride;
                s_n2 = -1;
                if (n2 < p.n) {
                    s_n2 = __ldg(p.c_rowptr + n2);
                    e_n2 = __ldg(p.c_rowptr + n2 + 1);
                }
                if (s_nx >= 0 && s_nx + rl.lig < e_nx) jn = __ldg(p.c_col + s_nx + rl.lig);
            }
        }
        A acc[CPL][4];
#pragma unroll
        for (int c = 0; c < CPL; ++c)
#pragma unroll
            for (int e = 0; e < 4; ++e) acc[c][e] = A(0);
        if (act) {
            int64_t s = s_cur >= 0 ? s_cur : __ldg(p.c_rowptr + i);
            const int64_t e_ = s_cur >= 0 ? e_cur : __ldg(p.c_rowptr + i + 1);
            // nonzeros in flight per lane: with one unit per lane, all the gathers of a
            // row of up to 8 stored entries are issued together (masked slots load nothing)
            constexpr int UN = CPL == 1 ? 8 : (CPL == 2 ? 4 : 3);
            for (; s < e_; s += UN) {
                if (CPL != 1 && s + UN > e_) break;
                int j[UN];
                A w[UN];
#pragma unroll
                for (int u = 0; u < UN; ++u) {
                    const bool ok = s + u < e_;
                    j[u] = ok ? __ldg(p.c_col + s + u) : -1;
                    w[u] = ok ? A(ldv(cv + s + u)) : A(0);
                }
                Unit<TX> x[UN][CPL];
#pragma unroll
                for (int u = 0; u < UN; ++u) {
                    if (j[u] >= 0) load_row<TX, CPL>(x[u], X, j[u], ld, L, Q, rl.lig);
                    else
#pragma unroll
                        for (int c = 0; c < CPL; ++c)
#pragma unroll
                            for (int e = 0; e < 4; ++e) x[u][c].v[e] = 0;
                }
#pragma unroll
                for (int u = 0; u < UN; ++u)
                    if (j[u] >= 0)
#pragma unroll
                        for (int c = 0; c < CPL; ++c)
#pragma unroll
                            for (int e = 0; e < 4; ++e) acc[c][e] = fma(w[u], A(x[u][c].v[e]), acc[c][e]);
            }
            for (; s < e_; ++s) {
                const int j0 = __ldg(p.c_col + s);
                const A w0 = A(ldv(cv + s));
                Unit<TX> x0[CPL];
                load_row<TX, CPL>(x0, X, j0, ld, L, Q, rl.lig);
#pragma unroll
                for (int c = 0; c < CPL; ++c)
#pragma unroll
                    for (int e = 0; e < 4; ++e) acc[c][e] = fma(w0, A(x0[c].v[e]), acc[c][e]);
            }
            if constexpr (PF == 2) {
                // one neighbour row of the next row (its first and last element), and the
                // stored entries of the row after next
                if (jn >= 0) {
                    const TX* rowp = X + (int64_t)jn * ld;
                    prefetch_l2(rowp);
                    prefetch_l2(rowp + ld - 1);
                }
                if (s_n2 >= 0 && rl.lig < 2 && e_n2 > s_n2) {
                    const int64_t q = rl.lig == 0 ? s_n2 : e_n2 - 1;
                    prefetch_l2(p.c_col + q);
                    prefetch_l2(cv + q);
                }
            } else if (s_nx >= 0 && rl.lig < 2 && e_nx > s_nx) {
                // the next row's stored entries (first and last sector) and multiplier terms
                const int64_t q = rl.lig == 0 ? s_nx : e_nx - 1;
                prefetch_l2(p.c_col + q);
                prefetch_l2(cv + q);
            }
            if (k_nx >= 0) {
                if (v != nullptr) prefetch_l2(v + k_nx);
                if constexpr (EPI == EPI_LS) {
                    prefetch_l2(ydf ? static_cast<const void*>(ydf + k_nx) : static_cast<const void*>(y + k_nx));
                    if (zrow == nullptr) prefetch_l2(p.b_df ? static_cast<const void*>(p.b_df + k_nx)
                                                            : static_cast<const void*>(p.b + k_nx));
                }
            }
            if (v != nullptr && p.dk != nullptr) {
                const int k = __ldg(p.dk + i);
                if (k >= 0) {
                    const A w = A(-__ldg(p.da + i) * __ldg(v + k));
                    Unit<TX> xi[CPL];
                    load_row<TX, CPL>(xi, X, i, ld, L, Q, rl.lig);
#pragma unroll
                    for (int c = 0; c < CPL; ++c)
#pragma unroll
                        for (int e = 0; e < 4; ++e) acc[c][e] = fma(w, A(xi[c].v[e]), acc[c][e]);
                }
            }
            if (write_out) {
                Unit<TO> o[CPL];
#pragma unroll
                for (int c = 0; c < CPL; ++c)
#pragma unroll
                    for (int e = 0; e < 4; ++e) o[c].v[e] = acc[c][e];
                store_row<TO, CPL>(o, out, i, ld, L, Q, rl.lig);
            }
        }
        if constexpr (EPI == EPI_OBJ) {
            if (act) {
                Unit<TX> xi[CPL];
                load_row<TX, CPL>(xi, X, i, ld, L, Q, rl.lig);
                A t = A(0);
#pragma unroll
                for (int c = 0; c < CPL; ++c)
#pragma unroll
                    for (int e = 0; e < 4; ++e) t = fma(acc[c][e], A(xi[c].v[e]), t);
                accq[PO_CRR] += PA(t);
            }
        }
        if constexpr (EPI == EPI_LS) {
            using AW = wide_t<TR, TX>;           // |r|^2 (when not cached) and <CD, R>
            using AD = arith_t<TX>;              // products of D with D and with R
            AW t_p1 = AW(0), t_rr = AW(0);
            AD t_p2 = AD(0), t_rd = AD(0), t_dd = AD(0);
            if (act) {
                Unit<TX> di[CPL];
                Unit<TR> ri[CPL];
                load_row<TX, CPL>(di, X, i, ld, L, Q, rl.lig);
                load_row_stream<TR, CPL>(ri, R, i, ld, L, Q, rl.lig);
#pragma unroll
                for (int c = 0; c < CPL; ++c)
#pragma unroll
                    for (int e = 0; e < 4; ++e) {
                        const AD d = AD(di[c].v[e]);
                        const AD rlow = AD(ri[c].v[e]);
                        t_p2 = fma(AD(acc[c][e]), d, t_p2);
                        t_rd = fma(rlow, d, t_rd);
                        t_dd = fma(d, d, t_dd);
                        if (zrow == nullptr) {
                            const AW r = AW(ri[c].v[e]);
                            t_p1 = fma(AW(acc[c][e]), r, t_p1);
                            t_rr = fma(r, r, t_rr);
                        }
                    }
            }
            accq[PL_P2] += t_p2;
            if (zrow == nullptr) accq[PL_P1] += PA(AW(2) * t_p1);
            if (p.dk != nullptr) {
                if constexpr (DENSE) {
                    if (zrow == nullptr) t_rr = group_sum_packed(t_rr, L, rl.base_lane);
                    t_rd = group_sum_packed(t_rd, L, rl.base_lane);
                    t_dd = group_sum_packed(t_dd, L, rl.base_lane);
                } else {
                    if (zrow == nullptr) t_rr = group_sum(t_rr, L);
                    t_rd = group_sum(t_rd, L);
                    t_dd = group_sum(t_dd, L);
                }
                if (act && rl.lig == 0) {
                    const int k = __ldg(p.dk + i);
                    if (k >= 0) {
                        if constexpr (std::is_same_v<LS, double>) {
                            const double a = __ldg(p.da + i);
                            const double z = zrow ? zrow[i] : a * double(t_rr) - __ldg(p.b + k);
                            const double yt = __ldg(y + k) - rho * z;
                            const double q1 = 2.0 * a * double(t_rd);
                            const double q2 = a * double(t_dd);
                            accq[PL_YQ1] += PA(yt * q1);
                            accq[PL_YQ2] += PA(yt * q2);
                            accq[PL_Q1Q1] += PA(q1 * q1);
                            accq[PL_Q1Q2] += PA(q1 * q2);
                            accq[PL_Q2Q2] += PA(q2 * q2);
                        } else {
                            // line-search terms in the direction's arithmetic; z from the
                            // row cache, else |r|^2 in double-float
                            const LS a = ld_scalar<LS>(p.da, p.da_df, i);
                            LS z;
                            if (zrow) {
                                z = zrow[i];
                            } else {
                                const dfloat zz = dfloat(t_rr) * ld_scalar<dfloat>(p.da, p.da_df, i) -
                                                  ld_scalar<dfloat>(p.b, p.b_df, k);
                                z = LS(zz);
                            }
                            const LS yv = ydf ? ld_scalar<LS>(y, ydf, k) : LS(__ldg(y + k));
                            const LS yt = yv - rho_s * z;
                            const LS q1 = LS(2) * a * LS(t_rd);
                            const LS q2 = a * LS(t_dd);
                            accq[PL_YQ1] += PA(yt * q1);
                            accq[PL_YQ2] += PA(yt * q2);
                            accq[PL_Q1Q1] += PA(q1 * q1);
                            accq[PL_Q1Q2] += PA(q1 * q2);
                            accq[PL_Q2Q2] += PA(q2 * q2);
                        }
                    }
                }
            }
        }
    }
    if constexpr (EPI != EPI_NONE) block_partials<NQ>(accq, part, vg.pslot);
}

// ================================================================== SpMM over the
// off-diagonal constraint pattern:  out = beta_acc * out + alpha * A*_off(v) X
// VDF: v holds double-float values and each weight alpha a v_k is formed in the
// output's arithmetic from the double-float coefficient mirror (no FP64
// operation); otherwise v is double and the weight is formed in FP64.
template <typename TX, typename TO, int CPL, bool VDF>
__device__ __forceinline__ A_of_t<TO> spmm_a_weight(const ProbDev& p, const void* v, double alpha, A_of_t<TO> alpha_a,
                                                   int64_t s) {
    using A = A_of_t<TO>;
    const int k = __ldg(p.a_k + s);
    if constexpr (VDF) {
        return alpha_a * ld_scalar<A>(nullptr, p.a_adf, s) * ld_scalar<A>(nullptr, static_cast<const dfloat*>(v), k);
    } else {
        return A(alpha * __ldg(p.a_a + s) * __ldg(static_cast<const double*>(v) + k));
    }
}

template <typename TX, typename TO, int CPL, bool VDF>
__device__ __forceinline__ void
k_spmm_a_body(ProbDev p, const TX* __restrict__ X, TO* __restrict__ out, int ld, int L, int Q,
         const void* __restrict__ v, double alpha, int accumulate, VGrid vg) {
    using A = arith_t<TO>;
    const A alpha_a = A(alpha);
    RowLoop rl(L, vg);
    for (int64_t base = rl.first; base < p.n; base += rl.stride) {
        const int64_t i = base + rl.gw;
        if (i >= p.n) continue;
        A acc[CPL][4];
#pragma unroll
        for (int c = 0; c < CPL; ++c)
#pragma unroll
            for (int e = 0; e < 4; ++e) acc[c][e] = A(0);
        const int64_t s0 = __ldg(p.a_rowptr + i), s1 = __ldg(p.a_rowptr + i + 1);
        int64_t s = s0;
        constexpr int UN = CPL == 1 ? 4 : 2;           // entries in flight per lane
        for (; s + UN <= s1; s += UN) {
            int j[UN];
            A w[UN];
#pragma unroll
            for (int u = 0; u < UN; ++u) {
                j[u] = __ldg(p.a_col + s + u);
                w[u] = spmm_a_weight<TX, TO, CPL, VDF>(p, v, alpha, alpha_a, s + u);
            }
            Unit<TX> x[UN][CPL];
#pragma unroll
            for (int u = 0; u < UN; ++u) load_row<TX, CPL>(x[u], X, j[u], ld, L, Q, rl.lig);
#pragma unroll
            for (int u = 0; u < UN; ++u)
#pragma unroll
                for (int c = 0; c < CPL; ++c)
#pragma unroll
                    for (int e = 0; e < 4; ++e) acc[c][e] = fma(w[u], A(x[u][c].v[e]), acc[c][e]);
        }
        for (; s < s1; ++s) {
            const int j = __ldg(p.a_col + s);
            const A w = spmm_a_weight<TX, TO, CPL, VDF>(p, v, alpha, alpha_a, s);
            Unit<TX> x[CPL];
            load_row<TX, CPL>(x, X, j, ld, L, Q, rl.lig);
#pragma unroll
            for (int c = 0; c < CPL; ++c)
#pragma unroll
                for (int e = 0; e < 4; ++e) acc[c][e] = fma(w, A(x[c].v[e]), acc[c][e]);
        }
        Unit<TO> o[CPL];
        if (accumulate) {
            load_row<TO, CPL>(o, out, i, ld, L, Q, rl.lig);
#pragma unroll
            for (int c = 0; c < CPL; ++c)
#pragma unroll
                for (int e = 0; e < 4; ++e) o[c].v[e] = arith_t<TO>(o[c].v[e]) + acc[c][e];
        } else {
#pragma unroll
            for (int c = 0; c < CPL; ++c)
#pragma unroll
                for (int e = 0; e < 4; ++e) o[c].v[e] = acc[c][e];
        }
        store_row<TO, CPL>(o, out, i, ld, L, Q, rl.lig);
    }
}

// ================================================================== constraint pass
// One group of L lanes per constraint t in [k0, k1) of the ordered list
// (diagonal constraints first).  With f = 1 (i == j) or 2 (i < j):
//   CONS_EVAL: out[k] = a (u_i.v_j + [i!=j] u_j.v_i)                  = <A_k, U V^T>
//   CONS_LS  : z = f a r_i.r_j - b, y~ = y - rho z, q1 = f a (r_i.d_j + d_i.r_j),
//              q2 = f a d_i.d_j; partials of y~q1, y~q2, q1^2, q1q2, q2^2
//   CONS_YTIL: out[k] = y~ ;  partial |z|^2
//   CONS_YUPD: y[k] <- y~ (and its double-float mirror);  partials |z|^2, b^T y_new
//   CONS_ZZ  : partial |z|^2
enum { CONS_EVAL = 0, CONS_LS = 1, CONS_YTIL = 2, CONS_YUPD = 3, CONS_ZZ = 4 };

// General form of the constraint pass: list position q is one constraint whose
// triplets t (i <= j, a) are summed with the weights of the triplet convention:
//   <A_k, U V^T> = sum_t a (u_i.v_j + [i != j] u_j.v_i),
// and, with f = 1 (i == j) or 2, z = sum_t f a r_i.r_j - b_k, q1 = sum_t f a
// (r_i.d_j + d_i.r_j) / (1 + [i == j]) ... written per triplet as in the single-triplet
// path, then the same per-constraint formulas.  Each lane accumulates its share of
// every triplet's dots; the group sum follows the triplet loop (no shuffle inside
// the loop, whose trip count differs between the groups of a warp).
template <typename TU, typename TV, int CPL, int MODE>
__device__ __forceinline__ void
k_cons_general(ProbDev p, int64_t k0, int64_t k1, const TU* __restrict__ U, const TV* __restrict__ V, int ld, int L,
               int Q, double* y, void* __restrict__ out, void* zk, dfloat* ydf, const Ctrl* ctrl, double rho_arg,
               double* __restrict__ part, VGrid vg) {
    constexpr int NQ = MODE == CONS_LS ? PL_N : PC_N;
    using PA = part_t<TU, TV>;
    PA accq[NQ];
#pragma unroll
    for (int q = 0; q < NQ; ++q) accq[q] = PA(0);
    const double rho = ctrl ? ctrl->rho : rho_arg;
    const bool same = (const void*)U == (const void*)V;
    using AU = wide_t<TU, TU>;
    using AW = wide_t<TU, TV>;
    using AV = wide_t<TV, TV>;
    using CS = std::conditional_t<std::is_same_v<PA, double>, double, dfloat>;
    const CS rho_c = CS(rho);
    CS* zkc = static_cast<CS*>(zk);
    RowLoop rl(L, vg);
    const int64_t cnt = k1 - k0;
    for (int64_t base = rl.first; base < cnt; base += rl.stride) {
        const int64_t q = k0 + base + rl.gw;
        const bool act = q < k1;
        // per-lane weighted dots: z part (f a u_i.u_j), q1 part, q2 part / EVAL value
        AU s_z = AU(0);
        AW s_1 = AW(0);
        AV s_2 = AV(0);
        if (act) {
            const int64_t t0 = __ldg(p.k_ptr + q), t1 = __ldg(p.k_ptr + q + 1);
            for (int64_t t = t0; t < t1; ++t) {
                const int i = __ldg(p.k_row + t), j = __ldg(p.k_col + t);
                const bool dg = i == j;
                const double a = __ldg(p.k_a + t);
                const double fa = dg ? a : 2.0 * a;
                Unit<TU> ui[CPL], uj[CPL];
                load_row<TU, CPL>(ui, U, i, ld, L, Q, rl.lig);
                if (!dg) load_row<TU, CPL>(uj, U, j, ld, L, Q, rl.lig);
                if constexpr (MODE == CONS_EVAL) {
                    if (same) {
                        s_z = s_z + AU(fa) * (dg ? dot_units<AU>(ui, ui) : dot_units<AU>(ui, uj));
                    } else {
                        Unit<TV> vi[CPL], vj[CPL];
                        load_row<TV, CPL>(vi, V, i, ld, L, Q, rl.lig);
                        if (dg) {
                            s_1 = s_1 + AW(a) * dot_units<AW>(ui, vi);
                        } else {
                            load_row<TV, CPL>(vj, V, j, ld, L, Q, rl.lig);
                            s_1 = s_1 + AW(a) * (dot_units<AW>(ui, vj) + dot_units<AW>(uj, vi));
                        }
                    }
                } else {
                    if (MODE != CONS_LS || zk == nullptr)
                        s_z = s_z + AU(fa) * (dg ? dot_units<AU>(ui, ui) : dot_units<AU>(ui, uj));
                    if constexpr (MODE == CONS_LS) {
                        Unit<TV> vi[CPL], vj[CPL];
                        load_row<TV, CPL>(vi, V, i, ld, L, Q, rl.lig);
                        if (dg) {
                            const AW d = dot_units<AW>(ui, vi);
                            s_1 = s_1 + AW(fa) * (d + d);
                            s_2 = s_2 + AV(fa) * dot_units<AV>(vi, vi);
                        } else {
                            load_row<TV, CPL>(vj, V, j, ld, L, Q, rl.lig);
                            s_1 = s_1 + AW(fa) * (dot_units<AW>(ui, vj) + dot_units<AW>(vi, uj));
                            s_2 = s_2 + AV(fa) * dot_units<AV>(vi, vj);
                        }
                    }
                }
            }
        }
        s_z = group_sum(s_z, L);
        s_1 = group_sum(s_1, L);
        s_2 = group_sum(s_2, L);
        if (act && rl.lig == 0) {
            const int k = __ldg(p.k_id + q);
            if constexpr (MODE == CONS_EVAL) {
                static_cast<double*>(out)[k] = same ? double(s_z) : double(s_1);
            } else {
                CS yk = CS(0.0), bk;
                if constexpr (MODE != CONS_ZZ) {
                    if constexpr (std::is_same_v<CS, double>) yk = y[k];
                    else yk = ydf ? ld_scalar<CS>(y, ydf, k) : CS(y[k]);
                }
                if constexpr (std::is_same_v<CS, double>) bk = __ldg(p.b + k);
                else bk = p.b_df ? ld_scalar<CS>(p.b, p.b_df, k) : CS(__ldg(p.b + k));
                const CS z = (MODE == CONS_LS && zk != nullptr) ? zkc[k] : CS(s_z) - bk;
                if constexpr (MODE == CONS_LS) {
                    const CS yt = yk - rho_c * z;
                    const CS q1 = CS(s_1);
                    const CS q2 = CS(s_2);
                    accq[PL_YQ1] += PA(yt * q1);
                    accq[PL_YQ2] += PA(yt * q2);
                    accq[PL_Q1Q1] += PA(q1 * q1);
                    accq[PL_Q1Q2] += PA(q1 * q2);
                    accq[PL_Q2Q2] += PA(q2 * q2);
                } else {
                    accq[PC_ZZ] += PA(z * z);
                    if constexpr (MODE == CONS_YTIL) {
                        static_cast<CS*>(out)[k] = yk - rho_c * z;
                        if (zk != nullptr) zkc[k] = z;
                    } else if constexpr (MODE == CONS_YUPD) {
                        const CS yn = yk - rho_c * z;
                        y[k] = double(yn);
                        if constexpr (std::is_same_v<CS, dfloat>) {
                            if (ydf != nullptr) ydf[k] = yn;
                        } else {
                            if (ydf != nullptr) ydf[k] = dfloat(yn);
                        }
                        accq[PC_BY] += PA(bk * yn);
                    }
                }
            }
        }
    }
    if constexpr (MODE != CONS_EVAL) block_partials<NQ>(accq, part, vg.pslot);
}

template <typename TU, typename TV, int CPL, int MODE>
__device__ __forceinline__ void
k_cons_body(ProbDev p, int64_t k0, int64_t k1, const TU* __restrict__ U, const TV* __restrict__ V, int ld, int L, int Q,
       double* y, void* __restrict__ out, void* zk, dfloat* ydf, const Ctrl* ctrl, double rho_arg,
       double* __restrict__ part, VGrid vg) {
    if (p.k_ptr != nullptr) {
        k_cons_general<TU, TV, CPL, MODE>(p, k0, k1, U, V, ld, L, Q, y, out, zk, ydf, ctrl, rho_arg, part, vg);
        return;
    }
    constexpr int NQ = MODE == CONS_LS ? PL_N : PC_N;
    using PA = part_t<TU, TV>;
    PA accq[NQ];
#pragma unroll
    for (int q = 0; q < NQ; ++q) accq[q] = PA(0);
    const double rho = ctrl ? ctrl->rho : rho_arg;
    const bool same = (const void*)U == (const void*)V;
    using AU = wide_t<TU, TU>;
    using AW = wide_t<TU, TV>;
    using AV = wide_t<TV, TV>;
    // per-constraint scalars: double on the all-FP64 path, double-float otherwise
    // (GB300's FP64 rate is ~1/64 of FP32; conversions run on the FP64 pipe too).
    // z = A(RR^T)_k - b_k, y~ and the cached z use the same type (zk, out: CS arrays).
    using CS = std::conditional_t<std::is_same_v<PA, double>, double, dfloat>;
    const CS rho_c = CS(rho);
    CS* zkc = static_cast<CS*>(zk);
    // what each mode gathers besides u_i, u_j
    constexpr bool NEED_V = MODE == CONS_EVAL || MODE == CONS_LS;
    // constraints in flight per lane group: the index, coefficient and multiplier
    // loads and all row gathers of UC constraints are issued before any dot product
    constexpr int UC = CPL == 1 ? (MODE == CONS_LS || MODE == CONS_EVAL ? 2 : 3) : 1;
    RowLoop rl(L, vg);
    const int64_t cnt = k1 - k0;
    const int64_t step = (int64_t)rl.rows_per_warp;
    for (int64_t base = rl.first * UC; base < cnt; base += rl.stride * UC) {
        int64_t t[UC];
        bool act[UC], diag[UC];
        int i[UC], j[UC], kid[UC];
        CS ak[UC], yk[UC], zb[UC];          // coefficient, y_k, and z_k (cached) or b_k
        Unit<TU> ui[UC][CPL], uj[UC][CPL];
        Unit<TV> vi[UC][CPL], vj[UC][CPL];
#pragma unroll
        for (int u = 0; u < UC; ++u) {
            t[u] = k0 + base + u * step + rl.gw;
            act[u] = t[u] < k1;
            i[u] = act[u] ? __ldg(p.k_row + t[u]) : 0;
            j[u] = act[u] ? __ldg(p.k_col + t[u]) : 0;
            if constexpr (MODE == CONS_EVAL || std::is_same_v<CS, double>)
                ak[u] = act[u] ? CS(__ldg(p.k_a + t[u])) : CS(0.0);
            else
                ak[u] = act[u] ? (p.k_adf ? ld_scalar<CS>(p.k_a, p.k_adf, t[u]) : CS(__ldg(p.k_a + t[u]))) : CS(0.0);
            kid[u] = act[u] ? __ldg(p.k_id + t[u]) : 0;
            diag[u] = i[u] == j[u];
        }
#pragma unroll
        for (int u = 0; u < UC; ++u) {
            yk[u] = CS(0.0);
            zb[u] = CS(0.0);
            if (!act[u]) continue;
            if constexpr (MODE != CONS_EVAL) {
                if constexpr (MODE != CONS_ZZ) {
                    if constexpr (std::is_same_v<CS, double>) yk[u] = y[kid[u]];
                    else yk[u] = ydf ? ld_scalar<CS>(y, ydf, kid[u]) : CS(y[kid[u]]);
                }
                if (MODE == CONS_LS && zk != nullptr) zb[u] = zkc[kid[u]];
                else if constexpr (std::is_same_v<CS, double>) zb[u] = __ldg(p.b + kid[u]);
                else zb[u] = p.b_df ? ld_scalar<CS>(p.b, p.b_df, kid[u]) : CS(__ldg(p.b + kid[u]));
            }
            load_row<TU, CPL>(ui[u], U, i[u], ld, L, Q, rl.lig);
            if (!diag[u]) load_row<TU, CPL>(uj[u], U, j[u], ld, L, Q, rl.lig);
            if constexpr (NEED_V) {
                if (!(MODE == CONS_EVAL && same)) {
                    load_row<TV, CPL>(vi[u], V, i[u], ld, L, Q, rl.lig);
                    if (!diag[u]) load_row<TV, CPL>(vj[u], V, j[u], ld, L, Q, rl.lig);
                }
            }
        }
#pragma unroll
        for (int u = 0; u < UC; ++u) {
            // dots of the gathered rows; partial per lane, then group sums
            AU s_uu = AU(0);                  // u_i.u_j (EVAL with U==V, and R-only modes)
            AW s_uv = AW(0), s_vu = AW(0);    // u_i.v_j, u_j.v_i
            AV s_vv = AV(0);                  // v_i.v_j
            if (act[u]) {
                if constexpr (MODE == CONS_EVAL) {
                    if (same) {
                        s_uu = diag[u] ? dot_units<AU>(ui[u], ui[u]) : dot_units<AU>(ui[u], uj[u]);
                    } else if (diag[u]) {
                        s_uv = dot_units<AW>(ui[u], vi[u]);
                    } else {
                        s_uv = dot_units<AW>(ui[u], vj[u]);
                        s_vu = dot_units<AW>(uj[u], vi[u]);
                    }
                } else {
                    if (MODE != CONS_LS || zk == nullptr)
                        s_uu = diag[u] ? dot_units<AU>(ui[u], ui[u]) : dot_units<AU>(ui[u], uj[u]);
                    if constexpr (MODE == CONS_LS) {
                        if (diag[u]) {
                            s_uv = dot_units<AW>(ui[u], vi[u]);
                            s_vu = s_uv;
                            s_vv = dot_units<AV>(vi[u], vi[u]);
                        } else {
                            s_uv = dot_units<AW>(ui[u], vj[u]);
                            s_vu = dot_units<AW>(vi[u], uj[u]);
                            s_vv = dot_units<AV>(vi[u], vj[u]);
                        }
                    }
                }
            }
            s_uu = group_sum(s_uu, L);
            if constexpr (MODE == CONS_EVAL || MODE == CONS_LS) {
                s_uv = group_sum(s_uv, L);
                s_vu = group_sum(s_vu, L);
                s_vv = group_sum(s_vv, L);
            }
            if (act[u] && rl.lig == 0) {
                const int k = kid[u];
                if constexpr (MODE == CONS_EVAL) {
                    const double a = double(ak[u]);
                    const double f = diag[u] ? 1.0 : 2.0;
                    double val;
                    if (same) val = f * a * double(s_uu);
                    else if (diag[u]) val = a * double(s_uv);
                    else val = a * (double(s_uv) + double(s_vu));
                    static_cast<double*>(out)[k] = val;
                } else {
                    const CS fa = diag[u] ? ak[u] : CS(2.0f) * ak[u];
                    const CS z = (MODE == CONS_LS && zk != nullptr) ? zb[u] : fa * CS(s_uu) - zb[u];
                    if constexpr (MODE == CONS_LS) {
                        const CS yt = yk[u] - rho_c * z;
                        const CS q1 = fa * (CS(s_uv) + CS(s_vu));
                        const CS q2 = fa * CS(s_vv);
                        accq[PL_YQ1] += PA(yt * q1);
                        accq[PL_YQ2] += PA(yt * q2);
                        accq[PL_Q1Q1] += PA(q1 * q1);
                        accq[PL_Q1Q2] += PA(q1 * q2);
                        accq[PL_Q2Q2] += PA(q2 * q2);
                    } else {
                        accq[PC_ZZ] += PA(z * z);
                        if constexpr (MODE == CONS_YTIL) {
                            static_cast<CS*>(out)[k] = yk[u] - rho_c * z;
                            if (zk != nullptr) zkc[k] = z;
                        } else if constexpr (MODE == CONS_YUPD) {
                            const CS yn = yk[u] - rho_c * z;
                            y[k] = double(yn);
                            if constexpr (std::is_same_v<CS, dfloat>) {
                                if (ydf != nullptr) ydf[k] = yn;
                            } else {
                                if (ydf != nullptr) ydf[k] = dfloat(yn);
                            }
                            // b_k: zb holds it (z is recomputed in this mode)
                            accq[PC_BY] += PA(zb[u] * yn);
                        }
                    }
                }
            }
        }
    }
    if constexpr (MODE != CONS_EVAL) block_partials<NQ>(accq, part, vg.pslot);
}

// ================================================================== direction
// D = cG G + sum_u (cS_u S_u + cY_u Y_u) over the stored pairs (the two-loop
// recursion of Algorithm 1 carried out on coefficients); partials <G,D>, ||D||^2.
// TDIR: storage of D and of the stored pairs (they may be stored narrower than G;
// <G,D> and ||D||^2 are then taken of the stored direction).
template <typename TD, typename TDIR = TD>
__device__ __forceinline__ void
k_dir_body(int64_t nunits, const TD* __restrict__ G, TDIR* __restrict__ D, const TDIR* __restrict__ hist,
      int64_t slot_stride, const Ctrl* ctrl, double* __restrict__ part, VGrid vg) {
    using A = arith_t<TD>;
    using PA = part_t<TD, TD>;
    PA accq[PD_N] = {PA(0), PA(0)};
    const int mem = ctrl->mem_count;
    const A cG = A(ctrl->cG);
    A cS[kMaxMem], cY[kMaxMem];
    const TDIR* Sp[kMaxMem];
    const TDIR* Yp[kMaxMem];
#pragma unroll
    for (int t = 0; t < kMaxMem; ++t) {
        const int s = ctrl->order[t];
        cS[t] = A(ctrl->cS[s]);
        cY[t] = A(ctrl->cY[s]);
        Sp[t] = hist + (int64_t)(2 * s) * slot_stride;
        Yp[t] = hist + (int64_t)(2 * s + 1) * slot_stride;
    }
    const int64_t stride = (int64_t)vg.nblk * blockDim.x;
    for (int64_t u = vg.bid * (int64_t)blockDim.x + threadIdx.x; u < nunits; u += stride) {
        Unit<TD> g, d;
        g.load_stream(G + u * 4);
#pragma unroll
        for (int e = 0; e < 4; ++e) d.v[e] = cG * A(g.v[e]);
#pragma unroll
        for (int t = 0; t < kMaxMem; ++t) {
            if (t < mem) {
                Unit<TDIR> s, y;
                s.load_stream(Sp[t] + u * 4);
                y.load_stream(Yp[t] + u * 4);
#pragma unroll
                for (int e = 0; e < 4; ++e) d.v[e] = fma(cS[t], A(s.v[e]), fma(cY[t], A(y.v[e]), A(d.v[e])));
            }
        }
        Unit<TDIR> dst;
        A gd = A(0), dd = A(0);
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            dst.v[e] = as_stored<TDIR>(A(d.v[e]));
            const A dv = A(dst.v[e]);           // value as stored
            gd += A(g.v[e]) * dv;
            dd += dv * dv;
        }
        dst.store(D + u * 4);
        accq[PD_GD] += gd;
        accq[PD_DD] += dd;
    }
    block_partials<PD_N>(accq, part, vg.pslot);
}

// ================================================================== step (flat)
// R += tau D, CR += tau CD  (used when the gradient needs a separate pattern pass)
template <typename TR, typename TD, typename TDIR = TD>
__device__ __forceinline__ void
k_step_body(int64_t nunits, TR* __restrict__ R, TR* __restrict__ CR, const TDIR* __restrict__ D,
       const TD* __restrict__ CD, const Ctrl* ctrl, VGrid vg) {
    using A = arith_t<TR>;
    const A tau = A(ctrl->tau);
    const int64_t stride = (int64_t)vg.nblk * blockDim.x;
    for (int64_t u = vg.bid * (int64_t)blockDim.x + threadIdx.x; u < nunits; u += stride) {
        Unit<TR> r, cr;
        Unit<TDIR> d;
        Unit<TD> cd;
        r.load_stream(R + u * 4);
        cr.load_stream(CR + u * 4);
        d.load_stream(D + u * 4);
        cd.load_stream(CD + u * 4);
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            r.v[e] = fma(tau, A(d.v[e]), A(r.v[e]));
            cr.v[e] = fma(tau, A(cd.v[e]), A(cr.v[e]));
        }
        r.store_stream(R + u * 4);
        cr.store_stream(CR + u * 4);
    }
}

// ================================================================== row update
// Per row i (group of L lanes):
//   STEP : r += tau d, cr += tau cd                         (Algorithm 1 step)
//   grad : g' = 2 (cr - a_i y~_k r - w_i),  y~_k = y_k - rho (a_i |r|^2 - b_k)
//          for the diagonal constraint k of row i, w = A*_off(y~) R (if given)
//   HIST : s_new = tau d, y_new = g' - g   into the new slot, and the dot
//          products that keep the Gram data of the stored pairs current
//          (<s_new,y_new>, ||y_new||^2, <g',y_new>, and per stored pair v:
//          <s_new,y_v>, <s_v,y_new>, <y_new,y_v>)
// partials: ||g'||^2, sum z_k^2 (diagonal constraints), and the Gram dots.
// 3 resident blocks per SM where the registers allow it without real spills
// (one unit per lane, FP32-unit arithmetic), 2 otherwise.
template <typename TR, typename TD, int CPL>
constexpr int update_min_blocks() {
    return (CPL == 1 && !std::is_same_v<arith_t<TR>, double>) ? 3 : 2;
}

// MAXOLD: most stored pairs besides the new one (T - 1 of Algorithm 1) the pass is
// compiled for; the Gram accumulators of the others are compile-time zeros, which
// frees their registers (T = 2: 8 partial sums instead of 14).
template <typename TR, typename TD, int CPL, bool STEP, bool HIST, typename TDIR = TD, bool DENSE = false,
          int MAXOLD = kMaxMem - 1>
__device__ __forceinline__ void
k_update_body(ProbDev p, TR* __restrict__ R, TR* __restrict__ CR, const TDIR* __restrict__ D,
         const TD* __restrict__ CD, TD* __restrict__ G, const TD* __restrict__ W,
         TDIR* __restrict__ hist, int64_t slot_stride, int ld, int L, int Q,
         const double* __restrict__ y, const dfloat* __restrict__ ydf, void* __restrict__ zrow_v,
         const Ctrl* ctrl, double* __restrict__ part, VGrid vg, int pf = 0) {
    using AR = arith_t<TR>;
    using AD = arith_t<TD>;
    using PA = part_t<TR, TD>;
    using RS = rowscalar_t<TR, TD>;             // per-row scalars (no FP64 off the FP64 path)
    using ZS = zrow_t<TD, TR>;
    ZS* __restrict__ zrow = static_cast<ZS*>(zrow_v);
    const RS rho_r = RS(ctrl->rho);
    PA accq[PU_N];
#pragma unroll
    for (int q = 0; q < PU_N; ++q) accq[q] = PA(0);
    const double taud = ctrl->tau;
    const AR tau = AR(taud);
    const AD tau_d = AD(taud);
    int nold = 0;
    TDIR* Snew = nullptr;                       // pairs stored in the direction's type
    TDIR* Ynew = nullptr;
    static_assert(MAXOLD >= 1 && MAXOLD <= kMaxMem - 1, "stored pairs");
    const TDIR* So[MAXOLD];
    const TDIR* Yo[MAXOLD];
    if constexpr (HIST) {
        nold = ctrl->old_count;
        const int ns = ctrl->new_slot;
        Snew = hist + (int64_t)(2 * ns) * slot_stride;
        Ynew = hist + (int64_t)(2 * ns + 1) * slot_stride;
#pragma unroll
        for (int t = 0; t < MAXOLD; ++t) {
            const int s = ctrl->old_slots[t < nold ? t : 0];
            So[t] = hist + (int64_t)(2 * s) * slot_stride;
            Yo[t] = hist + (int64_t)(2 * s + 1) * slot_stride;
        }
    }
    static_assert(!DENSE || CPL == 1, "packed row groups hold one unit per lane");
    RowLoop rl(L, vg, DENSE);
    for (int64_t base = rl.first; base < p.n; base += rl.stride) {
        const int64_t i = base + rl.gw;
        const bool act = rl.live && i < p.n;
        int knx = -1;                            // constraint of the next row, loaded one iteration ahead
        if (pf != 0) {
            // Prefetch the next row of this group into L2: the several dependent load
            // phases of that iteration (R..C D, the old G, each stored pair) then wait
            // on L2 instead of HBM.
            const int64_t nx = i + rl.stride;
            if (rl.live && nx < p.n) {
                prefetch_row<TR, CPL>(R, nx, ld, L, Q, rl.lig);
                prefetch_row<TR, CPL>(CR, nx, ld, L, Q, rl.lig);
                if constexpr (STEP || HIST) prefetch_row<TDIR, CPL>(D, nx, ld, L, Q, rl.lig);
                if constexpr (STEP) prefetch_row<TD, CPL>(CD, nx, ld, L, Q, rl.lig);
                if (W != nullptr) prefetch_row<TD, CPL>(W, nx, ld, L, Q, rl.lig);
                if constexpr (HIST) {
                    prefetch_row<TD, CPL>(G, nx, ld, L, Q, rl.lig);
#pragma unroll
                    for (int t = 0; t < MAXOLD; ++t)
                        if (t < nold) {
                            prefetch_row<TDIR, CPL>(So[t], nx, ld, L, Q, rl.lig);
                            prefetch_row<TDIR, CPL>(Yo[t], nx, ld, L, Q, rl.lig);
                        }
                }
                if (p.dk != nullptr && rl.lig == 0) {
                    knx = __ldg(p.dk + nx);
                    if constexpr (std::is_same_v<RS, double>) prefetch_l2(p.da + nx);
                    else prefetch_l2(p.da_df + nx);
                }
            }
        }
        Unit<TR> r[CPL], cr[CPL];
        Unit<TDIR> d[CPL];
        AR rr = AR(0);
        if (act) {
            load_row_stream<TR, CPL>(r, R, i, ld, L, Q, rl.lig);
            load_row_stream<TR, CPL>(cr, CR, i, ld, L, Q, rl.lig);
            if constexpr (STEP || HIST) load_row_stream<TDIR, CPL>(d, D, i, ld, L, Q, rl.lig);
            if constexpr (STEP) {
                Unit<TD> cd[CPL];
                load_row_stream<TD, CPL>(cd, CD, i, ld, L, Q, rl.lig);
#pragma unroll
                for (int c = 0; c < CPL; ++c)
#pragma unroll
                    for (int e = 0; e < 4; ++e) {
                        r[c].v[e] = step_add<AR, AD>(AR(r[c].v[e]), tau, tau_d, AD(d[c].v[e]));
                        cr[c].v[e] = step_add<AR, AD>(AR(cr[c].v[e]), tau, tau_d, AD(cd[c].v[e]));
                    }
                store_row<TR, CPL>(r, R, i, ld, L, Q, rl.lig);
                store_row<TR, CPL>(cr, CR, i, ld, L, Q, rl.lig);
            }
#pragma unroll
            for (int c = 0; c < CPL; ++c)
#pragma unroll
                for (int e = 0; e < 4; ++e) rr = sq_add<AR>(rr, AR(r[c].v[e]));
        }
        // diagonal-constraint coefficient a_i y~_k of row i
        AR coef = AR(0);
        if (p.dk != nullptr) {
            if constexpr (DENSE) rr = group_sum_packed(rr, L, rl.base_lane);
            else rr = group_sum(rr, L);
            if (act) {
                const int k = __ldg(p.dk + i);
                if (k >= 0) {
                    const RS a = ld_scalar<RS>(p.da, p.da_df, i);
                    const RS z = a * RS(rr) - ld_scalar<RS>(p.b, p.b_df, k);
                    const RS yv = ydf ? ld_scalar<RS>(y, ydf, k) : RS(__ldg(y + k));
                    coef = AR(a * (yv - rho_r * z));
                    if (rl.lig == 0) {
                        accq[PU_ZZ] += PA(z * z);
                        if (zrow != nullptr) zrow[i] = ZS(z);
                    }
                }
            }
        }
        if (act) {
            Unit<TD> g[CPL];
            Unit<TD> w[CPL];
            if (W != nullptr) load_row_stream<TD, CPL>(w, W, i, ld, L, Q, rl.lig);
#pragma unroll
            for (int c = 0; c < CPL; ++c)
#pragma unroll
                for (int e = 0; e < 4; ++e) {
                    if (W != nullptr) {
                        const AR gv = AR(cr[c].v[e]) - coef * AR(r[c].v[e]) - AR(w[c].v[e]);
                        g[c].v[e] = AD(AR(2) * gv);
                    } else {
                        g[c].v[e] = grad_elem<AR, AD>(AR(cr[c].v[e]), coef, AR(r[c].v[e]));
                    }
                }
            if constexpr (HIST) {
                // the new pair as stored (rounded to TDIR): the Gram dots below are those
                // of the stored vectors, which the direction pass reads
                Unit<TD> gold[CPL];
                Unit<TDIR> sn[CPL], yn[CPL];
                load_row_stream<TD, CPL>(gold, G, i, ld, L, Q, rl.lig);
#pragma unroll
                for (int c = 0; c < CPL; ++c)
#pragma unroll
                    for (int e = 0; e < 4; ++e) {
                        sn[c].v[e] = as_stored<TDIR>(tau_d * AD(d[c].v[e]));
                        yn[c].v[e] = as_stored<TDIR>(AD(g[c].v[e]) - AD(gold[c].v[e]));
                    }
                store_row<TDIR, CPL>(sn, Snew, i, ld, L, Q, rl.lig);
                store_row<TDIR, CPL>(yn, Ynew, i, ld, L, Q, rl.lig);
                accq[PU_GYN] += dot_units<AD>(g, yn);
                accq[PU_SYN] += dot_units<AD>(sn, yn);
                accq[PU_YYN] += dot_units<AD>(yn, yn);
#pragma unroll
                for (int t = 0; t < MAXOLD; ++t) {
                    if (t < nold) {
                        Unit<TDIR> so[CPL], yo[CPL];
                        load_row_stream<TDIR, CPL>(so, So[t], i, ld, L, Q, rl.lig);
                        load_row_stream<TDIR, CPL>(yo, Yo[t], i, ld, L, Q, rl.lig);
                        PA* q = accq + PU_FIXED + PU_PER_OLD * t;
                        q[0] += dot_units<AD>(sn, yo);
                        q[1] += dot_units<AD>(so, yn);
                        q[2] += dot_units<AD>(yn, yo);
                    }
                }
            }
            store_row<TD, CPL>(g, G, i, ld, L, Q, rl.lig);
            accq[PU_GG] += dot_units<AD>(g, g);
        }
        if (knx >= 0) {
            // the next row's multiplier and right-hand side
            if constexpr (std::is_same_v<RS, double>) {
                prefetch_l2(y + knx);
                prefetch_l2(p.b + knx);
            } else {
                prefetch_l2(ydf ? static_cast<const void*>(ydf + knx) : static_cast<const void*>(y + knx));
                prefetch_l2(p.b_df + knx);
            }
        }
    }
    block_partials<PU_N>(accq, part, vg.pslot);
}

// ================================================================== kernels
// One launch per body over the hardware grid; a kernel of the captured
// iteration graph first checks the phase flags of the control block.

// Resident blocks per SM the SpMM over C is compiled for: for float rows 4 (64
// registers, no spills) with one unit per lane and 3 (85 registers) with more,
// for bf16 rows 3 (their conversions take more registers), where the pass is
// bound by the latency of its dependent loads; otherwise left to the compiler.
template <typename TX, typename TO, int CPL>
constexpr int spmm_min_blocks() {
    if constexpr (std::is_same_v<TX, float> && std::is_same_v<TO, float>) return CPL == 1 ? 4 : 3;
    else if constexpr (std::is_same_v<TX, __nv_bfloat16> && std::is_same_v<TO, float>) return 3;
    else return 1;
}

template <typename TX, typename TO, typename TR, int CPL, int EPI, bool DENSE = false, int PF = 0>
__global__ void __launch_bounds__(kThreads, (spmm_min_blocks<TX, TO, CPL>()))
k_spmm_c(ProbDev p, const TX* __restrict__ X, TO* __restrict__ out, int ld, int L, int Q,
         const double* __restrict__ v, int write_out,
         const TR* __restrict__ R, const double* __restrict__ y, const void* __restrict__ zrow_v,
         const dfloat* __restrict__ ydf, const Ctrl* ctrl, double rho_arg, double* __restrict__ part,
         const Ctrl* gate, int ph) {
    if (gated_off(gate, ph)) return;
    k_spmm_c_body<TX, TO, TR, CPL, EPI, DENSE, PF>(p, X, out, ld, L, Q, v, write_out, R, y, zrow_v, ydf, ctrl, rho_arg,
                                                   part, hw_grid());
}

template <typename TX, typename TO, int CPL, bool VDF>
__global__ void __launch_bounds__(kThreads)
k_spmm_a(ProbDev p, const TX* __restrict__ X, TO* __restrict__ out, int ld, int L, int Q,
         const void* __restrict__ v, double alpha, int accumulate, const Ctrl* gate, int ph) {
    if (gated_off(gate, ph)) return;
    k_spmm_a_body<TX, TO, CPL, VDF>(p, X, out, ld, L, Q, v, alpha, accumulate, hw_grid());
}

template <typename TU, typename TV, int CPL, int MODE>
__global__ void __launch_bounds__(kThreads, 2)
k_cons(ProbDev p, int64_t k0, int64_t k1, const TU* __restrict__ U, const TV* __restrict__ V, int ld, int L, int Q,
       double* y, void* __restrict__ out, void* zk, dfloat* ydf, const Ctrl* ctrl, double rho_arg,
       double* __restrict__ part, const Ctrl* gate, int ph) {
    if (gated_off(gate, ph)) return;
    k_cons_body<TU, TV, CPL, MODE>(p, k0, k1, U, V, ld, L, Q, y, out, zk, ydf, ctrl, rho_arg, part, hw_grid());
}

template <typename TD, typename TDIR = TD>
__global__ void __launch_bounds__(kThreads)
k_dir(int64_t nunits, const TD* __restrict__ G, TDIR* __restrict__ D, const TDIR* __restrict__ hist,
      int64_t slot_stride, const Ctrl* ctrl, double* __restrict__ part, const Ctrl* gate, int ph) {
    if (gated_off(gate, ph)) return;
    k_dir_body<TD, TDIR>(nunits, G, D, hist, slot_stride, ctrl, part, hw_grid());
}

template <typename TR, typename TD, typename TDIR = TD>
__global__ void __launch_bounds__(kThreads)
k_step(int64_t nunits, TR* __restrict__ R, TR* __restrict__ CR, const TDIR* __restrict__ D,
       const TD* __restrict__ CD, const Ctrl* ctrl, const Ctrl* gate, int ph) {
    if (gated_off(gate, ph)) return;
    k_step_body<TR, TD, TDIR>(nunits, R, CR, D, CD, ctrl, hw_grid());
}

template <typename TR, typename TD, int CPL, bool STEP, bool HIST, typename TDIR = TD>
__global__ void __launch_bounds__(kThreads, (update_min_blocks<TR, TD, CPL>()))
k_update(ProbDev p, TR* __restrict__ R, TR* __restrict__ CR, const TDIR* __restrict__ D,
         const TD* __restrict__ CD, TD* __restrict__ G, const TD* __restrict__ W,
         TDIR* __restrict__ hist, int64_t slot_stride, int ld, int L, int Q,
         const double* __restrict__ y, const dfloat* __restrict__ ydf, void* __restrict__ zrow_v,
         const Ctrl* ctrl, double* __restrict__ part, const Ctrl* gate, int ph) {
    if (gated_off(gate, ph)) return;
    k_update_body<TR, TD, CPL, STEP, HIST, TDIR>(p, R, CR, D, CD, G, W, hist, slot_stride, ld, L, Q, y, ydf, zrow_v, ctrl, part, hw_grid());
}

// The step update with EXTRA more resident blocks per SM (fewer registers per
// thread, some spilled to L1): more rows in flight for the latency-bound pass.
// DENSE: packed row groups of L = Q lanes (RowLoop).  MAXOLD: see k_update_body.
template <typename TR, typename TD, int CPL, int EXTRA, typename TDIR = TD, bool DENSE = false,
          int MAXOLD = kMaxMem - 1>
__global__ void __launch_bounds__(kThreads, (update_min_blocks<TR, TD, CPL>() + EXTRA))
k_update_step_occ(ProbDev p, TR* __restrict__ R, TR* __restrict__ CR, const TDIR* __restrict__ D,
                  const TD* __restrict__ CD, TD* __restrict__ G, const TD* __restrict__ W,
                  TDIR* __restrict__ hist, int64_t slot_stride, int ld, int L, int Q,
                  const double* __restrict__ y, const dfloat* __restrict__ ydf, void* __restrict__ zrow_v,
                  const Ctrl* ctrl, double* __restrict__ part, const Ctrl* gate, int ph, int pf) {
    if (gated_off(gate, ph)) return;
    k_update_body<TR, TD, CPL, true, true, TDIR, DENSE, MAXOLD>(p, R, CR, D, CD, G, W, hist, slot_stride, ld, L, Q, y,
                                                                 ydf, zrow_v, ctrl, part, hw_grid(), pf);
}

}  // namespace lorads
