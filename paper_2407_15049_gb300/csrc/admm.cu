// Launchers, control kernels and instantiations of the splitting (ADMM)
// stage of Sec. 2.2 (kernels in admm.cuh).
//
// Control (one block, FP64, partial sums folded in a fixed order):
//   cg_init : ||r_0||, the stop threshold eps = cg_rel ||r_0|| of Algorithm 2;
//   alpha   : alpha = <r,r> / <p, frakA_V(p)> with <p, frakA_V(p)> = rho (||p||^2 + ||A(p V^T)||^2);
//   beta    : ||r_new||, stop test, beta = <r_new,r_new> / <r,r>;
//   outer   : after y <- y - rho (A(U V^T) - b) and R = (U + V)/2: err1 and err3
//             of Sec. 4.2 at R, the stop test, the iteration cap.
// The CG kernels of a block step return at once once `cg_active` is cleared,
// so a captured graph can hold cg_max steps of which only the needed ones work.
#include <math.h>
#include "admm.cuh"
#include "admm.h"

namespace lorads {

namespace {

__device__ void fold_sum(const double* part, int nb, int NQ, double* out) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (int q = warp; q < NQ; q += nw) {
        double s = 0.0;
        for (int b = lane; b < nb; b += 32) s += part[(size_t)b * NQ + q];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
        if (lane == 0) out[q] = s;
    }
}

__global__ void k_admm_cg_init(AdmmCtrl* ac, const double* part_r, int nb) {
    __shared__ double s[PA_N];
    fold_sum(part_r, nb, PA_N, s);
    __syncthreads();
    if (threadIdx.x == 0) admm_cg_init_apply(ac, s[PA_RR]);
}

__global__ void k_admm_alpha(AdmmCtrl* ac, const double* part_q, int nb, const double* part_w, int nb_w) {
    if (!ac->cg_active) return;
    __shared__ double s[PQ_N + 1];
    fold_sum(part_q, nb, PQ_N, s);
    if (part_w != nullptr) fold_sum(part_w, nb_w, 1, s + PQ_N);
    else if (threadIdx.x == 0) s[PQ_N] = 0.0;
    __syncthreads();
    if (threadIdx.x == 0) admm_alpha_apply(ac, s[PQ_PP], s[PQ_WW] + s[PQ_N]);
}

__global__ void k_admm_beta(AdmmCtrl* ac, const double* part_r, int nb) {
    if (!ac->cg_active) return;
    __shared__ double s[PA_N];
    fold_sum(part_r, nb, PA_N, s);
    __syncthreads();
    if (threadIdx.x == 0) admm_beta_apply(ac, s[PA_RR]);
}

__global__ void k_admm_outer(AdmmCtrl* ac, const double* part_y, int nb_y, const double* part_zz, int nb_zz,
                             const double* part_obj, int nb_obj) {
    __shared__ double sy[PY_N], sz[PC_N], so[PO_N];
    fold_sum(part_y, nb_y, PY_N, sy);
    fold_sum(part_zz, nb_zz, PC_N, sz);
    fold_sum(part_obj, nb_obj, PO_N, so);
    __syncthreads();
    if (threadIdx.x == 0) admm_outer_apply(ac, sz[PC_ZZ], sy[PY_BY], so[PO_CRR]);
}

}  // namespace

#define ADMM_CPL_SWITCH(cpl, ...)                                     \
    switch (cpl) {                                                      \
        case 1: { constexpr int CPL = 1; __VA_ARGS__; } break;         \
        case 2: { constexpr int CPL = 2; __VA_ARGS__; } break;         \
        case 3: { constexpr int CPL = 3; __VA_ARGS__; } break;         \
        case 4: { constexpr int CPL = 4; __VA_ARGS__; } break;         \
        default: break;                                                 \
    }

template <typename TR>
void admm_omega(const AdmmRows& a, const void* X, const void* V, double* y, dfloat* ydf, void* om,
                const AdmmCtrl* ac) {
    ADMM_CPL_SWITCH(a.sh.CPL, {
        k_admm_cons<TR, CPL, 0><<<a.nb_cons, kThreads, 0, a.stream>>>(
            *a.p, static_cast<const TR*>(X), static_cast<const TR*>(V), a.ld, a.sh.L, a.sh.Q, y, ydf, om, ac,
            nullptr);
    })
}

template <typename TR>
void admm_yupd(const AdmmRows& a, const void* U, const void* V, double* y, dfloat* ydf, const AdmmCtrl* ac,
               double* part) {
    ADMM_CPL_SWITCH(a.sh.CPL, {
        k_admm_cons<TR, CPL, 1><<<a.nb_cons, kThreads, 0, a.stream>>>(
            *a.p, static_cast<const TR*>(U), static_cast<const TR*>(V), a.ld, a.sh.L, a.sh.Q, y, ydf, nullptr, ac,
            part);
    })
}

template <typename TR, typename TW>
void admm_resid(const AdmmRows& a, const void* X, const void* V, const void* om, void* r, void* pd,
                const AdmmCtrl* ac, double* part) {
    ADMM_CPL_SWITCH(a.sh.CPL, {
        k_admm_resid<TR, TW, CPL><<<a.nb_rows, kThreads, 0, a.stream>>>(
            *a.p, static_cast<const TR*>(X), static_cast<const TR*>(V), a.ld, a.sh.L, a.sh.Q, om,
            static_cast<TW*>(r), static_cast<TW*>(pd), ac, part);
    })
}

template <typename TR, typename TW>
void admm_op(const AdmmRows& a, const void* V, const void* r, void* pd, void* Q, const AdmmCtrl* ac,
             double rho_arg, int update_p, double* part, void* w, double* part_w) {
    // general form: the row pass covers p's update, rho p and the fused diagonal
    // constraints; the listed constraints follow in two passes (w, then A*(w) V)
    const bool general = a.p->k_ptr != nullptr;
    const bool fuse = update_p && (a.p->m_off == 0 || general);
    if (update_p && !fuse) {
        const int64_t nunits = a.p->n * (int64_t)a.ld / 4;
        k_admm_pupd<TW><<<a.nb_flat, kThreads, 0, a.stream>>>(nunits, static_cast<const TW*>(r),
                                                                static_cast<TW*>(pd), ac);
    }
    ADMM_CPL_SWITCH(a.sh.CPL, {
        if (fuse)
            k_admm_op<TR, TW, CPL, true><<<a.nb_rows, kThreads, 0, a.stream>>>(
                *a.p, static_cast<const TR*>(V), a.ld, a.sh.L, a.sh.Q, static_cast<const TW*>(r),
                static_cast<TW*>(pd), static_cast<TW*>(Q), ac, rho_arg, part);
        else
            k_admm_op<TR, TW, CPL, false><<<a.nb_rows, kThreads, 0, a.stream>>>(
                *a.p, static_cast<const TR*>(V), a.ld, a.sh.L, a.sh.Q, static_cast<const TW*>(r),
                static_cast<TW*>(pd), static_cast<TW*>(Q), ac, rho_arg, part);
        if (general && a.p->m_off > 0 && ac != nullptr) {
            k_admm_opw<TR, TW, CPL><<<a.nb_cons, kThreads, 0, a.stream>>>(
                *a.p, static_cast<const TR*>(V), a.ld, a.sh.L, a.sh.Q, static_cast<const TW*>(pd), w, ac, part_w);
            k_admm_opq<TR, TW, CPL><<<a.nb_rows, kThreads, 0, a.stream>>>(
                *a.p, static_cast<const TR*>(V), a.ld, a.sh.L, a.sh.Q, w, static_cast<TW*>(Q), ac);
        }
    })
}

template <typename TR, typename TW>
void admm_upd(const AdmmRows& a, void* X, const void* pd, void* r, const void* Q, const AdmmCtrl* ac,
              double* part) {
    const int64_t nunits = a.p->n * (int64_t)a.ld / 4;
    k_admm_upd<TR, TW><<<a.nb_flat, kThreads, 0, a.stream>>>(nunits, static_cast<TR*>(X),
                                                              static_cast<const TW*>(pd), static_cast<TW*>(r),
                                                              static_cast<const TW*>(Q), ac, part);
}

template <typename TR>
void admm_avg(const AdmmRows& a, const void* U, const void* V, void* R) {
    const int64_t nunits = a.p->n * (int64_t)a.ld / 4;
    k_admm_avg<TR><<<a.nb_flat, kThreads, 0, a.stream>>>(nunits, static_cast<const TR*>(U),
                                                          static_cast<const TR*>(V), static_cast<TR*>(R));
}

void admm_cg_init(cudaStream_t s, AdmmCtrl* ac, const double* part_r, int nb) {
    k_admm_cg_init<<<1, 256, 0, s>>>(ac, part_r, nb);
}
void admm_alpha(cudaStream_t s, AdmmCtrl* ac, const double* part_q, int nb, const double* part_w, int nb_w) {
    k_admm_alpha<<<1, 256, 0, s>>>(ac, part_q, nb, part_w, nb_w);
}
void admm_beta(cudaStream_t s, AdmmCtrl* ac, const double* part_r, int nb) {
    k_admm_beta<<<1, 256, 0, s>>>(ac, part_r, nb);
}
void admm_outer(cudaStream_t s, AdmmCtrl* ac, const double* part_y, int nb_y, const double* part_zz, int nb_zz,
                const double* part_obj, int nb_obj) {
    k_admm_outer<<<1, 256, 0, s>>>(ac, part_y, nb_y, part_zz, nb_zz, part_obj, nb_obj);
}

// (TR, TW): FP64 (double, double), mixed (dfloat, float), double-float (dfloat, dfloat),
// FP32 (float, float)
#define ADMM_INSTANTIATE_R(TR)                                                                              \
    template void admm_omega<TR>(const AdmmRows&, const void*, const void*, double*, dfloat*, void*,        \
                                 const AdmmCtrl*);                                                           \
    template void admm_yupd<TR>(const AdmmRows&, const void*, const void*, double*, dfloat*, const AdmmCtrl*, \
                                double*);                                                                    \
    template void admm_avg<TR>(const AdmmRows&, const void*, const void*, void*);
#define ADMM_INSTANTIATE_RW(TR, TW)                                                                         \
    template void admm_resid<TR, TW>(const AdmmRows&, const void*, const void*, const void*, void*, void*,  \
                                     const AdmmCtrl*, double*);                                              \
    template void admm_op<TR, TW>(const AdmmRows&, const void*, const void*, void*, void*, const AdmmCtrl*,  \
                                  double, int, double*, void*, double*);                                     \
    template void admm_upd<TR, TW>(const AdmmRows&, void*, const void*, void*, const void*, const AdmmCtrl*, \
                                   double*);

ADMM_INSTANTIATE_R(double)
ADMM_INSTANTIATE_R(dfloat)
ADMM_INSTANTIATE_R(float)
ADMM_INSTANTIATE_RW(double, double)
ADMM_INSTANTIATE_RW(dfloat, float)
ADMM_INSTANTIATE_RW(dfloat, dfloat)
ADMM_INSTANTIATE_RW(float, float)

}  // namespace lorads
