// Host launchers of the splitting (ADMM) stage kernels (admm.cuh, admm.cu).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>
#include "common.cuh"

namespace lorads {

struct ProbDev;

// Device control block of the stage (one per context).
struct AdmmCtrl {
    double rho, cg_rel, tol, bnorm_inf;
    double rr, eps, alpha, beta;          // CG state of the current block step
    double err1, err3, primal_obj, dual_obj;
    int cg_max, cg_k, cg_active, cg_total;
    int iters, max_iter, done, status;
};

// Row-pass launch data shared by the stage's kernels.
struct AdmmRows {
    const ProbDev* p;
    int ld; Shape sh;
    int nb_rows;        // blocks of the row passes (groups of L lanes per row)
    int nb_cons;        // blocks of the constraint passes (groups of L lanes per constraint)
    int nb_flat;        // blocks of the flat passes (one thread per 4 elements)
    cudaStream_t stream;
};

// TR: storage of U, V (double, dfloat, float); TW: storage of r, p, Q.
// w = y - rho (A(X V^T) - b) into om (double on the all-FP64 path, dfloat otherwise)
template <typename TR> void admm_omega(const AdmmRows& a, const void* X, const void* V, double* y, dfloat* ydf,
                                       void* om, const AdmmCtrl* ac);
// y <- y - rho (A(U V^T) - b); partials (PY_*) into part
template <typename TR> void admm_yupd(const AdmmRows& a, const void* U, const void* V, double* y, dfloat* ydf,
                                      const AdmmCtrl* ac, double* part);
// r = p = -(C - A*(w)) V + rho (V - X); partial ||r||^2
template <typename TR, typename TW> void admm_resid(const AdmmRows& a, const void* X, const void* V,
                                                    const void* om, void* r, void* pd, const AdmmCtrl* ac,
                                                    double* part);
// one CG operator application (p update first when update_p), Q = frakA_V(p); partials PQ_*;
// general form (constraints with several triplets): w (m-vector, scratch) and part_w
// (its sum of squares) for the listed constraints
template <typename TR, typename TW> void admm_op(const AdmmRows& a, const void* V, const void* r, void* pd, void* Q,
                                                 const AdmmCtrl* ac, double rho_arg, int update_p, double* part,
                                                 void* w, double* part_w);
// X += alpha p, r -= alpha Q; partial ||r||^2
template <typename TR, typename TW> void admm_upd(const AdmmRows& a, void* X, const void* pd, void* r, const void* Q,
                                                  const AdmmCtrl* ac, double* part);
// R = (U + V) / 2
template <typename TR> void admm_avg(const AdmmRows& a, const void* U, const void* V, void* R);

// single-block control kernels (FP64)
void admm_cg_init(cudaStream_t s, AdmmCtrl* ac, const double* part_r, int nb);
void admm_alpha(cudaStream_t s, AdmmCtrl* ac, const double* part_q, int nb, const double* part_w, int nb_w);
void admm_beta(cudaStream_t s, AdmmCtrl* ac, const double* part_r, int nb);
void admm_outer(cudaStream_t s, AdmmCtrl* ac, const double* part_y, int nb_y, const double* part_zz, int nb_zz,
                const double* part_obj, int nb_obj);

}  // namespace lorads
