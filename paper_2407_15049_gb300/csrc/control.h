// Host launchers of the single-block control kernels (control.cu).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>
#include "common.cuh"

namespace lorads {

enum { HIST_STEP = 0, HIST_RESET = 1 };

void ctrl_root(cudaStream_t s, Ctrl* c, const double* part_dir, int nb_dir, const double* part_ls, int nb_ls,
               const double* part_cons, int nb_cons);
void ls_finish(cudaStream_t s, const double* part_ls, int nb_ls, const double* part_cons, int nb_cons,
               double rho, double* out);
void ctrl_hist(cudaStream_t s, Ctrl* c, int mode, const double* part_upd, int nb_upd, const double* part_ytil,
               int nb_ytil);
void ctrl_outer(cudaStream_t s, Ctrl* c, const double* part_cons, int nb_cons, const double* part_obj, int nb_obj);
void ctrl_init(cudaStream_t s, Ctrl* c, const double* part_cons, int nb_cons, const double* part_obj, int nb_obj);
void ctrl_resume(cudaStream_t s, Ctrl* c);
void quartic_step_dev(cudaStream_t s, const double* a, double* tau);
void fold_to(cudaStream_t s, const double* part, int nb, int NQ, double* out);

void lz_random(cudaStream_t s, int64_t n, uint64_t seed, double* v, double* part, int blocks);
void lz_scalar(cudaStream_t s, const double* part, int nb, double* lz, int slot, int mode);
void lz_scale(cudaStream_t s, int64_t n, double* v, const double* lz, int slot, int blocks);
void lz_dot(cudaStream_t s, int64_t n, const double* w, const double* v, double* part, int blocks);
void lz_orth(cudaStream_t s, int64_t n, double* w, const double* v, const double* vp, const double* lz, int a_slot,
             int b_slot, double* part, int blocks);
void lz_tridiag_min(cudaStream_t s, const double* lz, int k, int beta_off, double* out);

template <typename T> void sumsq(cudaStream_t s, int64_t n, int ld, int r, const void* X, double* part, int blocks);
template <typename T>
void rank_columns(cudaStream_t s, int64_t n, int ld, int r_old, int r_new, double scale, uint64_t seed,
                  uint64_t stream, void* X, int blocks);
template <typename T>
void random_start(cudaStream_t s, int64_t n, int ld, int r, uint64_t seed, int unit_rows, double scale, void* X,
                  int blocks);
void scale_c(cudaStream_t s, int64_t nnz, const double* c0, double scale, double* c, float* c32, dfloat* cdf,
             int blocks);
void rescale_y(cudaStream_t s, int64_t m, double* y, dfloat* ydf, double s_old, double s_new, int blocks);
template <typename TI, typename TO>
void convert(cudaStream_t s, int64_t n, int ld_in, int ld_out, int r, const void* in, void* out, int blocks);

}  // namespace lorads
