// Single-block control kernels of the device-resident solve loop and the
// scalar pieces of the method: the line-search coefficients and cubic root of
// App. A.2, the L-BFGS two-loop recursion of Algorithm 1 carried out on the
// Gram data of the stored pairs, the multiplier/penalty step of Sec. 2.1 and
// the error measures of Sec. 4.2.  All in FP64 on one block; the partial sums
// of the streaming kernels are folded in a fixed order (deterministic).
#include <math.h>
#include "control.h"
#include "kernels.cuh"
#include "control_dev.cuh"

namespace lorads {

// ---------------------------------------------------------------- reductions
// out[q] = sum over blocks of part[b*NQ + q]; warp w folds q = w, w+8, ...
__device__ void fold_parts(const double* part, int nb, int NQ, double* out) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (int q = warp; q < NQ; q += nw) {
        double s = 0.0;
        for (int b = lane; b < nb; b += 32) s += part[(size_t)b * NQ + q];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
        if (lane == 0) out[q] = s;
    }
}

__global__ void k_quartic_step(const double* a, double* tau) { *tau = quartic_step(a); }

// ---------------------------------------------------------------- root kernel
// Folds the line-search partials of the iteration, forms a1..a4 and tau.
// a4 = <G, D> (the directional derivative; equal to p1 - y~^T q1 of App. A.2).
__global__ void k_ctrl_root(Ctrl* c, const double* part_dir, int nb_dir, const double* part_ls, int nb_ls,
                            const double* part_cons, int nb_cons) {
    if (gated_off(c, PH_INNER)) return;
    __shared__ double sd[PD_N], sl[PL_N], sc[PL_N];
    fold_parts(part_dir, nb_dir, PD_N, sd);
    fold_parts(part_ls, nb_ls, PL_N, sl);
    if (part_cons != nullptr) fold_parts(part_cons, nb_cons, PL_N, sc);
    else if (threadIdx.x < PL_N) sc[threadIdx.x] = 0.0;
    __syncthreads();
    if (threadIdx.x != 0) return;
    ctrl_root_apply(c, sd, sl, sc);
}

// Standalone variant for lorads_linesearch_coeffs: paper's a4 = p1 - y~^T q1.
__global__ void k_ls_finish(const double* part_ls, int nb_ls, const double* part_cons, int nb_cons,
                            double rho, double* out /* a[4], tau */) {
    __shared__ double sl[PL_N], sc[PL_N];
    fold_parts(part_ls, nb_ls, PL_N, sl);
    if (part_cons != nullptr) fold_parts(part_cons, nb_cons, PL_N, sc);
    else if (threadIdx.x < PL_N) sc[threadIdx.x] = 0.0;
    __syncthreads();
    if (threadIdx.x != 0) return;
    const double yq1 = sl[PL_YQ1] + sc[PL_YQ1];
    const double yq2 = sl[PL_YQ2] + sc[PL_YQ2];
    const double q1q1 = sl[PL_Q1Q1] + sc[PL_Q1Q1];
    const double q1q2 = sl[PL_Q1Q2] + sc[PL_Q1Q2];
    const double q2q2 = sl[PL_Q2Q2] + sc[PL_Q2Q2];
    out[0] = 0.5 * rho * q2q2;
    out[1] = rho * q1q2;
    out[2] = sl[PL_P2] - yq2 + 0.5 * rho * q1q1;
    out[3] = sl[PL_P1] - yq1;
    out[4] = quartic_step(out);
}

// ---------------------------------------------------------------- history kernel
// mode HIST_STEP: after a step, store the new pair (s = tau D, y = G' - G) if
// its curvature <y,s> is positive enough, else clear the memory; then test the
// inner stop and prepare the next direction.
// mode HIST_RESET: start of an inner loop (memory empty).
__global__ void k_ctrl_hist(Ctrl* c, int mode, const double* part_upd, int nb_upd,
                            const double* part_ytil, int nb_ytil) {
    const bool reset = (mode == HIST_RESET);
    if (gated_off(c, reset ? PH_OUTER : PH_INNER)) return;
    const bool fresh = reset || c->step_ok;
    __shared__ double su[PU_N], sy[PC_N];
    if (fresh) {
        fold_parts(part_upd, nb_upd, PU_N, su);
        if (part_ytil != nullptr) fold_parts(part_ytil, nb_ytil, PC_N, sy);
        else if (threadIdx.x < PC_N) sy[threadIdx.x] = 0.0;
    }
    __syncthreads();
    if (threadIdx.x != 0) return;
    ctrl_hist_apply(c, reset, fresh, su, sy);
}

// ---------------------------------------------------------------- outer kernel
// Multiplier step of Sec. 2.1 has been applied by the constraint pass (y <- y~);
// here: err1 = ||A(RR^T) - b|| / (1 + ||b||_inf), err3 of Sec. 4.2, stop test,
// penalty growth when err1 did not shrink enough, and the rank-update request
// of App. A.1 when the inner loop hit its cap in consecutive outer steps.
__global__ void k_ctrl_outer(Ctrl* c, const double* part_cons, int nb_cons, const double* part_obj, int nb_obj) {
    if (gated_off(c, PH_OUTER)) return;
    __shared__ double sc[PC_N], so[PO_N];
    fold_parts(part_cons, nb_cons, PC_N, sc);
    fold_parts(part_obj, nb_obj, PO_N, so);
    __syncthreads();
    if (threadIdx.x != 0) return;
    ctrl_outer_apply(c, sc, so);
}

// Start of a solve: err1 at R0 and the outer phase for the first gradient.
__global__ void k_ctrl_init(Ctrl* c, const double* part_cons, int nb_cons, const double* part_obj, int nb_obj) {
    __shared__ double sc[PC_N], so[PO_N];
    fold_parts(part_cons, nb_cons, PC_N, sc);
    fold_parts(part_obj, nb_obj, PO_N, so);
    __syncthreads();
    if (threadIdx.x != 0) return;
    ctrl_init_apply(c, sc, so);
}

// Resume after the host handled a pause (rank update): run the outer tail.
__global__ void k_ctrl_resume(Ctrl* c) {
    c->pause = 0;
    c->phase = PHASE_OUTER;
}

// ---------------------------------------------------------------- misc kernels
__global__ void k_fold_to(const double* part, int nb, int NQ, double* out) {
    __shared__ double s[32];
    fold_parts(part, nb, NQ, s);
    __syncthreads();
    if (threadIdx.x < NQ) out[threadIdx.x] = s[threadIdx.x];
}

template <typename T>
__global__ void k_sumsq(int64_t n, int ld, int r, const T* X, double* part) {
    double acc[1] = {0.0};
    const int64_t total = n * (int64_t)r;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = e / r;
        const int c = (int)(e - i * r);
        const double v = double(X[i * ld + c]);
        acc[0] += v * v;
    }
    block_partials<1>(acc, part);
}

// Columns r_old..r_new-1 of X get scale * N(0,1): entry (i, c) uses outputs
// 2e and 2e+1 (e = i*k + c - r_old, k = r_new - r_old) of the SplitMix64
// sequence started at seed ^ (stream * golden), Box-Muller on (u1, u2).
template <typename T>
__global__ void k_rank_columns(int64_t n, int ld, int r_old, int r_new, double scale, uint64_t seed,
                               uint64_t stream, T* X) {
    const uint64_t golden = 0x9E3779B97F4A7C15ull;
    const uint64_t base = seed ^ (stream * golden);
    const int k = r_new - r_old;
    const int64_t total = n * (int64_t)k;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = e / k;
        const int c = (int)(e - i * k);
        X[i * ld + r_old + c] = T(scale * normal_at(base, e));
    }
}

// Row i of X gets rows of N(0,1) draws (same generator, stream = ~0), scaled
// to unit norm when unit_rows (diagonal constraints) or by `scale` otherwise.
template <typename T>
__global__ void k_random_start(int64_t n, int ld, int r, uint64_t seed, int unit_rows, double scale, T* X) {
    const uint64_t golden = 0x9E3779B97F4A7C15ull;
    const uint64_t base = seed ^ (~0ull * golden);
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        double nrm = 0.0;
        for (int pass = 0; pass < 2; ++pass) {
            for (int c = 0; c < r; ++c) {
                const int64_t e = i * r + c;
                const double g = normal_at(base, e);
                if (pass == 0) nrm += g * g;
                else X[i * ld + c] = T(unit_rows ? g / sqrt(nrm) : scale * g);
            }
        }
    }
}

// Re-opt (Sec. 4.1): C <- s C_0 in every stored precision (FP64 product, then
// the float and double-float mirrors of it, as lorads_create builds them).
__global__ void k_scale_c(int64_t nnz, const double* c0, double s, double* c, float* c32, dfloat* cdf) {
    for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < nnz; q += (int64_t)gridDim.x * blockDim.x) {
        const double v = c0[q] * s;
        c[q] = v;
        c32[q] = (float)v;
        const float h = (float)v;
        cdf[q] = dfloat(h, (float)(v - (double)h));
    }
}

// y <- (y / s_old) s_new (the multiplier of the original problem, rescaled), and
// its double-float mirror
__global__ void k_rescale_y(int64_t m, double* y, dfloat* ydf, double s_old, double s_new) {
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < m; k += (int64_t)gridDim.x * blockDim.x) {
        const double v = (y[k] / s_old) * s_new;
        y[k] = v;
        if (ydf != nullptr) ydf[k] = dfloat(v);
    }
}

template <typename TI, typename TO>
__global__ void k_convert(int64_t n, int ld_in, int ld_out, int r, const TI* in, TO* out) {
    const int64_t total = n * (int64_t)ld_out;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = e / ld_out;
        const int c = (int)(e - i * ld_out);
        out[e] = (c < r) ? TO(in[i * ld_in + c]) : TO(0.0);
    }
}

// ---------------------------------------------------------------- Lanczos on C - A*(y)
// Vectors are n x 4 row-major with the value in column 0 (the SpMM's layout).
// lz[0..]: alpha_j, lz[kLzBeta + j]: beta_j, lz[kLzScalar]: scratch scalars.
__global__ void k_lz_random(int64_t n, uint64_t seed, double* v, double* part) {
    double acc[1] = {0.0};
    const uint64_t golden = 0x9E3779B97F4A7C15ull;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const uint64_t x = splitmix_out(seed + (uint64_t)(i + 1) * golden);
        const double u = (double)(x >> 11) * (1.0 / 9007199254740992.0) - 0.5;
        v[i * 4] = u;
        v[i * 4 + 1] = v[i * 4 + 2] = v[i * 4 + 3] = 0.0;
        acc[0] += u * u;
    }
    block_partials<1>(acc, part);
}

// out[q] <- sum over blocks (first thread), scalar post-processing by `mode`
__global__ void k_lz_scalar(const double* part, int nb, double* lz, int slot, int mode) {
    __shared__ double s[1];
    fold_parts(part, nb, 1, s);
    __syncthreads();
    if (threadIdx.x != 0) return;
    lz[slot] = mode == 1 ? sqrt(fmax(s[0], 0.0)) : s[0];
}

// v <- v / lz[slot]
__global__ void k_lz_scale(int64_t n, double* v, const double* lz, int slot) {
    const double nrm = lz[slot];
    const double inv = nrm > 0.0 ? 1.0 / nrm : 0.0;          // exhausted Krylov space: stop at 0
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        v[i * 4] *= inv;
}

// partial <w, v>
__global__ void k_lz_dot(int64_t n, const double* w, const double* v, double* part) {
    double acc[1] = {0.0};
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        acc[0] += w[i * 4] * v[i * 4];
    block_partials<1>(acc, part);
}

// w <- w - alpha v - beta v_prev ; partial |w|^2
__global__ void k_lz_orth(int64_t n, double* w, const double* v, const double* vp, const double* lz, int a_slot,
                          int b_slot, double* part) {
    const double alpha = lz[a_slot];
    const double beta = b_slot >= 0 ? lz[b_slot] : 0.0;
    double acc[1] = {0.0};
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const double x = w[i * 4] - alpha * v[i * 4] - beta * vp[i * 4];
        w[i * 4] = x;
        acc[0] += x * x;
    }
    block_partials<1>(acc, part);
}

// smallest eigenvalue of the k x k tridiagonal (alpha, beta) by Sturm-count bisection
__global__ void k_lz_tridiag_min(const double* lz, int k, int beta_off, double* out) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    const double* a = lz;
    const double* b = lz + beta_off;          // b[j] couples j-1 and j (b[0] unused)
    double lo = 1e300, hi = -1e300;
    for (int j = 0; j < k; ++j) {             // Gershgorin
        const double rad = (j > 0 ? fabs(b[j]) : 0.0) + (j + 1 < k ? fabs(b[j + 1]) : 0.0);
        lo = fmin(lo, a[j] - rad);
        hi = fmax(hi, a[j] + rad);
    }
    for (int it = 0; it < 200 && hi - lo > 1e-15 * fmax(fabs(lo), fabs(hi)); ++it) {
        const double x = 0.5 * (lo + hi);
        int neg = 0;
        double q = 1.0;
        for (int j = 0; j < k; ++j) {
            const double bb = j > 0 ? b[j] * b[j] : 0.0;
            q = (a[j] - x) - (j > 0 ? bb / q : 0.0);
            if (q == 0.0) q = -1e-300;
            if (q < 0.0) ++neg;
        }
        if (neg >= 1) hi = x; else lo = x;
    }
    *out = 0.5 * (lo + hi);
}

// ---------------------------------------------------------------- host launchers
void ctrl_root(cudaStream_t s, Ctrl* c, const double* pd, int nbd, const double* pl, int nbl, const double* pc, int nbc) {
    k_ctrl_root<<<1, 256, 0, s>>>(c, pd, nbd, pl, nbl, pc, nbc);
}
void ls_finish(cudaStream_t s, const double* pl, int nbl, const double* pc, int nbc, double rho, double* out) {
    k_ls_finish<<<1, 256, 0, s>>>(pl, nbl, pc, nbc, rho, out);
}
void ctrl_hist(cudaStream_t s, Ctrl* c, int mode, const double* pu, int nbu, const double* py, int nby) {
    k_ctrl_hist<<<1, 256, 0, s>>>(c, mode, pu, nbu, py, nby);
}
void ctrl_outer(cudaStream_t s, Ctrl* c, const double* pc, int nbc, const double* po, int nbo) {
    k_ctrl_outer<<<1, 256, 0, s>>>(c, pc, nbc, po, nbo);
}
void ctrl_init(cudaStream_t s, Ctrl* c, const double* pc, int nbc, const double* po, int nbo) {
    k_ctrl_init<<<1, 256, 0, s>>>(c, pc, nbc, po, nbo);
}
void ctrl_resume(cudaStream_t s, Ctrl* c) { k_ctrl_resume<<<1, 1, 0, s>>>(c); }
void quartic_step_dev(cudaStream_t s, const double* a, double* tau) { k_quartic_step<<<1, 1, 0, s>>>(a, tau); }
void fold_to(cudaStream_t s, const double* part, int nb, int NQ, double* out) {
    k_fold_to<<<1, 256, 0, s>>>(part, nb, NQ, out);
}
void lz_random(cudaStream_t s, int64_t n, uint64_t seed, double* v, double* part, int blocks) {
    k_lz_random<<<blocks, kThreads, 0, s>>>(n, seed, v, part);
}
void lz_scalar(cudaStream_t s, const double* part, int nb, double* lz, int slot, int mode) {
    k_lz_scalar<<<1, 256, 0, s>>>(part, nb, lz, slot, mode);
}
void lz_scale(cudaStream_t s, int64_t n, double* v, const double* lz, int slot, int blocks) {
    k_lz_scale<<<blocks, kThreads, 0, s>>>(n, v, lz, slot);
}
void lz_dot(cudaStream_t s, int64_t n, const double* w, const double* v, double* part, int blocks) {
    k_lz_dot<<<blocks, kThreads, 0, s>>>(n, w, v, part);
}
void lz_orth(cudaStream_t s, int64_t n, double* w, const double* v, const double* vp, const double* lz, int a_slot,
             int b_slot, double* part, int blocks) {
    k_lz_orth<<<blocks, kThreads, 0, s>>>(n, w, v, vp, lz, a_slot, b_slot, part);
}
void lz_tridiag_min(cudaStream_t s, const double* lz, int k, int beta_off, double* out) {
    k_lz_tridiag_min<<<1, 32, 0, s>>>(lz, k, beta_off, out);
}

template <typename T>
void sumsq(cudaStream_t s, int64_t n, int ld, int r, const void* X, double* part, int blocks) {
    k_sumsq<T><<<blocks, kThreads, 0, s>>>(n, ld, r, static_cast<const T*>(X), part);
}
template void sumsq<double>(cudaStream_t, int64_t, int, int, const void*, double*, int);
template void sumsq<float>(cudaStream_t, int64_t, int, int, const void*, double*, int);
template void sumsq<dfloat>(cudaStream_t, int64_t, int, int, const void*, double*, int);

template <typename T>
void rank_columns(cudaStream_t s, int64_t n, int ld, int r_old, int r_new, double scale, uint64_t seed,
                  uint64_t stream, void* X, int blocks) {
    k_rank_columns<T><<<blocks, kThreads, 0, s>>>(n, ld, r_old, r_new, scale, seed, stream, static_cast<T*>(X));
}
template void rank_columns<double>(cudaStream_t, int64_t, int, int, int, double, uint64_t, uint64_t, void*, int);
template void rank_columns<float>(cudaStream_t, int64_t, int, int, int, double, uint64_t, uint64_t, void*, int);
template void rank_columns<dfloat>(cudaStream_t, int64_t, int, int, int, double, uint64_t, uint64_t, void*, int);

template <typename T>
void random_start(cudaStream_t s, int64_t n, int ld, int r, uint64_t seed, int unit_rows, double scale, void* X,
                  int blocks) {
    k_random_start<T><<<blocks, kThreads, 0, s>>>(n, ld, r, seed, unit_rows, scale, static_cast<T*>(X));
}
template void random_start<double>(cudaStream_t, int64_t, int, int, uint64_t, int, double, void*, int);
template void random_start<float>(cudaStream_t, int64_t, int, int, uint64_t, int, double, void*, int);
template void random_start<dfloat>(cudaStream_t, int64_t, int, int, uint64_t, int, double, void*, int);

void scale_c(cudaStream_t s, int64_t nnz, const double* c0, double scale, double* c, float* c32, dfloat* cdf,
             int blocks) {
    k_scale_c<<<blocks, 256, 0, s>>>(nnz, c0, scale, c, c32, cdf);
}

void rescale_y(cudaStream_t s, int64_t m, double* y, dfloat* ydf, double s_old, double s_new, int blocks) {
    k_rescale_y<<<blocks, 256, 0, s>>>(m, y, ydf, s_old, s_new);
}

template <typename TI, typename TO>
void convert(cudaStream_t s, int64_t n, int ld_in, int ld_out, int r, const void* in, void* out, int blocks) {
    k_convert<TI, TO><<<blocks, kThreads, 0, s>>>(n, ld_in, ld_out, r, static_cast<const TI*>(in),
                                                   static_cast<TO*>(out));
}
template void convert<double, double>(cudaStream_t, int64_t, int, int, int, const void*, void*, int);
template void convert<double, float>(cudaStream_t, int64_t, int, int, int, const void*, void*, int);
template void convert<float, double>(cudaStream_t, int64_t, int, int, int, const void*, void*, int);
template void convert<float, float>(cudaStream_t, int64_t, int, int, int, const void*, void*, int);
template void convert<double, dfloat>(cudaStream_t, int64_t, int, int, int, const void*, void*, int);
template void convert<dfloat, double>(cudaStream_t, int64_t, int, int, int, const void*, void*, int);
template void convert<dfloat, dfloat>(cudaStream_t, int64_t, int, int, int, const void*, void*, int);

}  // namespace lorads
