// Argument blocks and declarations of the kernel launchers (host side).
#pragma once

#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <stdint.h>
#include "common.cuh"

namespace lorads {

struct ProbDev;

struct SpmmCArgs {
    const ProbDev& p;
    const void* X; void* out; int ld; Shape sh;
    const double* v; int write_out; int epi;
    const void* R; const double* y; const void* zrow; const dfloat* ydf; const Ctrl* ctrl; double rho; double* part;
    int blocks; const Ctrl* gate; int ph; cudaStream_t stream;
    int prefetch = 0;   // 1: carry the next row's bounds and prefetch its entries and row terms into L2;
                        // 2: also the bounds of the row after next and one neighbour row of the next row
    int dense = 0;      // line-search epilogue: packed row groups of Q lanes (one unit per lane)
};

// v: double[m], or double-float[m] when v_df (weights then formed without FP64)
struct SpmmAArgs {
    const ProbDev& p;
    const void* X; void* out; int ld; Shape sh;
    const void* v; double alpha; int accumulate;
    int blocks; const Ctrl* gate; int ph; cudaStream_t stream; int v_df;
};

// out: double[m] (CONS_EVAL) or y~ in the pass's scalar type (CONS_YTIL: double on
// the FP64 path, double-float otherwise); zk: cached z in that same type
struct ConsArgs {
    const ProbDev& p;
    int mode; int64_t k0, k1;
    const void* U; const void* V; int ld; Shape sh;
    double* y; void* out; void* zk; dfloat* ydf; const Ctrl* ctrl; double rho; double* part;
    int blocks; const Ctrl* gate; int ph; cudaStream_t stream;
};

struct DirArgs {
    int64_t nunits; const void* G; void* D; const void* hist; int64_t slot_stride;
    const Ctrl* ctrl; double* part; int blocks; const Ctrl* gate; int ph; cudaStream_t stream;
};

struct StepArgs {
    int64_t nunits; void* R; void* CR; const void* D; const void* CD;
    const Ctrl* ctrl; int blocks; const Ctrl* gate; int ph; cudaStream_t stream;
};

struct UpdateArgs {
    const ProbDev& p;
    bool step; bool hist_on;
    void* R; void* CR; const void* D; const void* CD; void* G; const void* W; void* hist;
    int64_t slot_stride; int ld; Shape sh; const double* y; const dfloat* ydf; void* zrow; const Ctrl* ctrl;
    double* part;
    int blocks; const Ctrl* gate; int ph; cudaStream_t stream;
    int extra_blocks;   // step update: 0, or the variant with 1 or 2 more resident blocks per SM
    int prefetch = 0;   // step update with extra blocks: 1 = L2 prefetch of each group's next row
    int dense = 0;      // step update with extra blocks: packed row groups of Q lanes (one unit per lane)
    int max_old = 3;    // step update with extra blocks: stored pairs besides the new one (T - 1) at most
};

template <typename TX, typename TO, typename TR> void launch_spmm_c(const SpmmCArgs& a);
template <typename TX, typename TO> void launch_spmm_a(const SpmmAArgs& a);
template <typename TU, typename TV> void launch_cons(const ConsArgs& a);
// TDIR: storage type of the direction D (defaults to the work type TD)
template <typename TD, typename TDIR = TD> void launch_dir(const DirArgs& a);
template <typename TR, typename TD, typename TDIR = TD> void launch_step(const StepArgs& a);
template <typename TR, typename TD, typename TDIR = TD> void launch_update(const UpdateArgs& a);

using bf16 = __nv_bfloat16;

// instantiated in kern_fp64.cu
extern template void launch_spmm_c<double, double, double>(const SpmmCArgs&);
extern template void launch_spmm_a<double, double>(const SpmmAArgs&);
extern template void launch_cons<double, double>(const ConsArgs&);
extern template void launch_dir<double, double>(const DirArgs&);
extern template void launch_step<double, double, double>(const StepArgs&);
extern template void launch_update<double, double, double>(const UpdateArgs&);
// kern_mixed.cu: double-float master R / C R, FP32 direction, gradient and history
extern template void launch_spmm_c<float, float, dfloat>(const SpmmCArgs&);
extern template void launch_spmm_a<dfloat, float>(const SpmmAArgs&);
extern template void launch_cons<dfloat, float>(const ConsArgs&);
extern template void launch_step<dfloat, float, float>(const StepArgs&);
extern template void launch_update<dfloat, float, float>(const UpdateArgs&);
// kern_df.cu: double-float everywhere
extern template void launch_spmm_c<dfloat, dfloat, dfloat>(const SpmmCArgs&);
extern template void launch_spmm_a<dfloat, dfloat>(const SpmmAArgs&);
extern template void launch_cons<dfloat, dfloat>(const ConsArgs&);
extern template void launch_dir<dfloat, dfloat>(const DirArgs&);
extern template void launch_step<dfloat, dfloat, dfloat>(const StepArgs&);
extern template void launch_update<dfloat, dfloat, dfloat>(const UpdateArgs&);
// kern_fp32.cu
extern template void launch_spmm_c<float, float, float>(const SpmmCArgs&);
extern template void launch_spmm_a<float, float>(const SpmmAArgs&);
extern template void launch_cons<float, float>(const ConsArgs&);
extern template void launch_dir<float, float>(const DirArgs&);
extern template void launch_step<float, float, float>(const StepArgs&);
extern template void launch_update<float, float, float>(const UpdateArgs&);
// kern_mixed_bf16.cu: the mixed form with the direction D stored in bf16
extern template void launch_dir<float, bf16>(const DirArgs&);
extern template void launch_spmm_c<bf16, float, dfloat>(const SpmmCArgs&);
extern template void launch_cons<dfloat, bf16>(const ConsArgs&);
extern template void launch_step<dfloat, float, bf16>(const StepArgs&);
extern template void launch_update<dfloat, float, bf16>(const UpdateArgs&);
// kern_bf16.cu: bf16 storage, FP32 arithmetic (standalone entry points)
extern template void launch_spmm_c<bf16, float, bf16>(const SpmmCArgs&);
extern template void launch_spmm_a<bf16, float>(const SpmmAArgs&);
extern template void launch_cons<bf16, bf16>(const ConsArgs&);

}  // namespace lorads
