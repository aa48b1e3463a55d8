// Shared device helpers of the LoRADS GB300 library: vector units, block
// reductions, the device control block and the launch-shape rules.
#pragma once

#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <stdint.h>
#include "dfloat.cuh"

namespace lorads {

constexpr int kThreads = 256;        // threads per block of every streaming kernel
constexpr int kWarps = kThreads / 32;
constexpr int kMaxMem = 4;           // L-BFGS memory cap (T of Algorithm 1)

// ------------------------------------------------------------------ row shapes
// A row of ld elements is cut into Q = ld/4 units of 4 elements.  A group of
// L lanes (the power of two >= Q, at most 32) owns a row; lane l handles units
// c*L + l < Q for c < CPL = ceil(Q/L), so that each load instruction of a group
// reads up to L consecutive units.  Lanes past Q idle.
constexpr int kMaxCPL = 4;
constexpr int kMaxLd = 4 * 32 * kMaxCPL;   // widest supported row (512 elements)

struct Shape {
    int L;     // lanes per row (power of two)
    int CPL;   // units per lane
    int Q;     // units per row
};

inline bool shape_for_ld(int ld, Shape* s) {
    if (ld <= 0 || (ld % 4) != 0 || ld > kMaxLd) return false;
    const int Q = ld / 4;
    int L = 1;
    while (L < Q && L < 32) L <<= 1;
    s->L = L;
    s->Q = Q;
    s->CPL = (Q + L - 1) / L;
    return s->CPL <= kMaxCPL;
}

// Narrow row groups for the gather-bound SpMM: the fewest lanes per row (a
// power of two, at most kMaxCPL units each) whose idle unit slots do not exceed
// those of shape_for_ld.  More rows per warp means more independent row gathers
// in flight (ld = 24: 2 lanes x 3 units, 16 rows per warp, no idle lane, instead
// of 8 lanes with 2 idle and 4 rows per warp).  Element sums are unchanged: each
// output element is still accumulated by one lane in the order of the stored entries.
inline bool shape_narrow(int ld, Shape* s) {
    Shape d;
    if (!shape_for_ld(ld, &d)) return false;
    const int waste = d.L * d.CPL - d.Q;
    for (int L = 1; L <= d.L; L <<= 1) {
        const int cpl = (d.Q + L - 1) / L;
        if (cpl <= kMaxCPL && L * cpl - d.Q <= waste) {
            s->L = L;
            s->Q = d.Q;
            s->CPL = cpl;
            return true;
        }
    }
    *s = d;
    return true;
}

// Packed row groups (Q lanes, one unit each, floor(32/Q) rows per warp) keep more
// lanes busy than the power-of-two groups of shape_for_ld (ld = 24: 30 of 32 lanes
// instead of 24; ld = 20: 30 instead of 20; ld = 28: 28 either way).
inline bool packed_rows_gain(const Shape& s) {
    return s.CPL == 1 && s.Q <= 32 && (32 / s.Q) * s.Q > (32 / s.L) * s.Q;
}

// Row width used for rank r: r rounded up to a multiple of 4.
inline int padded_ld(int r) { return (r + 3) / 4 * 4; }

// ------------------------------------------------------------------ vector units
// L2 prefetch size of the read-once 16-byte loads of the streaming passes: 128
// (default), 256, or 0 for none.  The context's L2 fetch granularity limit is 64
// bytes on some GB300s and 128 on others; at 64 the step update's streams ran
// 3% faster with the 128-byte hint (2.92 -> 2.83 ms at n = 1e7, r = 24), at 128
// the hint changes nothing.  The neighbour-row gathers of the SpMMs keep plain
// loads: they gain from the smaller granularity (2.37 ms at 64, 2.46 at 128).
#ifndef LORADS_STREAM_L2PF
#define LORADS_STREAM_L2PF 128
#endif
// Read-once load of 16 bytes (evict-first), with the L2 prefetch size above.
__device__ __forceinline__ float4 ld_stream_f4(const float* p) {
#if LORADS_STREAM_L2PF == 128
    float4 a;
    asm volatile("ld.global.cs.L2::128B.v4.f32 {%0, %1, %2, %3}, [%4];"
                 : "=f"(a.x), "=f"(a.y), "=f"(a.z), "=f"(a.w) : "l"(p));
    return a;
#elif LORADS_STREAM_L2PF == 256
    float4 a;
    asm volatile("ld.global.cs.L2::256B.v4.f32 {%0, %1, %2, %3}, [%4];"
                 : "=f"(a.x), "=f"(a.y), "=f"(a.z), "=f"(a.w) : "l"(p));
    return a;
#else
    return __ldcs(reinterpret_cast<const float4*>(p));
#endif
}

template <typename T> struct Unit;      // 4 consecutive elements of type T

template <> struct Unit<double> {
    double v[4];
    __device__ __forceinline__ void load(const double* p) {
        double2 a = *reinterpret_cast<const double2*>(p);
        double2 b = *reinterpret_cast<const double2*>(p + 2);
        v[0] = a.x; v[1] = a.y; v[2] = b.x; v[3] = b.y;
    }
    __device__ __forceinline__ void load_stream(const double* p) {   // read once
        double2 a = __ldcs(reinterpret_cast<const double2*>(p));
        double2 b = __ldcs(reinterpret_cast<const double2*>(p + 2));
        v[0] = a.x; v[1] = a.y; v[2] = b.x; v[3] = b.y;
    }
    __device__ __forceinline__ void store(double* p) const {
        *reinterpret_cast<double2*>(p) = make_double2(v[0], v[1]);
        *reinterpret_cast<double2*>(p + 2) = make_double2(v[2], v[3]);
    }
    __device__ __forceinline__ void store_stream(double* p) const {
        __stcs(reinterpret_cast<double2*>(p), make_double2(v[0], v[1]));
        __stcs(reinterpret_cast<double2*>(p + 2), make_double2(v[2], v[3]));
    }
};

template <> struct Unit<float> {
    float v[4];
    __device__ __forceinline__ void load(const float* p) {
        float4 a = *reinterpret_cast<const float4*>(p);
        v[0] = a.x; v[1] = a.y; v[2] = a.z; v[3] = a.w;
    }
    __device__ __forceinline__ void load_stream(const float* p) {
        float4 a = ld_stream_f4(p);
        v[0] = a.x; v[1] = a.y; v[2] = a.z; v[3] = a.w;
    }
    __device__ __forceinline__ void store(float* p) const {
        *reinterpret_cast<float4*>(p) = make_float4(v[0], v[1], v[2], v[3]);
    }
    __device__ __forceinline__ void store_stream(float* p) const {
        __stcs(reinterpret_cast<float4*>(p), make_float4(v[0], v[1], v[2], v[3]));
    }
};

// bf16 storage, values widened to float on load.
template <> struct Unit<__nv_bfloat16> {
    float v[4];
    __device__ __forceinline__ void from_raw(uint2 a) {
        v[0] = __uint_as_float(a.x << 16);
        v[1] = __uint_as_float(a.x & 0xffff0000u);
        v[2] = __uint_as_float(a.y << 16);
        v[3] = __uint_as_float(a.y & 0xffff0000u);
    }
    __device__ __forceinline__ void load(const __nv_bfloat16* p) {
        from_raw(*reinterpret_cast<const uint2*>(p));
    }
    __device__ __forceinline__ void load_stream(const __nv_bfloat16* p) {
        from_raw(__ldcs(reinterpret_cast<const uint2*>(p)));
    }
    __device__ __forceinline__ void store(__nv_bfloat16* p) const {
        __nv_bfloat162 a = __floats2bfloat162_rn(v[0], v[1]);
        __nv_bfloat162 b = __floats2bfloat162_rn(v[2], v[3]);
        uint2 u;
        u.x = *reinterpret_cast<uint32_t*>(&a);
        u.y = *reinterpret_cast<uint32_t*>(&b);
        *reinterpret_cast<uint2*>(p) = u;
    }
    __device__ __forceinline__ void store_stream(__nv_bfloat16* p) const { store(p); }
};

// double-float storage: (hi, lo) pairs, 8 bytes per element
template <> struct Unit<dfloat> {
    dfloat v[4];
    __device__ __forceinline__ void load(const dfloat* p) {
        const float4 a = *reinterpret_cast<const float4*>(p);
        const float4 b = *reinterpret_cast<const float4*>(p + 2);
        v[0] = dfloat(a.x, a.y); v[1] = dfloat(a.z, a.w); v[2] = dfloat(b.x, b.y); v[3] = dfloat(b.z, b.w);
    }
    __device__ __forceinline__ void load_stream(const dfloat* p) {
        const float4 a = ld_stream_f4(reinterpret_cast<const float*>(p));
        const float4 b = ld_stream_f4(reinterpret_cast<const float*>(p + 2));
        v[0] = dfloat(a.x, a.y); v[1] = dfloat(a.z, a.w); v[2] = dfloat(b.x, b.y); v[3] = dfloat(b.z, b.w);
    }
    __device__ __forceinline__ void store(dfloat* p) const {
        *reinterpret_cast<float4*>(p) = make_float4(v[0].hi, v[0].lo, v[1].hi, v[1].lo);
        *reinterpret_cast<float4*>(p + 2) = make_float4(v[2].hi, v[2].lo, v[3].hi, v[3].lo);
    }
    __device__ __forceinline__ void store_stream(dfloat* p) const {
        __stcs(reinterpret_cast<float4*>(p), make_float4(v[0].hi, v[0].lo, v[1].hi, v[1].lo));
        __stcs(reinterpret_cast<float4*>(p + 2), make_float4(v[2].hi, v[2].lo, v[3].hi, v[3].lo));
    }
};

// arithmetic type of an element once loaded
template <typename T> struct Arith { using type = T; };
template <> struct Arith<__nv_bfloat16> { using type = float; };

// ------------------------------------------------------------------ reductions
// Sums NQ per-thread partials (double or double-float) over the block (up to
// 1024 threads) and
// writes them as doubles to part[bid * NQ + q].  Fixed order:
// deterministic for a fixed grid.
// Block index and count a kernel body runs with: the hardware grid for a
// launch of its own, or one block standing for the whole grid when a
// persistent kernel runs the body for one instance.
// `pslot` is the partial-sum slot the block writes (its index in its own grid).
struct VGrid {
    int bid, nblk, pslot;
};
__device__ __forceinline__ VGrid hw_grid() { return VGrid{(int)blockIdx.x, (int)gridDim.x, (int)blockIdx.x}; }

template <int NQ, typename PA>
__device__ __forceinline__ void block_partials(PA (&acc)[NQ], double* part, int bid) {
    __shared__ double red[32][NQ > 0 ? NQ : 1];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
    for (int q = 0; q < NQ; ++q) {
        PA v = acc[q];                       // warp tree in the partial's own type
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v += shfl_xor(v, o);
        if (lane == 0) red[warp][q] = double(v);
    }
    __syncthreads();
    for (int q = threadIdx.x; q < NQ; q += blockDim.x) {
        double s = 0.0;
        for (int w = 0; w < nw; ++w) s += red[w][q];
        part[(size_t)bid * NQ + q] = s;
    }
}
template <int NQ, typename PA>
__device__ __forceinline__ void block_partials(PA (&acc)[NQ], double* part) {
    block_partials<NQ, PA>(acc, part, (int)blockIdx.x);
}

// Reduces a group-of-L-lanes value; every lane of the group gets the sum.
template <typename V>
__device__ __forceinline__ V group_sum(V v, int L) {
    for (int o = L >> 1; o > 0; o >>= 1) v += shfl_xor(v, o);
    return v;
}

// ------------------------------------------------------------------ control block
enum { PHASE_INNER = 0, PHASE_OUTER = 1 };

// Device-resident state of one solve.  Written by the single-block control
// kernels, read by every streaming kernel (which skip their work when the
// phase flags say so).
struct Ctrl {
    // scalars of the current inner iteration
    double rho;
    double tau;
    double a[4];
    double gD;                  // <G, D>
    double DD;                  // ||D||^2
    double gnorm2;              // ||G||^2 at the current R
    double znorm2;              // ||A(RR^T) - b||^2 at the current R
    // two-loop coefficients of the next direction: D = cG G + sum cS S_u + sum cY Y_u
    double cG, cS[kMaxMem], cY[kMaxMem];
    // Gram data of the stored pairs, indexed by physical slot
    double g_s[kMaxMem], g_y[kMaxMem];          // <G, S_u>, <G, Y_u>
    double SY[kMaxMem][kMaxMem];                // <S_u, Y_v>
    double YY[kMaxMem][kMaxMem];                // <Y_u, Y_v>
    double SS_new;                              // ||S_new||^2 of the last step
    int order[kMaxMem];                         // physical slot by age (0 = oldest)
    int mem_count;
    int new_slot;                               // slot the next pair is written to
    int old_count;                              // pairs kept besides the new slot
    int old_slots[kMaxMem];
    // phase flags
    int phase;                  // PHASE_INNER (L-BFGS) or PHASE_OUTER (multiplier step)
    int step_ok;                // 1 if the current iteration takes a step (tau > 0)
    int inner_done;
    int solve_done;
    int pause;                  // host action needed (rank update)
    int status;                 // lorads_status of the solve
    int dev_error;              // set by a kernel whose bounded wait expired
    int inner_k;                // directions computed in this outer step
    int outer;
    int total_inner;
    int hit_cap_streak;
    int lbfgs_mem;
    int max_inner;
    int max_outer;
    int rank_threshold;
    int total_limit;            // > 0: stop after this many L-BFGS iterations in total
    int lbfgs_scaling;
    int rho_policy;
    int inner_scale;
    int stop_rule;              // 0: err1 and |err3| <= tol; 1: err1 <= tol alone (the stop before re-opt)
    // outer-loop state
    double tol, inner_rel, inner_progress, gnorm0, bnorm1, bnorm_inf;
    double rho_growth, rho_max, infeas_decrease;
    double err1, err1_prev, err3, primal_obj, dual_obj;
    double last_iter_rho;
};

// Partial-sum slots of each producing kernel.
enum {
    // direction kernel
    PD_GD = 0, PD_DD, PD_N,
    // SpMM with line-search epilogue (and constraint pass, same slots)
    PL_P1 = 0, PL_P2, PL_YQ1, PL_YQ2, PL_Q1Q1, PL_Q1Q2, PL_Q2Q2, PL_N,
    // constraint pass in y~ / multiplier mode
    PC_ZZ = 0, PC_BY, PC_N,
    // SpMM C R with objective
    PO_CRR = 0, PO_N,
};
// row-update kernel: fixed slots then 3 per old pair; <G',S_v>, <G',Y_v>,
// <G',S_new> and ||S_new||^2 follow from these and the previous Gram data
enum { PU_GG = 0, PU_ZZ, PU_GYN, PU_SYN, PU_YYN, PU_FIXED };
constexpr int PU_PER_OLD = 3;          // <S_new,Y_v>, <S_v,Y_new>, <Y_new,Y_v>
constexpr int PU_N = PU_FIXED + PU_PER_OLD * (kMaxMem - 1);

}  // namespace lorads
