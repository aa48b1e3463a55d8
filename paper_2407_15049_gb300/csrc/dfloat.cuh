// Double-float ("double-word") arithmetic on FP32 units.
//
// A value is the unevaluated sum hi + lo of two floats with |lo| <= ulp(hi)/2,
// i.e. a ~48-bit significand.  GB300 executes FP32 at ~64x its FP64 rate, so
// this keeps FP64-class accuracy for the master iterate (R, C R) and for the
// partial sums of every reduction without touching the FP64 pipe.
//
// Building blocks: Knuth's TwoSum, Dekker's Fast2Sum and the FMA form of the
// exact product (TwoProd); the double-word add, multiply and FP multiply
// follow the algorithms analysed by Joldes, Muller and Popescu, "Tight and
// rigorous error bounds for basic building blocks of double-word arithmetic"
// (ACM TOMS 44(2), 2017): AccurateDWPlusDW, DWTimesDW (FMA variant),
// DWTimesFP (FMA variant), DWPlusFP.  Written here from those definitions.
#pragma once

#include <cuda_runtime.h>

namespace lorads {

struct dfloat {
    float hi, lo;
    __host__ __device__ __forceinline__ dfloat() : hi(0.f), lo(0.f) {}
    __host__ __device__ __forceinline__ dfloat(float h, float l) : hi(h), lo(l) {}
    __host__ __device__ __forceinline__ dfloat(int x) : hi((float)x), lo(0.f) {}
    __host__ __device__ __forceinline__ dfloat(float x) : hi(x), lo(0.f) {}
    __host__ __device__ __forceinline__ dfloat(double x) {
        hi = (float)x;
        lo = (float)(x - (double)hi);
    }
    __host__ __device__ __forceinline__ explicit operator double() const { return (double)hi + (double)lo; }
    __host__ __device__ __forceinline__ explicit operator float() const { return hi + lo; }
};

// ----------------------------------------------------------------- error-free transformations
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
    s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}
__device__ __forceinline__ void fast_two_sum(float a, float b, float& s, float& e) {  // |a| >= |b|
    s = __fadd_rn(a, b);
    e = __fsub_rn(b, __fsub_rn(s, a));
}
__device__ __forceinline__ void two_prod(float a, float b, float& p, float& e) {
    p = __fmul_rn(a, b);
    e = __fmaf_rn(a, b, -p);
}

// ----------------------------------------------------------------- arithmetic
__device__ __forceinline__ dfloat operator+(dfloat x, dfloat y) {        // AccurateDWPlusDW
    float sh, sl, th, tl, vh, vl, zh, zl;
    two_sum(x.hi, y.hi, sh, sl);
    two_sum(x.lo, y.lo, th, tl);
    const float c = __fadd_rn(sl, th);
    fast_two_sum(sh, c, vh, vl);
    const float w = __fadd_rn(tl, vl);
    fast_two_sum(vh, w, zh, zl);
    return dfloat(zh, zl);
}
__device__ __forceinline__ dfloat operator-(dfloat x) { return dfloat(-x.hi, -x.lo); }
__device__ __forceinline__ dfloat operator-(dfloat x, dfloat y) { return x + (-y); }
__device__ __forceinline__ dfloat operator*(dfloat x, dfloat y) {        // DWTimesDW (FMA)
    float ch, cl1;
    two_prod(x.hi, y.hi, ch, cl1);
    const float tl0 = __fmul_rn(x.lo, y.lo);
    const float tl1 = __fmaf_rn(x.hi, y.lo, tl0);
    const float cl2 = __fmaf_rn(x.lo, y.hi, tl1);
    const float cl3 = __fadd_rn(cl1, cl2);
    float zh, zl;
    fast_two_sum(ch, cl3, zh, zl);
    return dfloat(zh, zl);
}
__device__ __forceinline__ dfloat mul_fp(dfloat x, float y) {             // DWTimesFP (FMA)
    float ch, cl1;
    two_prod(x.hi, y, ch, cl1);
    const float cl3 = __fmaf_rn(x.lo, y, cl1);
    float zh, zl;
    fast_two_sum(ch, cl3, zh, zl);
    return dfloat(zh, zl);
}
__device__ __forceinline__ dfloat add_fp(dfloat x, float y) {             // DWPlusFP
    float sh, sl;
    two_sum(x.hi, y, sh, sl);
    const float v = __fadd_rn(x.lo, sl);
    float zh, zl;
    fast_two_sum(sh, v, zh, zl);
    return dfloat(zh, zl);
}
__device__ __forceinline__ dfloat& operator+=(dfloat& x, dfloat y) { return x = x + y; }
__device__ __forceinline__ dfloat& operator+=(dfloat& x, float y) { return x = add_fp(x, y); }
__device__ __forceinline__ dfloat& operator-=(dfloat& x, dfloat y) { return x = x - y; }
// fma for every arithmetic type of the kernels (a lorads::fma would otherwise hide
// the float and double ones inside this namespace)
__device__ __forceinline__ float fma(float a, float b, float c) { return __fmaf_rn(a, b, c); }
__device__ __forceinline__ double fma(double a, double b, double c) { return __fma_rn(a, b, c); }
__device__ __forceinline__ dfloat fma(dfloat a, dfloat b, dfloat c) { return a * b + c; }

// ----------------------------------------------------------------- fused row-update helpers
// Generic forms (double, float, double-float with a double-float operand) and
// cheaper forms for a double-float master with float work arrays.

// r + tau*d: the float product tau*d is the step actually taken (and stored as s)
template <typename AR, typename AD>
__device__ __forceinline__ AR step_add(AR r, AR tau, AD tau_d, AD d) { return fma(tau, AR(d), r); }
template <>
__device__ __forceinline__ dfloat step_add<dfloat, float>(dfloat r, dfloat, float tau_d, float d) {
    return add_fp(r, __fmul_rn(tau_d, d));
}

// acc + r*r
template <typename AR>
__device__ __forceinline__ AR sq_add(AR acc, AR r) { return fma(r, r, acc); }
template <>
__device__ __forceinline__ dfloat sq_add<dfloat>(dfloat acc, dfloat r) {
    float ph, pl;
    two_prod(r.hi, r.hi, ph, pl);                       // exact hi^2
    pl = __fmaf_rn(2.f * r.hi, r.lo, pl);               // + 2 hi lo (lo^2 below the precision)
    return add_fp(add_fp(acc, ph), pl);
}

// 2 (cr - coef r), rounded to the work type
template <typename AR, typename AD>
__device__ __forceinline__ AD grad_elem(AR cr, AR coef, AR r) { return AD(AR(2) * (cr - coef * r)); }
template <>
__device__ __forceinline__ float grad_elem<dfloat, float>(dfloat cr, dfloat coef, dfloat r) {
    float ph, pl, sh, sl;
    two_prod(coef.hi, r.hi, ph, pl);                    // exact coef_hi r_hi
    two_sum(cr.hi, -ph, sh, sl);                        // exact cr_hi - coef_hi r_hi
    const float low = sl - pl + cr.lo - __fmaf_rn(coef.hi, r.lo, coef.lo * r.hi);
    return 2.f * (sh + low);
}

// full-warp butterfly exchange for every arithmetic type used in reductions
__device__ __forceinline__ float shfl_xor(float v, int o) { return __shfl_xor_sync(0xffffffffu, v, o); }
__device__ __forceinline__ double shfl_xor(double v, int o) { return __shfl_xor_sync(0xffffffffu, v, o); }
__device__ __forceinline__ dfloat shfl_xor(dfloat v, int o) {
    return dfloat(__shfl_xor_sync(0xffffffffu, v.hi, o), __shfl_xor_sync(0xffffffffu, v.lo, o));
}

}  // namespace lorads
