// Double-word arithmetic on the FP32 pipes: a value is the unevaluated sum
// hi + lo of two floats with |lo| <= ulp(hi)/2, about 48 significant bits.
//
// GB300 runs FP64 at about 1/64 of the FP32 rate, so FP64-accurate work that
// is long (the multipole recurrences and translations that feed the MAC)
// runs faster as double-word FP32. The building blocks are the error-free
// transformations (Knuth's TwoSum, Dekker's FastTwoSum, and the product
// error by one fused multiply-add) and the double-word algorithms of Joldes,
// Muller and Popescu, "Tight and rigorous error bounds for basic building
// blocks of double-word arithmetic", ACM TOMS 44 (2017): the accurate
// DW + DW sum, DW x DW with FMA and DW x FP with FMA, each with a relative
// error of a few u^2, u = 2^-24 (the bounds are proved there).
//
// Every operation uses the _rn intrinsics, so the compiler neither
// contracts nor reorders them (the transformations need each rounding as
// written). Values must stay in the normal FP32 range (|x| > 2^-100 or
// zero, |x| < 2^100) for the bounds to hold.
#pragma once

#include <cuda_runtime.h>

namespace gbfmm {

struct dw {
    float hi, lo;
};

__device__ __forceinline__ dw dw_make(float h, float l) { return dw{h, l}; }

// FP64 -> double-word (exact to 48 bits) and back
__device__ __forceinline__ dw dw_from(double x) {
    const float h = __double2float_rn(x);
    return dw{h, __double2float_rn(x - (double)h)};
}
__device__ __forceinline__ double dw_to(dw a) { return (double)a.hi + (double)a.lo; }

// s + e = a + b exactly (Knuth)
__device__ __forceinline__ dw ew_two_sum(float a, float b) {
    const float s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    const float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
    return dw{s, e};
}
// the same when |a| >= |b| or a == 0 (Dekker)
__device__ __forceinline__ dw ew_fast_two_sum(float a, float b) {
    const float s = __fadd_rn(a, b);
    return dw{s, __fsub_rn(b, __fsub_rn(s, a))};
}
// p + e = a * b exactly (one FMA gives the rounding error of the product)
__device__ __forceinline__ dw ew_two_prod(float a, float b) {
    const float p = __fmul_rn(a, b);
    return dw{p, __fmaf_rn(a, b, -p)};
}

// accurate DW + DW
__device__ __forceinline__ dw dw_add(dw x, dw y) {
    const dw s = ew_two_sum(x.hi, y.hi);
    const dw t = ew_two_sum(x.lo, y.lo);
    const float c = __fadd_rn(s.lo, t.hi);
    const dw v = ew_fast_two_sum(s.hi, c);
    const float w = __fadd_rn(t.lo, v.lo);
    return ew_fast_two_sum(v.hi, w);
}
__device__ __forceinline__ dw dw_neg(dw x) { return dw{-x.hi, -x.lo}; }
__device__ __forceinline__ dw dw_sub(dw x, dw y) { return dw_add(x, dw_neg(y)); }

// DW x DW with FMA
__device__ __forceinline__ dw dw_mul(dw x, dw y) {
    const dw c = ew_two_prod(x.hi, y.hi);
    const float t0 = __fmul_rn(x.lo, y.lo);
    const float t1 = __fmaf_rn(x.hi, y.lo, t0);
    const float c2 = __fmaf_rn(x.lo, y.hi, t1);
    const float c3 = __fadd_rn(c.lo, c2);
    return ew_fast_two_sum(c.hi, c3);
}

// DW x FP with FMA
__device__ __forceinline__ dw dw_mul_f(dw x, float y) {
    const dw c = ew_two_prod(x.hi, y);
    const float c3 = __fmaf_rn(x.lo, y, c.lo);
    return ew_fast_two_sum(c.hi, c3);
}

}  // namespace gbfmm
