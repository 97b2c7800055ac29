// ep_ff.cuh -- float-float ("double-single") arithmetic for the FP64 side of
// the refined solver.
//
// A value is carried as an unevaluated sum hi + lo of two floats with
// |lo| <= ulp(hi)/2, a 48-bit significand (relative precision ~3.6e-15).
// Products are split exactly with an FMA (the error of a*b is fma(a, b, -ab)),
// sums with Knuth's TwoSum; every operation uses the _rn intrinsics so the
// compiler cannot contract a multiply into a following add, which would
// break these error-free transformations.
//
// Why: on GB300 the FP64 pipe runs at about 1/60 of the FP32 rate
// (1.2 vs 73 TFLOP/s measured), so a 27-point FP64 stencil row costs 27 slow
// DFMAs, while the same row in float-float costs ~12 FP32 operations per
// coupling on the fast pipe.  The refinement only needs the residual to
// ~1e-13 relative (its target is 1e-10).
#pragma once

#include <cuda_runtime.h>

namespace epk {

// s + e = a + b exactly
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
    s = __fadd_rn(a, b);
    const float bp = __fsub_rn(s, a);
    e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bp)), __fsub_rn(b, bp));
}

// s + e = a + b exactly, assuming |a| >= |b| (or a == 0)
__device__ __forceinline__ void quick_two_sum(float a, float b, float& s, float& e) {
    s = __fadd_rn(a, b);
    e = __fsub_rn(b, __fsub_rn(s, a));
}

// (sh, sl) += (ah + al) * (xh + xl), dropping al*xl (below 2^-48 relative)
__device__ __forceinline__ void ff_mac(float ah, float al, float xh, float xl, float& sh, float& sl) {
    const float p = __fmul_rn(ah, xh);
    float e = __fmaf_rn(ah, xh, -p);
    e = __fmaf_rn(ah, xl, __fmaf_rn(al, xh, e));
    float s, t;
    two_sum(sh, p, s, t);
    sh = s;
    sl = __fadd_rn(sl, __fadd_rn(t, e));
}

__device__ __forceinline__ void ff_normalize(float& hi, float& lo) {
    float s, e;
    quick_two_sum(hi, lo, s, e);
    hi = s;
    lo = e;
}

// (rh, rl) = (ah + al) - (bh + bl)
__device__ __forceinline__ void ff_sub(float ah, float al, float bh, float bl, float& rh, float& rl) {
    float s, e;
    two_sum(ah, -bh, s, e);
    e = __fadd_rn(e, __fsub_rn(al, bl));
    quick_two_sum(s, e, rh, rl);
}

// (rh, rl) = (ah + al) + b
__device__ __forceinline__ void ff_add_f(float ah, float al, float b, float& rh, float& rl) {
    float s, e;
    two_sum(ah, b, s, e);
    e = __fadd_rn(e, al);
    quick_two_sum(s, e, rh, rl);
}

// (rh, rl) = (ah + al) * (bh + bl), dropping al*bl
__device__ __forceinline__ void ff_mul(float ah, float al, float bh, float bl, float& rh, float& rl) {
    const float p = __fmul_rn(ah, bh);
    float e = __fmaf_rn(ah, bh, -p);
    e = __fmaf_rn(ah, bl, __fmaf_rn(al, bh, e));
    quick_two_sum(p, e, rh, rl);
}

// (sh, sl) += c * (xh + xl) for a power-of-two c (the product is exact)
__device__ __forceinline__ void ff_acc_pow2(float c, float xh, float xl, float& sh, float& sl) {
    float s, t;
    two_sum(sh, __fmul_rn(c, xh), s, t);
    sh = s;
    sl = __fadd_rn(sl, __fadd_rn(t, __fmul_rn(c, xl)));
}

// nearest float-float of a double (exact for doubles with <= 48 significant bits)
__device__ __forceinline__ void ff_from_double(double x, float& hi, float& lo) {
    hi = __double2float_rn(x);
    lo = __double2float_rn(x - (double)hi);
}

__device__ __forceinline__ double ff_to_double(float hi, float lo) { return (double)hi + (double)lo; }

}  // namespace epk
