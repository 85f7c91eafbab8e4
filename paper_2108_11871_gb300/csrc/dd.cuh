// Double-float ("df32") arithmetic on the FP32 pipe.
//
// A value is hi + lo with two FP32 numbers, |lo| <= ulp(hi)/2: about 48
// significant bits, relative rounding ~2^-47.  On GB300 the FP32 pipe is about
// 60 times faster than the FP64 pipe, so FFT butterflies written this way run
// several times faster than in FP64 while keeping errors near 1e-14 relative.
// The building blocks are the classic error-free transformations (Dekker,
// Knuth two-sum; the product error from one FMA) and the "sloppy" double-word
// sum, whose error is bounded relative to |a| + |b| -- enough for FFTs, whose
// error analysis is normwise.  All operations use the _rn intrinsics so the
// compiler cannot contract or reassociate them.
#pragma once
#include <cuda_runtime.h>

namespace idp {

struct ddr {
    float hi, lo;
};
struct ddc {
    ddr re, im;
};

__device__ __forceinline__ ddr dd_make(float h, float l) { ddr r; r.hi = h; r.lo = l; return r; }

__device__ __forceinline__ ddr dd_from(double x)
{
    const float h = __double2float_rn(x);
    return dd_make(h, __double2float_rn(x - (double)h));
}
__device__ __forceinline__ double dd_to(ddr a) { return (double)a.hi + (double)a.lo; }

// s + e = a + b exactly, |a| >= |b| not required
__device__ __forceinline__ ddr two_sum(float a, float b)
{
    const float s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    const float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
    return dd_make(s, e);
}
// s + e = a + b exactly for |a| >= |b|
__device__ __forceinline__ ddr quick_two_sum(float a, float b)
{
    const float s = __fadd_rn(a, b);
    return dd_make(s, __fsub_rn(b, __fsub_rn(s, a)));
}

__device__ __forceinline__ ddr dd_neg(ddr a) { return dd_make(-a.hi, -a.lo); }

__device__ __forceinline__ ddr dd_add(ddr a, ddr b)
{
    const ddr s = two_sum(a.hi, b.hi);
    return quick_two_sum(s.hi, __fadd_rn(s.lo, __fadd_rn(a.lo, b.lo)));
}
__device__ __forceinline__ ddr dd_sub(ddr a, ddr b) { return dd_add(a, dd_neg(b)); }

// unnormalised product p + e = a * b (error ~2^-47 relative)
__device__ __forceinline__ ddr dd_mul_raw(ddr a, ddr b)
{
    const float p = __fmul_rn(a.hi, b.hi);
    float e = __fmaf_rn(a.hi, b.hi, -p);
    e = __fmaf_rn(a.hi, b.lo, e);
    e = __fmaf_rn(a.lo, b.hi, e);
    return dd_make(p, e);
}
__device__ __forceinline__ ddr dd_mul(ddr a, ddr b)
{
    const ddr p = dd_mul_raw(a, b);
    return quick_two_sum(p.hi, p.lo);
}
// a + (unnormalised) p
__device__ __forceinline__ ddr dd_add_raw(ddr a, ddr p)
{
    const ddr s = two_sum(a.hi, p.hi);
    return quick_two_sum(s.hi, __fadd_rn(s.lo, __fadd_rn(a.lo, p.lo)));
}
__device__ __forceinline__ ddr dd_sub_raw(ddr a, ddr p) { return dd_add_raw(a, dd_make(-p.hi, -p.lo)); }
// multiply by a power of two (exact)
__device__ __forceinline__ ddr dd_scale2(ddr a, float s) { return dd_make(__fmul_rn(a.hi, s), __fmul_rn(a.lo, s)); }

__device__ __forceinline__ ddc ddc_add(ddc a, ddc b) { ddc r; r.re = dd_add(a.re, b.re); r.im = dd_add(a.im, b.im); return r; }
__device__ __forceinline__ ddc ddc_sub(ddc a, ddc b) { ddc r; r.re = dd_sub(a.re, b.re); r.im = dd_sub(a.im, b.im); return r; }

// twiddle in ratio form for the double-float butterfly (see Tw in idp_internal.cuh)
struct TwD {
    ddr r, mre, mim;
    int swap, pad;
};

}  // namespace idp
