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

struct __align__(8) ddr {
    float hi, lo;
};
struct __align__(16) ddc {
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

namespace idp {

// FP64 <-> double-float conversions with integer operations only (the FP64
// pipe is the scarce unit, and conversions F2F run on it).
//   hi = x with the low 29 mantissa bits cleared (exact as FP32 if the
//        exponent is in FP32 range), lo = the cleared bits as FP32 (rounded to
//        24 bits).  |x| < 2^-126 gives (0, 0); lo underflows gracefully for
//        |x| < 2^-74.  Relative error at most 2^-48.
__device__ __forceinline__ ddr dd_from_bits(double x)
{
    const unsigned long long b = (unsigned long long)__double_as_longlong(x);
    const unsigned int hiw = (unsigned int)(b >> 32), low = (unsigned int)b;
    const int e = (int)((hiw >> 20) & 0x7FF) - 1023;
    if (e < -126) return dd_make(0.f, 0.f);
    const unsigned int sign = hiw & 0x80000000u;
    // top 23 mantissa bits: 20 from the high word, 3 from the low word
    const unsigned int m23 = ((hiw & 0xFFFFFu) << 3) | (low >> 29);
    const float hi = __int_as_float((int)(sign | ((unsigned int)(e + 127) << 23) | m23));
    // remaining 29 bits, value rest * 2^(e-52)
    const unsigned int rest = low & 0x1FFFFFFFu;
    // exact FP32 of the two parts of rest (magic-number conversion), then one rounding
    const float r_lo = __fsub_rn(__int_as_float(0x4B000000 | (rest & 0x7FFFFFu)), 8388608.0f);
    const float r_hi = __fsub_rn(__int_as_float(0x4B000000 | (rest >> 23)), 8388608.0f);
    const float rf = __fmaf_rn(r_hi, 8388608.0f, r_lo);
    const int se = e - 52 + 127;
    float lo = 0.f;
    if (se > 0) lo = __fmul_rn(rf, __int_as_float(se << 23));
    else if (se > -23) lo = __fmul_rn(__fmul_rn(rf, __int_as_float((se + 24) << 23)), 5.9604645e-8f);  // 2^-24
    lo = sign ? -lo : lo;
    return dd_make(hi, lo);
}

// FP32 -> FP64 by bits (normal or zero inputs; FP32 denormals flush to 0)
__device__ __forceinline__ double f2d_bits(float f)
{
    const unsigned int u = (unsigned int)__float_as_int(f);
    const unsigned int ex = (u >> 23) & 0xFF;
    if (ex == 0) return 0.0;
    const unsigned int sign = u & 0x80000000u;
    const unsigned int hiw = sign | ((ex - 127 + 1023) << 20) | ((u & 0x7FFFFFu) >> 3);
    const unsigned int low = (u & 7u) << 29;
    return __hiloint2double((int)hiw, (int)low);
}

// hi + lo as FP64: two bit conversions and one FP64 addition
__device__ __forceinline__ double dd_to_bits(ddr a) { return f2d_bits(a.hi) + f2d_bits(a.lo); }

}  // namespace idp
