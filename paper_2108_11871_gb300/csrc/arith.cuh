// Scalar and complex arithmetic used by the transform kernels, for two real
// types: double (FP64 pipe) and ddr (double-float on the FP32 pipe, dd.cuh).
// The double versions are exactly the FP64 operations the kernels always used.
#pragma once
#include "dd.cuh"
#include "idp_internal.cuh"

namespace idp {

template <class R>
struct Ar;

template <>
struct Ar<double> {
    using C = double2;
    using T = Tw;
    static __device__ __forceinline__ double add(double a, double b) { return a + b; }
    static __device__ __forceinline__ double sub(double a, double b) { return a - b; }
    // a*b + c
    static __device__ __forceinline__ double fma(double a, double b, double c) { return ::fma(a, b, c); }
    static __device__ __forceinline__ double mul(double a, double b) { return a * b; }
    // a*b - c*d and a*b + c*d as the FP64 kernels write them
    static __device__ __forceinline__ double mul_sub(double a, double b, double c, double d) { return ::fma(a, b, -c * d); }
    static __device__ __forceinline__ double mul_add(double a, double b, double c, double d) { return ::fma(a, b, c * d); }
    static __device__ __forceinline__ double times4(double a) { return 4.0 * a; }
    static __device__ __forceinline__ double neg(double a) { return -a; }
    static __device__ __forceinline__ double times2(double a) { return 2.0 * a; }
    static __device__ __forceinline__ double zero() { return 0.0; }
    static __device__ __forceinline__ double shfl_up(double v, int d, int w) { return __shfl_up_sync(0xffffffffu, v, d, w); }
    static __device__ __forceinline__ double2 cmake(double a, double b) { return make_double2(a, b); }
    static __device__ __forceinline__ double re(double2 c) { return c.x; }
    static __device__ __forceinline__ double im(double2 c) { return c.y; }
    static __device__ __forceinline__ double2 cadd(double2 a, double2 b) { return make_double2(a.x + b.x, a.y + b.y); }
    static __device__ __forceinline__ double2 csub(double2 a, double2 b) { return make_double2(a.x - b.x, a.y - b.y); }
    // 3-point DFT: y0 = a0 + t, y1,2 = a0 - t/2 -+ i s3 (a1 - a2) (forward; +- for inverse),
    // t = a1 + a2, s3 = sqrt(3)/2
    static __device__ __forceinline__ void radix3(double2 a0, double2 a1, double2 a2, bool inv, double2 &y0,
                                                  double2 &y1, double2 &y2)
    {
        const double s3 = inv ? -0.86602540378443864676 : 0.86602540378443864676;
        const double tr = a1.x + a2.x, ti = a1.y + a2.y;
        const double dr = a1.x - a2.x, di = a1.y - a2.y;
        y0 = make_double2(a0.x + tr, a0.y + ti);
        const double mr = ::fma(-0.5, tr, a0.x), mi = ::fma(-0.5, ti, a0.y);
        y1 = make_double2(::fma(s3, di, mr), ::fma(-s3, dr, mi));
        y2 = make_double2(::fma(-s3, di, mr), ::fma(s3, dr, mi));
    }
    // A = a + w c, B = a - w c with w in ratio form
    static __device__ __forceinline__ void bfly(double2 a, double2 c, const Tw &w, double2 &A, double2 &B)
    {
        const double P = w.swap ? c.y : c.x;
        const double Q = w.swap ? c.x : c.y;
        const double u = ::fma(-w.r, Q, P);
        const double v = ::fma(w.r, P, Q);
        A.x = ::fma(w.mre, u, a.x);
        B.x = ::fma(-w.mre, u, a.x);
        A.y = ::fma(w.mim, v, a.y);
        B.y = ::fma(-w.mim, v, a.y);
    }
};

template <>
struct Ar<ddr> {
    using C = ddc;
    using T = TwD;
    static __device__ __forceinline__ ddr add(ddr a, ddr b) { return dd_add(a, b); }
    static __device__ __forceinline__ ddr sub(ddr a, ddr b) { return dd_sub(a, b); }
    static __device__ __forceinline__ ddr fma(ddr a, ddr b, ddr c) { return dd_add_raw(c, dd_mul_raw(a, b)); }
    static __device__ __forceinline__ ddr mul(ddr a, ddr b) { return dd_mul(a, b); }
    static __device__ __forceinline__ ddr mul_sub(ddr a, ddr b, ddr c, ddr d)
    {
        return dd_sub_raw(dd_mul(a, b), dd_mul_raw(c, d));
    }
    static __device__ __forceinline__ ddr mul_add(ddr a, ddr b, ddr c, ddr d)
    {
        return dd_add_raw(dd_mul(a, b), dd_mul_raw(c, d));
    }
    static __device__ __forceinline__ ddr times4(ddr a) { return dd_scale2(a, 4.0f); }
    static __device__ __forceinline__ ddr neg(ddr a) { return dd_neg(a); }
    static __device__ __forceinline__ ddr times2(ddr a) { return dd_scale2(a, 2.0f); }
    static __device__ __forceinline__ ddr zero() { return dd_make(0.f, 0.f); }
    static __device__ __forceinline__ ddr shfl_up(ddr v, int d, int w)
    {
        return dd_make(__shfl_up_sync(0xffffffffu, v.hi, d, w), __shfl_up_sync(0xffffffffu, v.lo, d, w));
    }
    static __device__ __forceinline__ ddc cmake(ddr a, ddr b) { ddc c; c.re = a; c.im = b; return c; }
    static __device__ __forceinline__ ddr re(ddc c) { return c.re; }
    static __device__ __forceinline__ ddr im(ddc c) { return c.im; }
    static __device__ __forceinline__ ddc cadd(ddc a, ddc b) { return ddc_add(a, b); }
    static __device__ __forceinline__ ddc csub(ddc a, ddc b) { return ddc_sub(a, b); }
    static __device__ __forceinline__ void radix3(ddc a0, ddc a1, ddc a2, bool inv, ddc &y0, ddc &y1, ddc &y2)
    {
        // sqrt(3)/2 as a double-float pair
        const ddr s3 = inv ? dd_make(-0.866025388240814208984375f, -1.5543625e-08f)
                           : dd_make(0.866025388240814208984375f, 1.5543625e-08f);
        const ddr tr = dd_add(a1.re, a2.re), ti = dd_add(a1.im, a2.im);
        const ddr dr = dd_sub(a1.re, a2.re), di = dd_sub(a1.im, a2.im);
        y0.re = dd_add(a0.re, tr);
        y0.im = dd_add(a0.im, ti);
        const ddr mr = dd_sub(a0.re, dd_scale2(tr, 0.5f)), mi = dd_sub(a0.im, dd_scale2(ti, 0.5f));
        const ddr pr = dd_mul_raw(s3, di), pi = dd_mul_raw(s3, dr);
        y1.re = dd_add_raw(mr, pr);
        y1.im = dd_sub_raw(mi, pi);
        y2.re = dd_sub_raw(mr, pr);
        y2.im = dd_add_raw(mi, pi);
    }
    static __device__ __forceinline__ void bfly(ddc a, ddc c, const TwD &w, ddc &A, ddc &B)
    {
        const ddr P = w.swap ? c.im : c.re;
        const ddr Q = w.swap ? c.re : c.im;
        const ddr u = dd_sub_raw(P, dd_mul_raw(w.r, Q));
        const ddr v = dd_add_raw(Q, dd_mul_raw(w.r, P));
        const ddr mu = dd_mul_raw(w.mre, u);
        const ddr mv = dd_mul_raw(w.mim, v);
        A.re = dd_add_raw(a.re, mu);
        B.re = dd_sub_raw(a.re, mu);
        A.im = dd_add_raw(a.im, mv);
        B.im = dd_sub_raw(a.im, mv);
    }
};

// complex multiply by i or -i (exact)
template <class C>
__device__ __forceinline__ C mul_mi(C c);   // -i c
template <>
__device__ __forceinline__ double2 mul_mi(double2 c) { return make_double2(c.y, -c.x); }
template <>
__device__ __forceinline__ ddc mul_mi(ddc c) { ddc r; r.re = c.im; r.im = dd_neg(c.re); return r; }
template <class C>
__device__ __forceinline__ C mul_pi(C c);   // +i c
template <>
__device__ __forceinline__ double2 mul_pi(double2 c) { return make_double2(-c.y, c.x); }
template <>
__device__ __forceinline__ ddc mul_pi(ddc c) { ddc r; r.re = dd_neg(c.im); r.im = c.re; return r; }

}  // namespace idp
