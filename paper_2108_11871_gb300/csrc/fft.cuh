// CTA-cooperative complex FFT in shared memory (Stockham, natural order in and
// out; one radix-3 stage first when the length is 3 * 2^m, then radix-4
// passes and at most one radix-2 pass), for FP64 (double2) or double-float
// (ddc) elements.
// FP64 arithmetic is the scarce resource on GB300 (about 1/60 of the FP32
// rate), so the FP64 butterfly uses the ratio ("tangent") form of the
// twiddle: 6 FP64 instructions per butterfly instead of 8, and the first two
// stages use no multiplications.  The double-float butterfly runs the same
// schedule on the FP32 pipe.
#pragma once
#include <type_traits>
#include "arith.cuh"

namespace idp {

__device__ __forceinline__ double2 cadd(double2 a, double2 b) { return make_double2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ double2 csub(double2 a, double2 b) { return make_double2(a.x - b.x, a.y - b.y); }

// Double-float twiddles staged in shared memory.  Each 32-byte TwD is kept as
// two 16-byte halves in two planes of L/2 entries, entry m at slot
// m ^ fold(m >> 3), fold being the XOR of the 3-bit groups of its argument.  A
// pass of span Ns reads w^(k s) for eight consecutive k in a quarter-warp (s a
// power of two); with 32-byte entries at their natural places those reads fell
// into the same bank group, up to eight-fold, where the permutation (a
// bijection within every aligned group of eight entries, and linear over XOR,
// so that offsets by a larger power of two keep it) gives eight different ones.
// L / 2 must be a multiple of 8 (TwSwz).
template <int L>
struct TwSwz {
    static constexpr bool ok = (L % 16) == 0;
};
__device__ __forceinline__ int tw_slot(int m)
{
    int x = m >> 3;
    x ^= x >> 3;
    x ^= x >> 6;
    return m ^ (x & 7);
}
template <int L>
__device__ __forceinline__ void tw_stage(TwD *dst, const TwD *__restrict__ src, int tid, int nt)
{
    static_assert(TwSwz<L>::ok, "the twiddle permutation works on groups of eight entries");
    float4 *pa = reinterpret_cast<float4 *>(dst), *pb = pa + L / 2;
    for (int i = tid; i < L / 2; i += nt) {
        const TwD t = src[i];
        const int sl = tw_slot(i);
        pa[sl] = make_float4(t.r.hi, t.r.lo, t.mre.hi, t.mre.lo);
        pb[sl] = make_float4(t.mim.hi, t.mim.lo, __int_as_float(t.swap), 0.f);
    }
}
template <int L, class T>
__device__ __forceinline__ T tw_load(const T *tw, int m)
{
    const float4 *pa = reinterpret_cast<const float4 *>(tw), *pb = pa + L / 2;
    const int sl = tw_slot(m);
    const float4 A = pa[sl], B = pb[sl];
    T t;
    t.r = dd_make(A.x, A.y);
    t.mre = dd_make(A.z, A.w);
    t.mim = dd_make(B.x, B.y);
    t.swap = __float_as_int(B.z);
    t.pad = 0;
    return t;
}

// barrier of the threads that share the buffers: the block, or one warp
template <bool WARP>
__device__ __forceinline__ void fft_sync()
{
    if constexpr (WARP) __syncwarp();
    else __syncthreads();
}

// FFT of LB lines of length L stored contiguously (line stride L) in X;
// Y is scratch of the same size.  Returns the buffer holding the result.
// INV selects e^{+2 pi i jk/L} (unnormalised).  If zero_half, the second
// half of every input line is known to be zero (saves the first stage).
// The NT threads that share X and Y call it with tid = 0..NT-1: the whole block
// (WARP = false; ends with __syncthreads()) or one warp (WARP = true, NT = 32;
// ends with __syncwarp()).  ns0 > 1 (powers of two only): X already holds the
// result of the stages up to span ns0 (the caller fused them into its load).
// TWS: tw is a double-float table staged by tw_stage<L> (planes, permuted slots).
template <class R, int L, int LB, int NT, bool INV, bool WARP = false, bool TWS = false>
__device__ __forceinline__ typename Ar<R>::C *cta_fft_t(typename Ar<R>::C *X, typename Ar<R>::C *Y,
                                                        const typename Ar<R>::T *__restrict__ tw, bool zero_half,
                                                        int tid = -1, int ns0 = 1)
{
    if (tid < 0) tid = threadIdx.x;
    using C = typename Ar<R>::C;
    static_assert(!TWS || (!std::is_same<R, double>::value && TwSwz<L>::ok), "staged twiddles: double-float");
    constexpr int H = L / 2;
    constexpr bool P2 = (L & (L - 1)) == 0;
    int first = ns0;
    if (!P2 && ns0 == 1) {
        // radix-3 stage (lengths 3 * 2^m): y[3j + r] = sum_q x[j + q L/3] w3^{qr}
        constexpr int T = L / 3;
        for (int b = tid; b < LB * T; b += NT) {
            const int line = b / T;
            const int j = b - line * T;
            const C *x = X + line * L;
            C *y = Y + line * L;
            Ar<R>::radix3(x[j], x[j + T], x[j + 2 * T], INV, y[3 * j], y[3 * j + 1], y[3 * j + 2]);
        }
        fft_sync<WARP>();
        C *t = X;
        X = Y;
        Y = t;
        first = 3;
        zero_half = false;
    }
    // radix-4 passes: two radix-2 stages fused in registers, four ratio-form
    // butterflies per four points (the FP64 operation count of the radix-2 form),
    // half the shared-memory round trips and barriers
    int Ns = first;
    constexpr int Q = L / 4;
#pragma unroll 1
    for (; Ns * 4 <= L; Ns <<= 2) {
#pragma unroll
        for (int b = tid; b < LB * Q; b += NT) {
            const int line = b / Q;
            const int j = b - line * Q;
            const C *x = X + line * L;
            C *y = Y + line * L;
            const int k = P2 ? (j & (Ns - 1)) : (j % Ns);
            const C a0 = x[j], a1 = x[j + Q];
            C y0, y1, y2, y3;
            if (Ns == 1) {
                C c0, c1, e0, e1;
                if (zero_half) {
                    c0 = a0; c1 = a0; e0 = a1; e1 = a1;
                } else {
                    const C a2 = x[j + 2 * Q], a3 = x[j + 3 * Q];
                    c0 = Ar<R>::cadd(a0, a2); c1 = Ar<R>::csub(a0, a2);
                    e0 = Ar<R>::cadd(a1, a3); e1 = Ar<R>::csub(a1, a3);
                }
                y0 = Ar<R>::cadd(c0, e0);
                y2 = Ar<R>::csub(c0, e0);
                const C t = INV ? mul_pi(e1) : mul_mi(e1);
                y1 = Ar<R>::cadd(c1, t);
                y3 = Ar<R>::csub(c1, t);
            } else {
                const C a2 = x[j + 2 * Q], a3 = x[j + 3 * Q];
                const int s1 = L / (4 * Ns);
                C c0, c1, e0, e1;
                if constexpr (TWS) {
                    const auto w2 = tw_load<L>(tw, 2 * k * s1);
                    Ar<R>::bfly(a0, a2, w2, c0, c1);
                    Ar<R>::bfly(a1, a3, w2, e0, e1);
                    Ar<R>::bfly(c0, e0, tw_load<L>(tw, k * s1), y0, y2);
                    Ar<R>::bfly(c1, e1, tw_load<L>(tw, (k + Ns) * s1), y1, y3);
                } else {
                    Ar<R>::bfly(a0, a2, tw[2 * k * s1], c0, c1);       // w^2k
                    Ar<R>::bfly(a1, a3, tw[2 * k * s1], e0, e1);
                    Ar<R>::bfly(c0, e0, tw[k * s1], y0, y2);           // w^k
                    Ar<R>::bfly(c1, e1, tw[(k + Ns) * s1], y1, y3);    // -+ i w^k
                }
            }
            const int base = ((j - k) << 2) + k;
            y[base] = y0;
            y[base + Ns] = y1;
            y[base + 2 * Ns] = y2;
            y[base + 3 * Ns] = y3;
        }
        fft_sync<WARP>();
        C *t = X;
        X = Y;
        Y = t;
        zero_half = false;
    }
    if (Ns < L) {   // one radix-2 stage left
#pragma unroll
        for (int b = tid; b < LB * H; b += NT) {
            const int line = b / H;
            const int j = b - line * H;
            const C *x = X + line * L;
            C *y = Y + line * L;
            const int k = P2 ? (j & (Ns - 1)) : (j % Ns);
            const int o = ((j - k) << 1) + k;
            const C a = x[j];
            C A, B;
            if (Ns == 1) {
                if (zero_half) {
                    A = a;
                    B = a;
                } else {
                    const C c = x[j + H];
                    A = Ar<R>::cadd(a, c);
                    B = Ar<R>::csub(a, c);
                }
            } else {
                if constexpr (TWS) Ar<R>::bfly(a, x[j + H], tw_load<L>(tw, k * (L / (2 * Ns))), A, B);
                else Ar<R>::bfly(a, x[j + H], tw[k * (L / (2 * Ns))], A, B);
            }
            y[o] = A;
            y[o + Ns] = B;
        }
        fft_sync<WARP>();
        C *t = X;
        X = Y;
        Y = t;
    }
    return X;
}

// FP64 form used by the boundary kernels
template <int L, int LB, int NT, bool INV>
__device__ __forceinline__ double2 *cta_fft(double2 *X, double2 *Y, const Tw *__restrict__ tw, bool zero_half)
{
    return cta_fft_t<double, L, LB, NT, INV>(X, Y, tw, zero_half);
}

}  // namespace idp
