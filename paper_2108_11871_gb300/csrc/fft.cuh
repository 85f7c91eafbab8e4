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
#include "arith.cuh"

namespace idp {

__device__ __forceinline__ double2 cadd(double2 a, double2 b) { return make_double2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ double2 csub(double2 a, double2 b) { return make_double2(a.x - b.x, a.y - b.y); }

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
template <class R, int L, int LB, int NT, bool INV, bool WARP = false>
__device__ __forceinline__ typename Ar<R>::C *cta_fft_t(typename Ar<R>::C *X, typename Ar<R>::C *Y,
                                                        const typename Ar<R>::T *__restrict__ tw, bool zero_half,
                                                        int tid = -1, int ns0 = 1)
{
    if (tid < 0) tid = threadIdx.x;
    using C = typename Ar<R>::C;
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
                Ar<R>::bfly(a0, a2, tw[2 * k * s1], c0, c1);       // w^2k
                Ar<R>::bfly(a1, a3, tw[2 * k * s1], e0, e1);
                Ar<R>::bfly(c0, e0, tw[k * s1], y0, y2);           // w^k
                Ar<R>::bfly(c1, e1, tw[(k + Ns) * s1], y1, y3);    // -+ i w^k
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
                Ar<R>::bfly(a, x[j + H], tw[k * (L / (2 * Ns))], A, B);
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
