// CTA-cooperative complex FFT in shared memory (Stockham, natural order in and
// out; one radix-3 stage first when the length is 3 * 2^m, radix-2 stages
// otherwise), for FP64 (double2) or double-float (ddc) elements.
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

// FFT of LB lines of length L stored contiguously (line stride L) in X;
// Y is scratch of the same size.  Returns the buffer holding the result.
// INV selects e^{+2 pi i jk/L} (unnormalised).  If zero_half, the second
// half of every input line is known to be zero (saves the first stage).
// All NT threads of the block must call it; it ends with __syncthreads().
template <class R, int L, int LB, int NT, bool INV>
__device__ __forceinline__ typename Ar<R>::C *cta_fft_t(typename Ar<R>::C *X, typename Ar<R>::C *Y,
                                                        const typename Ar<R>::T *__restrict__ tw, bool zero_half)
{
    using C = typename Ar<R>::C;
    constexpr int H = L / 2;
    constexpr bool P2 = (L & (L - 1)) == 0;
    int first = 1;
    if (!P2) {
        // radix-3 stage (lengths 3 * 2^m): y[3j + r] = sum_q x[j + q L/3] w3^{qr}
        constexpr int T = L / 3;
        for (int b = threadIdx.x; b < LB * T; b += NT) {
            const int line = b / T;
            const int j = b - line * T;
            const C *x = X + line * L;
            C *y = Y + line * L;
            Ar<R>::radix3(x[j], x[j + T], x[j + 2 * T], INV, y[3 * j], y[3 * j + 1], y[3 * j + 2]);
        }
        __syncthreads();
        C *t = X;
        X = Y;
        Y = t;
        first = 3;
        zero_half = false;
    }
#pragma unroll 1
    for (int Ns = first; Ns < L; Ns <<= 1) {
#pragma unroll
        for (int b = threadIdx.x; b < LB * H; b += NT) {
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
            } else if (Ns == 2) {
                const C c = x[j + H];
                // w = 1 (k = 0) or -i (forward) / +i (inverse) (k = 1)
                const C t = k ? (INV ? mul_pi(c) : mul_mi(c)) : c;
                A = Ar<R>::cadd(a, t);
                B = Ar<R>::csub(a, t);
            } else {
                const C c = x[j + H];
                Ar<R>::bfly(a, c, tw[k * (L / (2 * Ns))], A, B);
            }
            y[o] = A;
            y[o + Ns] = B;
        }
        __syncthreads();
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
