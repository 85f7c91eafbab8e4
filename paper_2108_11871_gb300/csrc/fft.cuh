// CTA-cooperative FP64 complex FFT in shared memory (radix-2 Stockham,
// natural order in and out).  FP64 arithmetic is the scarce resource on
// GB300 (about 1/60 of the FP32 rate), so the butterfly uses the ratio
// ("tangent") form of the twiddle: 6 FP64 instructions per butterfly
// instead of 8, and the first two stages use no multiplications.
#pragma once
#include "idp_internal.cuh"

namespace idp {

__device__ __forceinline__ double2 cadd(double2 a, double2 b) { return make_double2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ double2 csub(double2 a, double2 b) { return make_double2(a.x - b.x, a.y - b.y); }

// FFT of LB lines of length L stored contiguously (line stride L) in X;
// Y is scratch of the same size.  Returns the buffer holding the result.
// INV selects e^{+2 pi i jk/L} (unnormalised).  If zero_half, the second
// half of every input line is known to be zero (saves the first stage).
// All NT threads of the block must call it; it ends with __syncthreads().
template <int L, int LB, int NT, bool INV>
__device__ __forceinline__ double2 *cta_fft(double2 *X, double2 *Y, const Tw *__restrict__ tw,
                                            bool zero_half)
{
    constexpr int H = L / 2;
#pragma unroll 1
    for (int Ns = 1; Ns < L; Ns <<= 1) {
        for (int b = threadIdx.x; b < LB * H; b += NT) {
            const int line = b / H;
            const int j = b - line * H;
            const double2 *x = X + line * L;
            double2 *y = Y + line * L;
            const int k = j & (Ns - 1);
            const int o = ((j - k) << 1) + k;
            const double2 a = x[j];
            double2 A, B;
            if (Ns == 1) {
                if (zero_half) {
                    A = a;
                    B = a;
                } else {
                    const double2 c = x[j + H];
                    A = cadd(a, c);
                    B = csub(a, c);
                }
            } else if (Ns == 2) {
                const double2 c = x[j + H];
                // w = 1 (k = 0) or -i (forward) / +i (inverse) (k = 1)
                double2 t;
                if (INV)
                    t = k ? make_double2(-c.y, c.x) : c;
                else
                    t = k ? make_double2(c.y, -c.x) : c;
                A = cadd(a, t);
                B = csub(a, t);
            } else {
                const double2 c = x[j + H];
                const Tw w = tw[k * (L / (2 * Ns))];
                const double P = w.swap ? c.y : c.x;
                const double Q = w.swap ? c.x : c.y;
                const double u = fma(-w.r, Q, P);
                const double v = fma(w.r, P, Q);
                A.x = fma(w.mre, u, a.x);
                B.x = fma(-w.mre, u, a.x);
                A.y = fma(w.mim, v, a.y);
                B.y = fma(-w.mim, v, a.y);
            }
            y[o] = A;
            y[o + Ns] = B;
        }
        __syncthreads();
        double2 *t = X;
        X = Y;
        Y = t;
    }
    return X;
}

}  // namespace idp
