// Sine-transform pass (section 3, eqs. rhoSinSeries / phiStarSoln2D; section 5,
// the sine eigenvectors of the compact operator): for every line of an
// interior box along one axis, U = 4 S x with S_{k,i} = sin(pi k i / M),
// k, i = 1..M-1, followed by a pointwise epilogue.
//
// Algorithm per line (M = 2K):
//   y'_j = 2 sin(pi j/M)(x_j + x_{M-j}) + (x_j - x_{M-j}),  y'_K = 4 x_K, y'_0 = 0
//   Z    = FFT_K(y'_{2m} + i y'_{2m+1})                    (complex, length K)
//   T_k  = (Z_k + conj Z_{K-k}) - i e^{-2 pi i k/M} (Z_k - conj Z_{K-k})
//   U_{2k} = -Im T_k,   U_{2k+1} = U_{2k-1} + Re T_k,   U_1 = Re Z_0 + Im Z_0
// (the real-FFT form of the DST-I; T = 4 Y where Y is the real FFT of y).
#include "fft.cuh"

namespace idp {

namespace {

constexpr int NT = 256;

template <int K>
struct DstCfg {
    static constexpr int M = 2 * K;
    static constexpr int N = M - 1;
    // lines per block: 2 buffers x LB x M doubles (32 KB for M >= 128), at
    // least 8 lines so that the scan groups fit a warp
    static constexpr int LB0 = (2048 / M) > 32 ? 32 : (2048 / M);
    static constexpr int LB = LB0 < 8 ? 8 : LB0;
    static constexpr int G = NT / LB;             // threads per line in the scan
    static constexpr int C = (K / G) > 0 ? K / G : 1;  // scan elements per thread
};

template <int K>
__global__ void __launch_bounds__(NT) dst_pass_kernel(const DstPass a)
{
    using Cfg = DstCfg<K>;
    constexpr int M = Cfg::M, N = Cfg::N, LB = Cfg::LB;
    extern __shared__ double2 smem[];
    double2 *bufA = smem;            // LB * K complex
    double2 *bufB = smem + LB * K;   // LB * K complex

    // line (u, v) coordinates: the two non-transform axes, v fastest
    int nv, nu;
    int64_t isu, isv, ise, osu, osv, ose, asu = 0, asv = 0, ase = 0, tsu, tsv, tse;
    const int64_t t0 = (int64_t)a.n1 * a.n2, t1 = a.n2;
    if (a.axis == 2) {
        nu = a.n0; nv = a.n1;
        isu = a.in.s0; isv = a.in.s1; ise = a.in.s2;
        osu = a.out.s0; osv = a.out.s1; ose = a.out.s2;
        asu = a.add.s0; asv = a.add.s1; ase = a.add.s2;
        tsu = t0; tsv = t1; tse = 1;
    } else if (a.axis == 1) {
        nu = a.n0; nv = a.n2;
        isu = a.in.s0; isv = a.in.s2; ise = a.in.s1;
        osu = a.out.s0; osv = a.out.s2; ose = a.out.s1;
        asu = a.add.s0; asv = a.add.s2; ase = a.add.s1;
        tsu = t0; tsv = 1; tse = t1;
    } else {
        nu = a.n1; nv = a.n2;
        isu = a.in.s1; isv = a.in.s2; ise = a.in.s0;
        osu = a.out.s1; osv = a.out.s2; ose = a.out.s0;
        asu = a.add.s1; asv = a.add.s2; ase = a.add.s0;
        tsu = t1; tsv = 1; tse = t0;
    }
    const int u = blockIdx.y;
    const int v0 = blockIdx.x * LB;
    const int nl = min(LB, nv - v0);
    const bool contig = (a.axis == 2);

    // 1. load raw lines into bufB viewed as double[LB][M] (entries 0..N-1)
    double *raw = reinterpret_cast<double *>(bufB);
    const double *inb = a.in.p + (int64_t)u * isu + (int64_t)v0 * isv;
    for (int f = threadIdx.x; f < LB * N; f += NT) {
        int l, e;
        if (contig) { l = f / N; e = f - l * N; }
        else { e = f / LB; l = f - e * LB; }
        double x = 0.0;
        if (l < nl) x = inb[(int64_t)l * isv + (int64_t)e * ise];
        raw[l * M + e] = x;
    }
    __syncthreads();

    // 2. pre-processing into bufA viewed as double[LB][M] (zf[j] = y'_j)
    double *zf = reinterpret_cast<double *>(bufA);
    for (int f = threadIdx.x; f < LB * K; f += NT) {
        const int l = f / K;
        const int j = f - l * K;
        const double *xl = raw + l * M;   // x_i at xl[i-1]
        double *zl = zf + l * M;
        if (j == 0) {
            zl[0] = 0.0;
            zl[K] = 4.0 * xl[K - 1];
        } else {
            const double xa = xl[j - 1], xb = xl[M - j - 1];
            const double s = a.sin2[j];
            const double p = xa + xb, m = xa - xb;
            zl[j] = fma(s, p, m);
            zl[M - j] = fma(s, p, -m);
        }
    }
    __syncthreads();

    // 3. complex FFT of length K
    double2 *Z = cta_fft<K, LB, NT, false>(bufA, bufB, a.tw, false);
    double *o = reinterpret_cast<double *>(Z == bufA ? bufB : bufA);   // double[LB][M]

    // 4. post-processing: even outputs final, odd slots get Re T_k
    for (int f = threadIdx.x; f < LB * (K / 2); f += NT) {
        const int l = f / (K / 2);
        const int k = f - l * (K / 2) + 1;      // 1..K/2
        const double2 *zl = Z + l * K;
        double *ol = o + l * M;
        const double2 zk = zl[k], zc = zl[K - k];
        const double Er = zk.x + zc.x, Ei = zk.y - zc.y;
        const double Or = zk.x - zc.x, Oi = zk.y + zc.y;
        const double2 w = a.half[k];
        const double Pr = fma(w.x, Or, -w.y * Oi);
        const double Pi = fma(w.x, Oi, w.y * Or);
        ol[2 * k - 1] = Pr - Ei;
        ol[2 * (K - k) - 1] = Ei + Pr;
        ol[2 * k] = Er + Pi;
        ol[2 * (K - k)] = Er - Pi;
        if (k == 1) ol[0] = zl[0].x + zl[0].y;
    }
    __syncthreads();

    // 5. prefix sum over the odd slots o[2k], k = 0..K-1
    {
        constexpr int G = Cfg::G, C = Cfg::C;
        const int l = threadIdx.x / G;
        const int g = threadIdx.x - l * G;
        double vals[C];
        double run = 0.0;
        if (g * C < K) {
#pragma unroll
            for (int c = 0; c < C; ++c) {
                run += o[l * M + 2 * (g * C + c)];
                vals[c] = run;
            }
        }
        // inclusive scan of the group totals (groups of G consecutive lanes)
        double incl = run;
#pragma unroll
        for (int dd = 1; dd < G; dd <<= 1) {
            const double nb = __shfl_up_sync(0xffffffffu, incl, dd, G);
            if (g >= dd) incl += nb;
        }
        const double off = incl - run;
        if (g * C < K) {
#pragma unroll
            for (int c = 0; c < C; ++c) o[l * M + 2 * (g * C + c)] = vals[c] + off;
        }
    }
    __syncthreads();

    // 6. epilogue and store
    double *outb = a.out.p + (int64_t)u * osu + (int64_t)v0 * osv;
    const double *tabb = a.tab ? a.tab + (int64_t)u * tsu + (int64_t)v0 * tsv : nullptr;
    const double *addb = a.add.p ? a.add.p + (int64_t)u * asu + (int64_t)v0 * asv : nullptr;
    for (int f = threadIdx.x; f < LB * N; f += NT) {
        int l, e;
        if (contig) { l = f / N; e = f - l * N; }
        else { e = f / LB; l = f - e * LB; }
        if (l >= nl) continue;
        double y = o[l * M + e];
        if (tabb) {
            const double t = tabb[(int64_t)l * tsv + (int64_t)e * tse];
            if (addb) y = fma(t, y, addb[(int64_t)l * asv + (int64_t)e * ase]);
            else y = t * y;
        } else if (addb) {
            y += addb[(int64_t)l * asv + (int64_t)e * ase];
        }
        outb[(int64_t)l * osv + (int64_t)e * ose] = y;
    }
}

template <int K>
cudaError_t launch_k(const DstPass &a, cudaStream_t st)
{
    using Cfg = DstCfg<K>;
    static_assert(Cfg::G <= 32, "scan group must fit a warp");
    static_assert(Cfg::LB * Cfg::G == NT, "every thread belongs to one scan group");
    const size_t sm = 2 * sizeof(double2) * Cfg::LB * K;
    int nu, nv;
    if (a.axis == 2) { nu = a.n0; nv = a.n1; }
    else if (a.axis == 1) { nu = a.n0; nv = a.n2; }
    else { nu = a.n1; nv = a.n2; }
    dim3 grid((nv + Cfg::LB - 1) / Cfg::LB, nu);
    dst_pass_kernel<K><<<grid, NT, sm, st>>>(a);
    return cudaGetLastError();
}

template <int K>
cudaError_t attr_k()
{
    using Cfg = DstCfg<K>;
    const int sm = (int)(2 * sizeof(double2) * Cfg::LB * K);
    return cudaFuncSetAttribute(dst_pass_kernel<K>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm);
}

}  // namespace

cudaError_t dst_set_attributes()
{
    cudaError_t e;
    if ((e = attr_k<8>()) != cudaSuccess) return e;
    if ((e = attr_k<16>()) != cudaSuccess) return e;
    if ((e = attr_k<32>()) != cudaSuccess) return e;
    if ((e = attr_k<64>()) != cudaSuccess) return e;
    if ((e = attr_k<128>()) != cudaSuccess) return e;
    return attr_k<256>();
}

cudaError_t launch_dst_pass(const DstPass &a, cudaStream_t st)
{
    switch (a.M) {
    case 16: return launch_k<8>(a, st);
    case 32: return launch_k<16>(a, st);
    case 64: return launch_k<32>(a, st);
    case 128: return launch_k<64>(a, st);
    case 256: return launch_k<128>(a, st);
    case 512: return launch_k<256>(a, st);
    default: return cudaErrorInvalidValue;
    }
}

}  // namespace idp
