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
#include <type_traits>

#include "fft.cuh"

namespace idp {

namespace {

constexpr int NT = 256;

template <int K, int LBO = 0, int NTB = NT>
struct DstCfg {
    static constexpr int M = 2 * K;
    static constexpr int N = M - 1;
    // lines per block: 2 buffers x LB x M reals (32 KB for M >= 128), at
    // least 8 lines so that the scan groups fit a warp; LBO = 8 gives the
    // minimum (more blocks for small launches)
    static constexpr int LBr = (2048 / M) > 32 ? 32 : (2048 / M);
    // a power of two (so that LB * G = 256)
    static constexpr int LB0 = LBr >= 32 ? 32 : LBr >= 16 ? 16 : LBr >= 8 ? 8 : 4;
    static constexpr int LB = LBO ? LBO : (LB0 < 8 ? 8 : LB0);
    static constexpr int T = NTB;                 // threads per block
    static constexpr int G = T / LB;              // threads per line in the scan
    static constexpr int C = (K + G - 1) / G;     // scan elements per thread (the last ones guarded)
};

// element access for the two storage forms of a real value: FP64, or a
// double-float pair (the DD kernels keep intermediates in that form)
template <class R>
struct Io;
template <>
struct Io<double> {
    static __device__ __forceinline__ double ld(const void *p, int64_t i, int) { return reinterpret_cast<const double *>(p)[i]; }
    static __device__ __forceinline__ void st(void *p, int64_t i, double v, int) { reinterpret_cast<double *>(p)[i] = v; }
};
template <>
struct Io<ddr> {
    static __device__ __forceinline__ ddr ld(const void *p, int64_t i, int dd)
    {
        if (dd) return reinterpret_cast<const ddr *>(p)[i];
        return dd_from_bits(reinterpret_cast<const double *>(p)[i]);
    }
    static __device__ __forceinline__ void st(void *p, int64_t i, ddr v, int dd)
    {
        if (dd) reinterpret_cast<ddr *>(p)[i] = v;
        else reinterpret_cast<double *>(p)[i] = dd_to_bits(v);
    }
};

// 4 x, exact: for a normal FP64 value by adding 2 to the exponent (integer
// pipe; FP64 issue is scarce and this runs on one lane per line), otherwise by
// the multiplication
__device__ __forceinline__ double times4_exact(double x)
{
    const long long b = __double_as_longlong(x);
    const int e = (int)((b >> 52) & 0x7ff);
    if (e >= 1 && e <= 2044) return __longlong_as_double(b + (2LL << 52));
    return x * 4.0;
}
__device__ __forceinline__ ddr times4_exact(ddr x) { return Ar<ddr>::times4(x); }

template <class R>
struct Tabs;
template <>
struct Tabs<double> {
    static __device__ __forceinline__ const Tw *tw(const DstPass &a) { return a.tw; }
    static __device__ __forceinline__ double2 half(const DstPass &a, int k) { return a.half[k]; }
    static __device__ __forceinline__ double sin2(const DstPass &a, int j) { return a.sin2[j]; }
};
template <>
struct Tabs<ddr> {
    static __device__ __forceinline__ const TwD *tw(const DstPass &a) { return a.twd; }
    static __device__ __forceinline__ ddc half(const DstPass &a, int k) { return a.halfd[k]; }
    static __device__ __forceinline__ ddr sin2(const DstPass &a, int j) { return a.sin2d[j]; }
};

// strides of a view along the line (u, v) coordinates and the element index e
// of a pass along `axis` (u, v = the other two axes in order)
__device__ __forceinline__ void view_strides(const View3 &w, int axis, int64_t &su, int64_t &sv, int64_t &se)
{
    if (axis == 2) { su = w.s0; sv = w.s1; se = w.s2; }
    else if (axis == 1) { su = w.s0; sv = w.s2; se = w.s1; }
    else { su = w.s1; sv = w.s2; se = w.s0; }
}

template <class R, int K, int LBO, int NTB>
__global__ void __launch_bounds__(NTB) dst_pass_kernel(const DstPass a)
{
    pdl_enter();
    using Cfg = DstCfg<K, LBO, NTB>;
    constexpr int NT = NTB;
    using A = Ar<R>;
    using Cx = typename A::C;
    constexpr int M = Cfg::M, N = Cfg::N, LB = Cfg::LB;
    extern __shared__ double2 smem_raw[];
    Cx *bufA = reinterpret_cast<Cx *>(smem_raw);   // LB * K complex
    Cx *bufB = bufA + LB * K;                      // LB * K complex
    // the FFT's K / 2 twiddles, copied into shared memory once (read in every pass; from
    // the global table they are long-scoreboard loads); visible after the first barrier
    using TwT = typename Ar<R>::T;
    static_assert(sizeof(TwT) <= 32, "the shared-memory size counts 32 bytes per twiddle");
    TwT *twsm = reinterpret_cast<TwT *>(bufB + LB * K);
    // (double-float: in the bank-spread planes of tw_stage)
    constexpr bool TWS = !std::is_same<R, double>::value && TwSwz<K>::ok;
    if constexpr (TWS) {
        tw_stage<K>(twsm, Tabs<R>::tw(a), threadIdx.x, NT);
    } else {
        const TwT *tg = Tabs<R>::tw(a);
        for (int i = threadIdx.x; i < K / 2; i += NT) twsm[i] = tg[i];
    }

    // line (u, v) coordinates: the two non-transform axes, v fastest.  The
    // strides are taken from the parameters where they are used, so that none
    // of them stays live across the FFT.
    const int nv = a.axis == 2 ? a.n1 : a.n2;
    const int u = blockIdx.y;
    const int v0 = blockIdx.x * LB;
    const int nl = min(LB, nv - v0);
    const bool contig = (a.axis == 2);

    // 1. load and pre-process in one step: the thread that forms y'_j and
    //    y'_{M-j} loads x_j and x_{M-j} itself (consecutive threads take
    //    consecutive j of a contiguous line, or consecutive lines), into bufA
    //    viewed as R[LB][M] (zf[j] = y'_j); lines past the end give zeros
    R *zf = reinterpret_cast<R *>(bufA);
    int64_t isu, isv, ise;
    view_strides(a.in, a.axis, isu, isv, ise);
    const int64_t inb = (int64_t)u * isu + (int64_t)v0 * isv;
    // all loads of the thread first (their latencies overlap), then the pre-pass
    // arithmetic and the shared-memory stores
    constexpr int IT = (LB * K + NT - 1) / NT;
    R xa[IT], xb[IT], sv[IT];
#pragma unroll
    for (int i = 0; i < IT; ++i) {
        const int f = threadIdx.x + i * NT;
        xa[i] = A::zero();
        xb[i] = A::zero();
        sv[i] = A::zero();
        if (f < LB * K) {
            int l, j;
            if (contig) { l = f / K; j = f - l * K; }
            else { j = f / LB; l = f - j * LB; }
            const int64_t lb = inb + (int64_t)l * isv;   // x_i at element i-1 of the line
            if (j == 0) {
                if (l < nl) xa[i] = Io<R>::ld(a.in.p, lb + (int64_t)(K - 1) * ise, a.in_dd);
            } else {
                if (l < nl) {
                    xa[i] = Io<R>::ld(a.in.p, lb + (int64_t)(j - 1) * ise, a.in_dd);
                    xb[i] = Io<R>::ld(a.in.p, lb + (int64_t)(M - j - 1) * ise, a.in_dd);
                }
                sv[i] = Tabs<R>::sin2(a, j);
            }
        }
    }
#pragma unroll
    for (int i = 0; i < IT; ++i) {
        const int f = threadIdx.x + i * NT;
        if (f >= LB * K) break;
        int l, j;
        if (contig) { l = f / K; j = f - l * K; }
        else { j = f / LB; l = f - j * LB; }
        R *zl = zf + l * M;
        if (j == 0) {
            zl[0] = A::zero();
            zl[K] = l < nl ? times4_exact(xa[i]) : A::zero();
        } else {
            const R p = A::add(xa[i], xb[i]), m = A::sub(xa[i], xb[i]);
            zl[j] = A::fma(sv[i], p, m);
            zl[M - j] = A::fma(sv[i], p, A::neg(m));
        }
    }
    __syncthreads();

    // 3. complex FFT of length K.  FP64: by each warp on its own lines (barriers of
    //    one warp between the passes, measured 6 % faster at M = 256 and 512) where
    //    that keeps every lane busy in the radix-4 passes; else, and in double-float
    //    (measured 2 % slower that way), by the block
    constexpr int NW = NT / 32;
    constexpr bool WFFT = std::is_same<R, double>::value && (LB % NW == 0) && (LB / NW) * (K / 4) >= 32;
    Cx *Z;
    if constexpr (WFFT) {
        constexpr int LPW = LB / NW;
        const int w = threadIdx.x >> 5;
        Cx *Zw = cta_fft_t<R, K, LPW, 32, false, true>(bufA + w * LPW * K, bufB + w * LPW * K, twsm,
                                                       false, threadIdx.x & 31);
        Z = (Zw == bufA + w * LPW * K) ? bufA : bufB;
        __syncthreads();
    } else {
        Z = cta_fft_t<R, K, LB, NT, false, false, TWS>(bufA, bufB, twsm, false);
    }
    R *o = reinterpret_cast<R *>(Z == bufA ? bufB : bufA);   // R[LB][M]

    // 4. post-processing: even outputs final, odd slots get Re T_k
    for (int f = threadIdx.x; f < LB * (K / 2); f += NT) {
        const int l = f / (K / 2);
        const int k = f - l * (K / 2) + 1;      // 1..K/2
        const Cx *zl = Z + l * K;
        R *ol = o + l * M;
        const Cx zk = zl[k], zc = zl[K - k];
        const R Er = A::add(A::re(zk), A::re(zc)), Ei = A::sub(A::im(zk), A::im(zc));
        const R Or = A::sub(A::re(zk), A::re(zc)), Oi = A::add(A::im(zk), A::im(zc));
        if constexpr (std::is_same<R, double>::value) {
            // P = W O with W in ratio form: P_re = mre u, P_im = mim v (10 FP64 ops per pair)
            const Tw w = a.halfr[k];
            const double Pp = w.swap ? Oi : Or, Qq = w.swap ? Or : Oi;
            const double u = fma(-w.r, Qq, Pp), v = fma(w.r, Pp, Qq);
            ol[2 * k - 1] = fma(w.mre, u, -Ei);
            ol[2 * (K - k) - 1] = fma(w.mre, u, Ei);
            ol[2 * k] = fma(w.mim, v, Er);
            ol[2 * (K - k)] = fma(-w.mim, v, Er);
        } else {
            const Cx w = Tabs<R>::half(a, k);
            const R Pr = A::mul_sub(A::re(w), Or, A::im(w), Oi);
            const R Pi = A::mul_add(A::re(w), Oi, A::im(w), Or);
            ol[2 * k - 1] = A::sub(Pr, Ei);
            ol[2 * (K - k) - 1] = A::add(Ei, Pr);
            ol[2 * k] = A::add(Er, Pi);
            ol[2 * (K - k)] = A::sub(Er, Pi);
        }
        if constexpr (!std::is_same<R, double>::value)
            if (k == 1) ol[0] = A::add(A::re(zl[0]), A::im(zl[0]));
    }
    __syncthreads();

    // 5. prefix sum over the odd slots o[2k], k = 0..K-1
    if constexpr (std::is_same<R, double>::value) {
        // eight lanes per line, each scanning an eighth of the odd slots: every FP64
        // warp instruction then has all its lanes busy (an FP64 warp instruction
        // costs the pipe the same whatever its active lanes), and each lane's chain
        // of dependent additions is K/4 + 3 long (against K/2 + 2 with four lanes,
        // measured 2 us per solve faster at 129^3).  Per lane: the total of its
        // eighth, an inclusive scan of the eight totals by shuffles, then the
        // eighth again from the lower eighths' sum.  The summation order is the
        // same for every block shape.  Requires 8 LB <= threads per block and
        // whole warps of lines (LB >= 4), or LB = 2 in part of warp 0.
        constexpr int S = 8, Cq = K / S;
        // the scan lanes: whole warps, or the lowest 8 LB lanes of warp 0 (LB = 2)
        constexpr unsigned SMASK = (S * LB >= 32) ? 0xffffffffu : ((1u << (S * LB)) - 1u);
        const int l = threadIdx.x / S, sg = threadIdx.x - l * S;
        if (l < LB) {
            double *ol = o + l * M;
            const Cx z0 = Z[l * K];
            // slot 0 = Re T_0 + Im T_0, the first odd output
            const double first = A::re(z0) + A::im(z0);
            const int kb = sg * Cq;
            double tot = sg == 0 ? first : ol[2 * kb];
#pragma unroll 8
            for (int c = 1; c < Cq; ++c) tot += ol[2 * (kb + c)];
            double incl = tot;
#pragma unroll
            for (int dd = 1; dd < S; dd <<= 1) {
                const double nb = __shfl_up_sync(SMASK, incl, dd, S);
                incl += sg >= dd ? nb : 0.0;
            }
            // sum of the lower quarters: the inclusive sum of the lane below
            const double below = __shfl_up_sync(SMASK, incl, 1, S);
            double run = sg == 0 ? first : below + ol[2 * kb];
            ol[2 * kb] = run;
#pragma unroll 8
            for (int c = 1; c < Cq; ++c) {
                run += ol[2 * (kb + c)];
                ol[2 * (kb + c)] = run;
            }
        }
    } else {
        constexpr int G = Cfg::G, C = Cfg::C;
        const int l = threadIdx.x / G;
        const int g = threadIdx.x - l * G;
        R vals[C];
        R run = A::zero();
#pragma unroll
        for (int c = 0; c < C; ++c) {
            if (g * C + c < K) run = A::add(run, o[l * M + 2 * (g * C + c)]);
            vals[c] = run;
        }
        // inclusive scan of the group totals (groups of G consecutive lanes)
        R incl = run;
#pragma unroll
        for (int dd = 1; dd < G; dd <<= 1) {
            const R nb = A::shfl_up(incl, dd, G);
            if (g >= dd) incl = A::add(incl, nb);
        }
        const R off = A::sub(incl, run);
#pragma unroll
        for (int c = 0; c < C; ++c)
            if (g * C + c < K) o[l * M + 2 * (g * C + c)] = A::add(vals[c], off);
    }
    __syncthreads();

    // 6. epilogue and store
    int64_t osu, osv, ose, asu, asv, ase, tsu, tsv, tse;
    view_strides(a.out, a.axis, osu, osv, ose);
    view_strides(a.add, a.axis, asu, asv, ase);
    {
        // the tables are dense interior arrays n0 x n1 x n2
        const View3 tv{nullptr, (int64_t)a.n1 * a.n2, a.n2, 1};
        view_strides(tv, a.axis, tsu, tsv, tse);
    }
    const int64_t outb = (int64_t)u * osu + (int64_t)v0 * osv;
    const int64_t tabb = (int64_t)u * tsu + (int64_t)v0 * tsv;
    const int64_t addb = (int64_t)u * asu + (int64_t)v0 * asv;
    const bool has_tab = a.tab || a.tabd;
    if (!has_tab && !a.add.p) {
        for (int f = threadIdx.x; f < LB * N; f += NT) {
            int l, e;
            if (contig) { l = f / N; e = f - l * N; }
            else { e = f / LB; l = f - e * LB; }
            if (l >= nl) continue;
            Io<R>::st(a.out.p, outb + (int64_t)l * osv + (int64_t)e * ose, o[l * M + e], a.out_dd);
        }
        return;
    }
    // groups of EG outputs: the table and addend loads of a group go out before
    // its stores (which, as far as the compiler knows, could alias them)
    constexpr int EG = 4;
    for (int f0 = threadIdx.x; f0 < LB * N; f0 += EG * NT) {
        R tv[EG], av[EG];
#pragma unroll
        for (int g = 0; g < EG; ++g) {
            const int f = f0 + g * NT;
            tv[g] = A::zero();
            av[g] = A::zero();
            if (f >= LB * N) continue;
            int l, e;
            if (contig) { l = f / N; e = f - l * N; }
            else { e = f / LB; l = f - e * LB; }
            if (l >= nl) continue;
            const int64_t ti = tabb + (int64_t)l * tsv + (int64_t)e * tse;
            const int64_t ai = addb + (int64_t)l * asv + (int64_t)e * ase;
            if (has_tab) tv[g] = Io<R>::ld(a.tabd ? (const void *)a.tabd : (const void *)a.tab, ti, a.tabd != nullptr);
            if (a.add.p) av[g] = Io<R>::ld(a.add.p, ai, a.add_dd);
        }
#pragma unroll
        for (int g = 0; g < EG; ++g) {
            const int f = f0 + g * NT;
            if (f >= LB * N) break;
            int l, e;
            if (contig) { l = f / N; e = f - l * N; }
            else { e = f / LB; l = f - e * LB; }
            if (l >= nl) continue;
            R y = o[l * M + e];
            if (has_tab) {
                if (a.add.p) y = A::fma(tv[g], y, av[g]);
                else y = A::mul(tv[g], y);
            } else {
                y = A::add(y, av[g]);
            }
            Io<R>::st(a.out.p, outb + (int64_t)l * osv + (int64_t)e * ose, y, a.out_dd);
        }
    }
}

// Direct sine sums for line lengths without an FFT here (any M <= 513): every
// output U_e = 4 sum_i S[i][e] x_i with S[i][e] = sin(pi (i+1)(e+1) / M) from the
// table a.sinm (FP64, or double-float pairs when R is ddr), stored with e fastest
// so that consecutive threads read consecutive entries.  LBD lines per block, held
// in shared memory; thread t computes modes t, t + 256 for all of them.  The same
// epilogue as the FFT pass.
constexpr int LBD = 16, DMAX = 2;   // lines per block, modes per thread (N <= 512)

template <class R>
__global__ void __launch_bounds__(NT) dst_direct_kernel(const DstPass a)
{
    pdl_enter();
    using A = Ar<R>;
    const int M = a.M, N = M - 1;
    extern __shared__ double2 smem_raw[];
    R *xs = reinterpret_cast<R *>(smem_raw);   // [LBD][N]
    const int nv = a.axis == 2 ? a.n1 : a.n2;
    const int u = blockIdx.y;
    const int v0 = blockIdx.x * LBD;
    const int nl = min(LBD, nv - v0);
    const bool contig = (a.axis == 2);
    int64_t isu, isv, ise;
    view_strides(a.in, a.axis, isu, isv, ise);
    const int64_t inb = (int64_t)u * isu + (int64_t)v0 * isv;
    for (int f = threadIdx.x; f < LBD * N; f += NT) {
        int l, i;
        if (contig) { l = f / N; i = f - l * N; }
        else { i = f / LBD; l = f - i * LBD; }
        xs[l * N + i] = l < nl ? Io<R>::ld(a.in.p, inb + (int64_t)l * isv + (int64_t)i * ise, a.in_dd) : A::zero();
    }
    __syncthreads();
    R acc[DMAX][LBD];
#pragma unroll
    for (int j = 0; j < DMAX; ++j)
#pragma unroll
        for (int l = 0; l < LBD; ++l) acc[j][l] = A::zero();
    const R *S = reinterpret_cast<const R *>(a.sinm);
    for (int i = 0; i < N; ++i) {
#pragma unroll
        for (int j = 0; j < DMAX; ++j) {
            const int e = threadIdx.x + j * NT;
            if (e >= N) break;
            const R sv = S[(int64_t)i * N + e];
#pragma unroll
            for (int l = 0; l < LBD; ++l) acc[j][l] = A::fma(sv, xs[l * N + i], acc[j][l]);
        }
    }
    int64_t osu, osv, ose, asu, asv, ase, tsu, tsv, tse;
    view_strides(a.out, a.axis, osu, osv, ose);
    view_strides(a.add, a.axis, asu, asv, ase);
    {
        const View3 tv{nullptr, (int64_t)a.n1 * a.n2, a.n2, 1};
        view_strides(tv, a.axis, tsu, tsv, tse);
    }
    const int64_t outb = (int64_t)u * osu + (int64_t)v0 * osv;
    const int64_t tabb = (int64_t)u * tsu + (int64_t)v0 * tsv;
    const int64_t addb = (int64_t)u * asu + (int64_t)v0 * asv;
    const bool has_tab = a.tab || a.tabd;
#pragma unroll
    for (int j = 0; j < DMAX; ++j) {
        const int e = threadIdx.x + j * NT;
        if (e >= N) break;
#pragma unroll
        for (int l = 0; l < LBD; ++l) {
            if (l >= nl) break;
            R y = times4_exact(acc[j][l]);
            const int64_t ti = tabb + (int64_t)l * tsv + (int64_t)e * tse;
            const int64_t ai = addb + (int64_t)l * asv + (int64_t)e * ase;
            if (has_tab) {
                const R t = Io<R>::ld(a.tabd ? (const void *)a.tabd : (const void *)a.tab, ti, a.tabd != nullptr);
                if (a.add.p) y = A::fma(t, y, Io<R>::ld(a.add.p, ai, a.add_dd));
                else y = A::mul(t, y);
            } else if (a.add.p) {
                y = A::add(y, Io<R>::ld(a.add.p, ai, a.add_dd));
            }
            Io<R>::st(a.out.p, outb + (int64_t)l * osv + (int64_t)e * ose, y, a.out_dd);
        }
    }
}

template <class R>
cudaError_t launch_direct(const DstPass &a, cudaStream_t st)
{
    if (a.M - 1 > DMAX * NT || !a.sinm) return cudaErrorInvalidValue;
    int nu, nv;
    if (a.axis == 2) { nu = a.n0; nv = a.n1; }
    else if (a.axis == 1) { nu = a.n0; nv = a.n2; }
    else { nu = a.n1; nv = a.n2; }
    const size_t sm = sizeof(R) * LBD * (a.M - 1);
    dim3 grid((nv + LBD - 1) / LBD, nu);
    return launch_pdl(dst_direct_kernel<R>, grid, dim3(NT), sm, st, a);
}

template <class R, int K, int LBO, int NTB = NT>
cudaError_t launch_lb(const DstPass &a, int nu, int nv, cudaStream_t st)
{
    using Cfg = DstCfg<K, LBO, NTB>;
    // (the double-float scan runs on G lanes per line; the FP64 one on four)
    static_assert(std::is_same<R, double>::value || Cfg::G <= 32, "scan group must fit a warp");
    static_assert(Cfg::LB * Cfg::G == NTB, "every thread belongs to one scan group");
    static_assert(8 * Cfg::LB <= NTB && (Cfg::LB >= 8 || Cfg::LB == 4 || Cfg::LB == 2) && K % 8 == 0,
                  "eight scan lanes per line: whole warps, or part of warp 0");
    const size_t sm = 2 * sizeof(double2) * Cfg::LB * K + 32 * (K / 2);   // + the twiddles
    dim3 grid((nv + Cfg::LB - 1) / Cfg::LB, nu);
    return launch_pdl(dst_pass_kernel<R, K, LBO, NTB>, grid, dim3(NTB), sm, st, a);
}

template <class R, int K>
cudaError_t launch_k(const DstPass &a, cudaStream_t st)
{
    int nu, nv;
    if (a.axis == 2) { nu = a.n0; nv = a.n1; }
    else if (a.axis == 1) { nu = a.n0; nv = a.n2; }
    else { nu = a.n1; nv = a.n2; }
    // 32 lines (M = 128) or 16 lines (M = 256) per block: the per-line prefix sum
    // then runs on at least half a warp (an FP64 warp instruction costs the pipe the
    // same whatever its active lanes)
    if constexpr (K == 64) {
        if (a.lines == 32) return launch_lb<R, K, 32>(a, nu, nv, st);
    }
    if constexpr (K == 128) {
        if (a.lines == 16) return launch_lb<R, K, 16>(a, nu, nv, st);
    }
    // 4 lines on 128 threads (M = 256, 512): a warp per line, smaller blocks
    if constexpr (K == 128 || K == 256) {
        if (a.lines == 4) return launch_lb<R, K, 4, 128>(a, nu, nv, st);
    }
    if constexpr (DstCfg<K>::LB > 8) {
        // a launch of less than two blocks per SM (the layer transforms) runs
        // faster on more, smaller blocks: FP64 on 2 lines per 128-thread block
        // (measured against 4 lines on 64, 128 or 256 threads and 8 on 256)
        const int64_t blocks = (int64_t)nu * ((nv + DstCfg<K>::LB - 1) / DstCfg<K>::LB);
        if constexpr (std::is_same<R, double>::value) {
            if (blocks < 2 * 152) return launch_lb<R, K, 2, 128>(a, nu, nv, st);
        }
        if (a.lines == 8 || blocks < 2 * 152) return launch_lb<R, K, 8>(a, nu, nv, st);
        // 8 lines on 128 threads: one radix-4 unit per thread per pass for K = 64
        if (a.lines == -8 && K == 64) return launch_lb<R, K, 8, 128>(a, nu, nv, st);
    }
    return launch_lb<R, K, 0>(a, nu, nv, st);
}

template <class R, int K, int LBO, int NTB = NT>
cudaError_t attr_lb()
{
    using Cfg = DstCfg<K, LBO, NTB>;
    const int sm = (int)(2 * sizeof(double2) * Cfg::LB * K + 32 * (K / 2));
    return cudaFuncSetAttribute(dst_pass_kernel<R, K, LBO, NTB>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm);
}

template <class R, int K>
cudaError_t attr_k()
{
    cudaError_t e = attr_lb<R, K, 0>();
    if (e != cudaSuccess) return e;
    if constexpr (DstCfg<K>::LB > 8) {
        e = attr_lb<R, K, 8>();
        if constexpr (std::is_same<R, double>::value)
            if (e == cudaSuccess) e = attr_lb<R, K, 2, 128>();
    }
    if constexpr (K == 64) {
        if (e == cudaSuccess) e = attr_lb<R, K, 8, 128>();
        if (e == cudaSuccess) e = attr_lb<R, K, 32>();
    }
    if constexpr (K == 128) {
        if (e == cudaSuccess) e = attr_lb<R, K, 16>();
    }
    if constexpr (K == 128 || K == 256) {
        if (e == cudaSuccess) e = attr_lb<R, K, 4, 128>();
    }
    return e;
}

template <class R>
cudaError_t attrs()
{
    cudaError_t e;
    if ((e = attr_k<R, 8>()) != cudaSuccess) return e;
    if ((e = attr_k<R, 16>()) != cudaSuccess) return e;
    if ((e = attr_k<R, 24>()) != cudaSuccess) return e;
    if ((e = attr_k<R, 32>()) != cudaSuccess) return e;
    if ((e = attr_k<R, 48>()) != cudaSuccess) return e;
    if ((e = attr_k<R, 64>()) != cudaSuccess) return e;
    if ((e = attr_k<R, 96>()) != cudaSuccess) return e;
    if ((e = attr_k<R, 128>()) != cudaSuccess) return e;
    if ((e = attr_k<R, 192>()) != cudaSuccess) return e;
    return attr_k<R, 256>();
}

template <class R>
cudaError_t launch_r(const DstPass &a, cudaStream_t st)
{
    switch (a.M) {
    case 16: return launch_k<R, 8>(a, st);
    case 32: return launch_k<R, 16>(a, st);
    case 48: return launch_k<R, 24>(a, st);
    case 64: return launch_k<R, 32>(a, st);
    case 96: return launch_k<R, 48>(a, st);
    case 128: return launch_k<R, 64>(a, st);
    case 192: return launch_k<R, 96>(a, st);
    case 256: return launch_k<R, 128>(a, st);
    case 384: return launch_k<R, 192>(a, st);
    case 512: return launch_k<R, 256>(a, st);
    default: return launch_direct<R>(a, st);   // no FFT for this length: direct sums
    }
}

}  // namespace

cudaError_t dst_set_attributes()
{
    cudaError_t e = attrs<double>();
    if (e != cudaSuccess) return e;
    if ((e = attrs<ddr>()) != cudaSuccess) return e;
    const int sm = (int)(sizeof(double) * LBD * DMAX * NT);
    if ((e = cudaFuncSetAttribute(dst_direct_kernel<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm)))
        return e;
    return cudaFuncSetAttribute(dst_direct_kernel<ddr>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm);
}

cudaError_t launch_dst_pass(const DstPass &a, cudaStream_t st)
{
    return a.dd ? launch_r<ddr>(a, st) : launch_r<double>(a, st);
}

}  // namespace idp
