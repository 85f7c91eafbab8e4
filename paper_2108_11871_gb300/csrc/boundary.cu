// Boundary values of the harmonic correction (section 4): the trapezoid sum
// of G * rho on every boundary node, evaluated as the paper rearranges it
// (eqs. Trap2D, Trap2Dconvolution, convolution): for each face, a sum over the
// slices parallel to it of aperiodic convolutions of the rho slice with
// G(sqrt(dist^2 + |.|^2)), done with zero-padded FFTs of length 2P, P >= M
// (P = M where M has an FFT here; otherwise the next length that has one: the
// zero-padded cyclic convolution is exact for any 2P >= 2M - 1).
//
// 3-D data flow (faces of axis a; b < c the other two axes):
//   stage 1  real FFT (length 2P_c) along c of every interior line of rho
//   stage 2  FFT (length 2P_b) along b of every slice p, multiplied by the
//            kernel spectra of distance p h_a and (M_a - p) h_a, summed over p
//   stage 3  inverse FFT along b, inverse real FFT along c, scatter to nodes.
// The kernel spectra are real and even (the cyclic kernel is even), so only
// frequencies 0..P are stored; they are computed once per plan.
#include <type_traits>

#include "fft.cuh"

namespace idp {

namespace {
constexpr int NT = 256;
// threads per block of the real-FFT pass: 256, except double-float at L = 512 on 128
// (the LB x L = 512 complex values of a block give 128 radix-4 units per pass, one per
// thread; that latency-bound pass ran 9 % faster at 513^3 so, while at L <= 256 the
// 96-problem batch ran 4.5 % slower, and FP64, bound by its pipe, gained nothing)
template <class R, int L>
struct RfftThreads {
    static constexpr int value = (!std::is_same<R, double>::value && L >= 512) ? 128 : 256;
};

// lines per block: 2 buffers of LB x L complex in 16 KB (small blocks: the
// all-zero line blocks of rho finish at once, and many blocks per SM keep the FP64
// pipe busy on the others; measured best at M = 128)
template <int L>
struct LineCfg {
    static constexpr int LB = (512 / L) > 32 ? 32 : ((512 / L) < 1 ? 1 : 512 / L);
};

// ---------------------------------------------------------------- stage 1
// L = P: complex FFT length; input line has M-1 reals (M = a.M <= L) at
// positions 1..M-1 of a zero-padded sequence of length 2L; output X'_m = 2 X_m,
// m = 0..L.
// 2 x, exact: for a normal FP64 value by adding 1 to the exponent (integer pipe),
// otherwise by the multiplication
__device__ __forceinline__ double times2_exact(double x)
{
    const long long b = __double_as_longlong(x);
    const int e = (int)((b >> 52) & 0x7ff);
    if (e >= 1 && e <= 2045) return __longlong_as_double(b + (1LL << 52));
    return x * 2.0;
}

template <class R>
__device__ __forceinline__ R ld_real(const double *p, int64_t i);
template <>
__device__ __forceinline__ double ld_real<double>(const double *p, int64_t i) { return p[i]; }
template <>
__device__ __forceinline__ ddr ld_real<ddr>(const double *p, int64_t i) { return dd_from_bits(p[i]); }
template <class R>
__device__ __forceinline__ void st_real(double *p, int64_t i, R v);
template <>
__device__ __forceinline__ void st_real<double>(double *p, int64_t i, double v) { p[i] = v; }
template <>
__device__ __forceinline__ void st_real<ddr>(double *p, int64_t i, ddr v) { p[i] = dd_to_bits(v); }

template <class R>
__device__ __forceinline__ const typename Ar<R>::T *fwd_tw(const FftTables &t);
template <>
__device__ __forceinline__ const Tw *fwd_tw<double>(const FftTables &t) { return t.fwd; }
template <>
__device__ __forceinline__ const TwD *fwd_tw<ddr>(const FftTables &t) { return t.fwdd; }
template <class R>
__device__ __forceinline__ const typename Ar<R>::T *inv_tw(const FftTables &t);
template <>
__device__ __forceinline__ const Tw *inv_tw<double>(const FftTables &t) { return t.inv; }
template <>
__device__ __forceinline__ const TwD *inv_tw<ddr>(const FftTables &t) { return t.invd; }
template <class R>
__device__ __forceinline__ typename Ar<R>::C half_tw(const FftTables &t, int k);
template <>
__device__ __forceinline__ double2 half_tw<double>(const FftTables &t, int k) { return t.half[k]; }
template <>
__device__ __forceinline__ ddc half_tw<ddr>(const FftTables &t, int k) { return t.halfd[k]; }

template <class R, int L>
__global__ void __launch_bounds__(RfftThreads<R, L>::value) rfft_kernel(const RfftPass a)
{
    constexpr int NTL = RfftThreads<R, L>::value;
    using A = Ar<R>;
    using Cx = typename A::C;
    constexpr int LB = LineCfg<L>::LB;
    const int M = a.M, N = M - 1;
    extern __shared__ double2 smem_raw[];
    Cx *bufA = reinterpret_cast<Cx *>(smem_raw), *bufB = bufA + LB * L;
    int nu, nv;
    int64_t isu, isv, ise, osu, osv, ose;
    if (a.axis == 2) {
        nu = a.n0; nv = a.n1;
        isu = a.is0; isv = a.is1; ise = a.is2; osu = a.os0; osv = a.os1; ose = a.os2;
    } else if (a.axis == 1) {
        nu = a.n0; nv = a.n2;
        isu = a.is0; isv = a.is2; ise = a.is1; osu = a.os0; osv = a.os2; ose = a.os1;
    } else {
        nu = a.n1; nv = a.n2;
        isu = a.is1; isv = a.is2; ise = a.is0; osu = a.os1; osv = a.os2; ose = a.os0;
    }
    const int u = blockIdx.y, v0 = blockIdx.x * LB;
    const int nl = min(LB, nv - v0);
    const bool contig = (ise == 1);
    // lines that are all zero (rho vanishes near the boundary): zero spectra
    auto write_zero = [&]() {
        Cx *outz = reinterpret_cast<Cx *>(a.out) + (int64_t)u * osu + (int64_t)v0 * osv;
        for (int f = threadIdx.x; f < nl * (L + 1); f += NTL) {
            const int l = f / (L + 1), m = f - l * (L + 1);
            outz[(int64_t)l * osv + (int64_t)m * ose] = A::cmake(A::zero(), A::zero());
        }
    };
    if (a.lineflag) {
        __shared__ int any_nz;
        if (threadIdx.x == 0) any_nz = 0;
        __syncthreads();
        if (threadIdx.x < nl && a.lineflag[(int64_t)u * nv + v0 + threadIdx.x]) any_nz = 1;
        __syncthreads();
        if (!any_nz) {
            write_zero();
            return;
        }
    }
    // stage 1a: non-zero marks of the block's lines and of their element
    // positions, in the FFT scratch (free until the FFT)
    const bool mk = a.fl_row2 != nullptr;
    int *colnz = reinterpret_cast<int *>(bufB), *rownz = colnz + L;
    R *zf = reinterpret_cast<R *>(bufA);   // [LB][2L] reals
    const int64_t inb = (int64_t)u * isu + (int64_t)v0 * isv;
    for (int f = threadIdx.x; f < LB * 2 * L; f += NTL) {
        const int l = f / (2 * L), q = f - l * 2 * L;
        if (q == 0 || q >= M) zf[f] = A::zero();
    }
    if (mk) {
        for (int f = threadIdx.x; f < L + LB; f += NTL) colnz[f] = 0;
        __syncthreads();
    }
    int nz = 0;
    for (int f = threadIdx.x; f < LB * N; f += NTL) {
        int l, e;
        if (contig) { l = f / N; e = f - l * N; }
        else { e = f / LB; l = f - e * LB; }
        R x = A::zero();
        if (l < nl) {
            const int64_t i = inb + (int64_t)l * isv + (int64_t)e * ise;
            const double xd = a.in[i];
            if (a.copy) a.copy[i] = xd;
            // zero test on the bits (+0 and -0 are zero), off the FP64 pipe
            if (mk && (__double_as_longlong(xd) << 1) != 0) {
                colnz[e] = 1;
                rownz[l] = 1;
                nz = 1;
            }
            x = ld_real<R>(&xd, 0);
        }
        zf[l * 2 * L + e + 1] = x;
    }
    if (mk) {
        const int any = __syncthreads_or(nz);
        if (threadIdx.x < nl) {
            const int rf = rownz[threadIdx.x];
            a.fl_row2[(int64_t)u * nv + v0 + threadIdx.x] = rf;
            // flags shared by many blocks are read before they are set (a store to
            // a line that many SMs write is slow; a stale 0 costs one more store)
            if (rf && !a.fl_sl1[v0 + threadIdx.x]) a.fl_sl1[v0 + threadIdx.x] = 1;
        }
        if (any) {
            if (threadIdx.x == 0 && !a.fl_sl0[u]) a.fl_sl0[u] = 1;
            for (int e = threadIdx.x; e < N; e += NTL)
                if (colnz[e]) {
                    int *f1 = a.fl_row1 + (int64_t)u * a.n2 + e;
                    if (!*f1) *f1 = 1;
                    if (!a.fl_sl2[e]) a.fl_sl2[e] = 1;
                }
        }
        __syncthreads();
        if (!any) {
            write_zero();
            return;
        }
    } else {
        __syncthreads();
    }
    // the FFT's L / 2 twiddles, copied into shared memory once (read in every pass;
    // from the global table they are long-scoreboard loads)
    using TwT = typename Ar<R>::T;
    static_assert(sizeof(TwT) <= 32, "the shared-memory size counts 32 bytes per twiddle");
    TwT *twsm = reinterpret_cast<TwT *>(bufB + LB * L);
    // (double-float: in the bank-spread planes of tw_stage)
    constexpr bool TWS = !std::is_same<R, double>::value && TwSwz<L>::ok;
    if constexpr (TWS) {
        tw_stage<L>(twsm, fwd_tw<R>(a.t), threadIdx.x, NTL);
    } else {
        const TwT *tg = fwd_tw<R>(a.t);
        for (int i = threadIdx.x; i < L / 2; i += NTL) twsm[i] = tg[i];
    }
    __syncthreads();
    Cx *Z = cta_fft_t<R, L, LB, NTL, false, false, TWS>(bufA, bufB, twsm, true);
    Cx *outb = reinterpret_cast<Cx *>(a.out) + (int64_t)u * osu + (int64_t)v0 * osv;
    for (int f = threadIdx.x; f < LB * (L / 2); f += NTL) {
        const int l = f / (L / 2);
        const int m = f - l * (L / 2) + 1;   // 1..L/2
        if (l >= nl) continue;
        const Cx *zl = Z + l * L;
        const Cx zm = zl[m], zc = zl[L - m];
        const R Er = A::add(A::re(zm), A::re(zc)), Ei = A::sub(A::im(zm), A::im(zc));
        const R Or = A::sub(A::re(zm), A::re(zc)), Oi = A::add(A::im(zm), A::im(zc));
        Cx *ol = outb + (int64_t)l * osv;
        if constexpr (std::is_same<R, double>::value) {
            // P = W O in ratio form (10 FP64 ops per pair of outputs)
            const Tw w = a.t.halfr[m];
            const double Pp = w.swap ? Oi : Or, Qq = w.swap ? Or : Oi;
            const double u = fma(-w.r, Qq, Pp), v = fma(w.r, Pp, Qq);
            ol[(int64_t)m * ose] = make_double2(fma(w.mim, v, Er), fma(-w.mre, u, Ei));
            ol[(int64_t)(L - m) * ose] = make_double2(fma(-w.mim, v, Er), -fma(w.mre, u, Ei));
        } else {
            const Cx w = half_tw<R>(a.t, m);
            const R Pr = A::mul_sub(A::re(w), Or, A::im(w), Oi);
            const R Pi = A::mul_add(A::re(w), Oi, A::im(w), Or);
            ol[(int64_t)m * ose] = A::cmake(A::add(Er, Pi), A::sub(Ei, Pr));
            ol[(int64_t)(L - m) * ose] = A::cmake(A::sub(Er, Pi), A::neg(A::add(Ei, Pr)));
        }
        if constexpr (!std::is_same<R, double>::value) {
            if (m == 1) {
                const Cx z0 = zl[0];
                ol[0] = A::cmake(A::times2(A::add(A::re(z0), A::im(z0))), A::zero());
                ol[(int64_t)L * ose] = A::cmake(A::times2(A::sub(A::re(z0), A::im(z0))), A::zero());
            }
        }
    }
    if constexpr (std::is_same<R, double>::value) {
        // m = 0 and m = L, one lane per line (an FP64 warp instruction costs the
        // pipe the same whatever its active lanes; Z is still intact)
        if (threadIdx.x < nl) {
            const double2 z0 = Z[threadIdx.x * L];
            double2 *ol = outb + (int64_t)threadIdx.x * osv;
            ol[0] = make_double2(times2_exact(z0.x + z0.y), 0.0);
            ol[(int64_t)L * ose] = make_double2(times2_exact(z0.x - z0.y), 0.0);
        }
    }
}

// ---------------------------------------------------------------- stage 2
// columns per block of the face pass: TC x L = 1024 complex per block
template <int L>
struct FaceCfg {
    static constexpr int TC = (1024 / L) > 32 ? 32 : ((1024 / L) < 1 ? 1 : 1024 / L);
};

// L = 2 Pb (Pb >= Mb).  Block: TC consecutive frequencies c, one chunk of slices p.
template <class R>
__device__ __forceinline__ R ld_khat(const FacePass &a, int64_t i);
template <>
__device__ __forceinline__ double ld_khat<double>(const FacePass &a, int64_t i) { return a.khat[i]; }
template <>
__device__ __forceinline__ ddr ld_khat<ddr>(const FacePass &a, int64_t i) { return a.khatd[i]; }

// asynchronous 16-byte copies global -> shared (no register holds the value in flight)
__device__ __forceinline__ void cp_async16(void *dst, const void *src)
{
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"((unsigned)__cvta_generic_to_shared(dst)),
                 "l"(src)
                 : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;\n" ::: "memory"); }

// four blocks per SM (64 registers; at 72, with the fused first pass, three fit
// and the pass ran 8 % slower; the cap costs a small spill at some lengths, 32
// bytes at L = 1024 in FP64, none at L = 256)
template <class R, int L>
__global__ void __launch_bounds__(NT, 4) face_kernel(const FacePass a)
{
    using A = Ar<R>;
    using Cx = typename A::C;
    constexpr int TC = FaceCfg<L>::TC;
    constexpr int Ph = L / 2;                     // frequencies 0..Ph of the even kernel spectra
    const int Mb = a.Mb;                          // data: positions 1..Mb-1 along b
    constexpr int OPT = (TC * L + NT - 1) / NT;   // outputs per thread
    extern __shared__ double2 smem_raw[];
    Cx *bufA = reinterpret_cast<Cx *>(smem_raw), *bufB = bufA + TC * L;
    const int c0 = blockIdx.x * TC;
    const int ncl = min(TC, a.nc - c0);
    const int chunk = blockIdx.y;
    const int p0 = chunk * a.pchunk;
    const int p1 = min(a.np, p0 + a.pchunk);
    Cx acc_lo[OPT], acc_hi[OPT];
#pragma unroll
    for (int r = 0; r < OPT; ++r) {
        acc_lo[r] = A::cmake(A::zero(), A::zero());
        acc_hi[r] = A::cmake(A::zero(), A::zero());
    }
    const int64_t kstride = (int64_t)(Ph + 1) * a.nc;
    const Cx *D = reinterpret_cast<const Cx *>(a.D);
    // L a power of two: the first radix-4 pass is fused with the load of the slice.
    // Double-float (latency-bound; the FP64 pass is bound by its pipe and keeps its
    // registers): the non-zero half of the next slice's columns (positions 0..L/2-1,
    // data at 1..Mb-1) is brought into stg[t][j] by asynchronous copies while the
    // current slice's FFT runs; the positions without data are zeroed once
    constexpr bool P2L = (L & (L - 1)) == 0;
    constexpr bool PF = P2L && !std::is_same<R, double>::value;
    constexpr int HL = L / 2;
    Cx *stg = bufB + TC * L;
    // L a power of two: the FFT's twiddles copied into shared memory once (read in
    // every pass of every slice; from the global table they are long-scoreboard loads
    // in double-float, which is latency-bound)
    using TwT = typename Ar<R>::T;
    static_assert(sizeof(TwT) <= 32, "the shared-memory size counts 32 bytes per twiddle");
    TwT *twsm = reinterpret_cast<TwT *>(stg + TC * HL);
    const TwT *twp = fwd_tw<R>(a.t);
    constexpr bool TWS = PF && TwSwz<L>::ok;   // double-float: the bank-spread planes of tw_stage
    if constexpr (P2L) {
        if constexpr (TWS) tw_stage<L>(twsm, twp, threadIdx.x, NT);
        else
            for (int i = threadIdx.x; i < L / 2; i += NT) twsm[i] = twp[i];
        twp = twsm;
        if constexpr (!PF) __syncthreads();   // (double-float: the barrier at the top of the slice loop)
    }
    auto next_slice = [&](int q) {
        while (q < p1 && a.sliceflag && !a.sliceflag[q]) ++q;   // slices of zeros contribute nothing
        return q;
    };
    auto prefetch = [&](int q) {
        const Cx *Dq = D + (int64_t)q * a.sp + (int64_t)c0 * a.sc;
        for (int f = threadIdx.x; f < TC * HL; f += NT) {
            const int j = f / TC, t = f - j * TC;   // consecutive threads: consecutive columns
            if (t < ncl && j >= 1 && j <= Mb - 1)
                cp_async16(stg + t * HL + j, Dq + (int64_t)(j - 1) * a.sb + (int64_t)t * a.sc);
        }
        cp_async_commit();
    };
    if constexpr (PF) {
        for (int f = threadIdx.x; f < TC * HL; f += NT) {
            const int j = f / TC, t = f - j * TC;
            if (!(t < ncl && j >= 1 && j <= Mb - 1)) stg[t * HL + j] = A::cmake(A::zero(), A::zero());
        }
        const int pn = next_slice(p0);
        if (pn < p1) prefetch(pn);
    }
    for (int p = next_slice(p0); p < p1; p = next_slice(p + 1)) {
        // TC columns of the slice: positions 1..Mb-1 (interior index 0..Mb-2), rest zero
        const Cx *Dp = D + (int64_t)p * a.sp + (int64_t)c0 * a.sc;
        const Cx *Z;
        if constexpr (P2L) {
            // the load fused with the first radix-4 pass: a thread takes the two
            // non-zero inputs x_j, x_{j+L/4} of its unit (the upper half is zero)
            // and writes the unit's four outputs
            constexpr int Q = L / 4;
            if constexpr (PF) {
                cp_async_wait_all();
                __syncthreads();   // every thread's copies have landed
            }
            for (int f = threadIdx.x; f < TC * Q; f += NT) {
                const int j = f / TC, t = f - j * TC;   // consecutive threads: consecutive columns
                Cx a0, a1;
                if constexpr (PF) {
                    a0 = stg[t * HL + j];
                    a1 = stg[t * HL + j + Q];
                } else {
                    a0 = A::cmake(A::zero(), A::zero());
                    a1 = a0;
                    if (t < ncl) {
                        if (j >= 1 && j <= Mb - 1) a0 = Dp[(int64_t)(j - 1) * a.sb + (int64_t)t * a.sc];
                        if (j + Q <= Mb - 1) a1 = Dp[(int64_t)(j + Q - 1) * a.sb + (int64_t)t * a.sc];
                    }
                }
                const Cx m1 = mul_mi(a1);
                Cx *y = bufB + t * L + 4 * j;
                y[0] = A::cadd(a0, a1);
                y[1] = A::cadd(a0, m1);
                y[2] = A::csub(a0, a1);
                y[3] = A::csub(a0, m1);
            }
            __syncthreads();
            // the next slice's inputs come in while this one is transformed
            if constexpr (PF) {
                const int pn = next_slice(p + 1);
                if (pn < p1) prefetch(pn);
            }
            Z = cta_fft_t<R, L, TC, NT, false, false, TWS>(bufB, bufA, twp, false, -1, 4);
        } else {
            for (int f = threadIdx.x; f < TC * L; f += NT) {
                const int q = f / TC, t = f - q * TC;
                Cx x = A::cmake(A::zero(), A::zero());
                if (q >= 1 && q <= Mb - 1 && t < ncl) x = Dp[(int64_t)(q - 1) * a.sb + (int64_t)t * a.sc];
                bufA[t * L + q] = x;
            }
            __syncthreads();
            Z = cta_fft_t<R, L, TC, NT, false>(bufA, bufB, fwd_tw<R>(a.t), true);
        }
        const int64_t klo = (int64_t)p * kstride + (int64_t)c0 * (Ph + 1);
        const int64_t khi = (int64_t)(a.np - 1 - p) * kstride + (int64_t)c0 * (Ph + 1);
#pragma unroll
        for (int r = 0; r < OPT; ++r) {
            const int o = threadIdx.x + r * NT;
            if (o < TC * L) {
                const int m = o / TC, t = o - m * TC;
                if (t < ncl) {
                    const int mm = m <= Ph ? m : L - m;
                    const Cx X = Z[t * L + m];
                    const R kl = ld_khat<R>(a, klo + (int64_t)t * (Ph + 1) + mm);
                    const R kh = ld_khat<R>(a, khi + (int64_t)t * (Ph + 1) + mm);
                    acc_lo[r] = A::cmake(A::fma(kl, A::re(X), A::re(acc_lo[r])), A::fma(kl, A::im(X), A::im(acc_lo[r])));
                    acc_hi[r] = A::cmake(A::fma(kh, A::re(X), A::re(acc_hi[r])), A::fma(kh, A::im(X), A::im(acc_hi[r])));
                }
            }
        }
        __syncthreads();
    }
    // partial sums: part[chunk][face][m][c]
    Cx *part = reinterpret_cast<Cx *>(a.part);
    Cx *plo = part + ((int64_t)chunk * 2 + 0) * L * a.nc + c0;
    Cx *phi = part + ((int64_t)chunk * 2 + 1) * L * a.nc + c0;
#pragma unroll
    for (int r = 0; r < OPT; ++r) {
        const int o = threadIdx.x + r * NT;
        if (o < TC * L) {
            const int m = o / TC, t = o - m * TC;
            if (t < ncl) {
                plo[(int64_t)m * a.nc + t] = acc_lo[r];
                phi[(int64_t)m * a.nc + t] = acc_hi[r];
            }
        }
    }
}

// 2-D contraction over slices (no second FFT)
__global__ void face2d_kernel(const FacePass2D a)
{
    const int m = blockIdx.x * blockDim.x + threadIdx.x;
    if (m >= a.nm) return;
    double2 lo = make_double2(0.0, 0.0), hi = make_double2(0.0, 0.0);
    for (int p = 0; p < a.np; ++p) {
        const double2 x = a.T[(int64_t)p * a.sp + (int64_t)m * a.sm];
        const double kl = a.khat[(int64_t)p * a.nm + m];
        const double kh = a.khat[(int64_t)(a.np - 1 - p) * a.nm + m];
        lo.x = fma(kl, x.x, lo.x); lo.y = fma(kl, x.y, lo.y);
        hi.x = fma(kh, x.x, hi.x); hi.y = fma(kh, x.y, hi.y);
    }
    a.acc[m] = lo;
    a.acc[a.nm + m] = hi;
}

// ---------------------------------------------------------------- stage 3a
// columns per block of face_invb: its cost is the FP64 sum of the slice-chunk
// partials, one value per thread (one column of 256 values at M = 128)
template <int L>
struct InvbCfg {
    static constexpr int TC = (256 / L) > 32 ? 32 : ((256 / L) < 1 ? 1 : 256 / L);
};
template <int L>
size_t smem_invb() { return 2 * sizeof(double2) * InvbCfg<L>::TC * L; }

// rows per block of face_c2r: a few hundred blocks at M = 128 (the launch is short
// and latency-bound)
template <int L>
struct C2rCfg {
    static constexpr int LB = (128 / L) > 32 ? 32 : ((128 / L) < 1 ? 1 : 128 / L);
};
template <int L>
size_t smem_c2r() { return 2 * sizeof(double2) * C2rCfg<L>::LB * L; }

template <class R, int L>
__global__ void __launch_bounds__(NT) face_invb_kernel(const FaceInvB a)
{
    using A = Ar<R>;
    using Cx = typename A::C;
    constexpr int TC = InvbCfg<L>::TC;
    const int Mb = a.Mb;   // rows 0..Mb are the face nodes along b (Mb <= L / 2)
    extern __shared__ double2 smem_raw[];
    Cx *bufA = reinterpret_cast<Cx *>(smem_raw), *bufB = bufA + TC * L;
    const int c0 = blockIdx.x * TC;
    const int face = blockIdx.y;
    const int ncl = min(TC, a.nc - c0);
    const Cx *part = reinterpret_cast<const Cx *>(a.part);
    for (int f = threadIdx.x; f < TC * L; f += NT) {
        const int m = f / TC, t = f - m * TC;
        R sr = A::zero(), si = A::zero();
        if (t < ncl) {
            for (int ch = 0; ch < a.nchunk; ++ch) {
                const Cx v = part[(((int64_t)ch * 2 + face) * L + m) * a.nc + c0 + t];
                sr = A::add(sr, A::re(v));
                si = A::add(si, A::im(v));
            }
        }
        bufA[t * L + m] = A::cmake(sr, si);
    }
    __syncthreads();
    const Cx *Z = cta_fft_t<R, L, TC, NT, true>(bufA, bufB, inv_tw<R>(a.t), false);
    Cx *out = reinterpret_cast<Cx *>(a.out);
    for (int f = threadIdx.x; f < TC * (Mb + 1); f += NT) {
        const int j = f / TC, t = f - j * TC;
        if (t < ncl) out[((int64_t)face * (Mb + 1) + j) * a.nc + c0 + t] = Z[t * L + j];
    }
}

// ---------------------------------------------------------------- stage 3b
// L = Pc (inverse real FFT of length 2Pc, Pc >= Mc).  One line = one row of one
// face; values 0..Mc of it are face nodes.
template <class R, int L>
__global__ void __launch_bounds__(NT) face_c2r_kernel(const FaceC2R a)
{
    using A = Ar<R>;
    using Cx = typename A::C;
    constexpr int LB = C2rCfg<L>::LB;
    extern __shared__ double2 smem_raw[];
    Cx *bufA = reinterpret_cast<Cx *>(smem_raw), *bufB = bufA + LB * L;
    const int face = blockIdx.y;
    const int r0 = blockIdx.x * LB;
    const int64_t fbase = face ? a.base[1] : a.base[0];
    const int nl = min(LB, a.nrows - r0);
    const Cx *inb = reinterpret_cast<const Cx *>(a.in) + ((int64_t)face * a.nrows + r0) * (L + 1);
    for (int f = threadIdx.x; f < LB * L; f += NT) {
        const int l = f / L, k = f - l * L;
        Cx z = A::cmake(A::zero(), A::zero());
        if (l < nl) {
            const Cx xk = inb[(int64_t)l * (L + 1) + k];
            const Cx xc = inb[(int64_t)l * (L + 1) + (L - k)];
            // A = X_k + conj X_{L-k};  B = e^{+i pi k/L} (X_k - conj X_{L-k});  Z' = A + i B
            const R Arr = A::add(A::re(xk), A::re(xc)), Ai = A::sub(A::im(xk), A::im(xc));
            const R Dr = A::sub(A::re(xk), A::re(xc)), Di = A::add(A::im(xk), A::im(xc));
            const Cx w = half_tw<R>(a.t, k);   // (cos, -sin)
            const R Br = A::mul_add(A::re(w), Dr, A::im(w), Di);   // cos*Dr + sin*Di
            const R Bi = A::mul_sub(A::re(w), Di, A::im(w), Dr);   // cos*Di - sin*Dr
            z = A::cmake(A::sub(Arr, Bi), A::add(Ai, Br));
        }
        bufA[l * L + k] = z;
    }
    __syncthreads();
    const Cx *Z = cta_fft_t<R, L, LB, NT, true>(bufA, bufB, inv_tw<R>(a.t), false);
    const int Mc = a.Mc;
    for (int f = threadIdx.x; f < LB * (Mc + 1); f += NT) {
        const int l = f / (Mc + 1), t = f - l * (Mc + 1);
        if (l >= nl) continue;
        const int row = r0 + l;
        if (a.skip_row_edges && (row == 0 || row == a.nrows - 1)) continue;
        if (a.skip_col_edges && (t == 0 || t == Mc)) continue;
        const Cx z = Z[l * L + (t >> 1)];   // t <= Mc <= L, so t/2 < L
        const R v = (t & 1) ? A::im(z) : A::re(z);
        const int64_t node = fbase + (int64_t)row * a.row_stride + (int64_t)t * a.col_stride;
        st_real<R>(a.dst0, node, v);
        if (a.dst1) st_real<R>(a.dst1, node, v);
    }
}

// ---------------------------------------------------------------- 1-D
// d = 1 (section 5): the trapezoid sums for g at the two ends, with G = |x|/2,
//   g(a) = (h^2/2) sum_{p=1}^{M-1} p rho_p,   g(b) = (h^2/2) sum_{p=1}^{M-1} (M-p) rho_p,
// and the harmonic correction, the straight line through them,
//   u_i = g(a) (1 - i/M) + g(b) i/M.
// One block; the sums are compensated (Neumaier per thread, error-free pair sums
// in the reduction).  mode: LINE1D_ENDS writes g at the ends and 0 inside,
// LINE1D_LINE writes u on every node, LINE1D_ADD writes g at the ends and adds u
// to the interior of phi.
constexpr int L1_NT = 256;

__device__ __forceinline__ void two_sum(double a, double b, double &s, double &e)
{
    s = a + b;
    const double bb = s - a;
    e = (a - (s - bb)) + (b - bb);
}

__global__ void __launch_bounds__(L1_NT) line1d_kernel(const double *rho, double *phi, int M, double h, int mode)
{
    __shared__ double red[4][L1_NT];
    double sa = 0.0, ca = 0.0, sb = 0.0, cb = 0.0;
    for (int p = 1 + (int)threadIdx.x; p < M; p += L1_NT) {
        const double r = rho[p];
        double e;
        two_sum(sa, (double)p * r, sa, e);
        ca += e;
        two_sum(sb, (double)(M - p) * r, sb, e);
        cb += e;
    }
    red[0][threadIdx.x] = sa;
    red[1][threadIdx.x] = ca;
    red[2][threadIdx.x] = sb;
    red[3][threadIdx.x] = cb;
    __syncthreads();
    for (int w = L1_NT / 2; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w) {
            const int o = threadIdx.x + w;
            double s, e;
            two_sum(red[0][threadIdx.x], red[0][o], s, e);
            red[0][threadIdx.x] = s;
            red[1][threadIdx.x] += red[1][o] + e;
            two_sum(red[2][threadIdx.x], red[2][o], s, e);
            red[2][threadIdx.x] = s;
            red[3][threadIdx.x] += red[3][o] + e;
        }
        __syncthreads();
    }
    const double ga = 0.5 * h * h * (red[0][0] + red[1][0]);
    const double gb = 0.5 * h * h * (red[2][0] + red[3][0]);
    for (int i = threadIdx.x; i <= M; i += L1_NT) {
        const double t = (double)i / (double)M;
        const double u = ga * (1.0 - t) + gb * t;
        if (i == 0 || i == M) phi[i] = (i == 0) ? ga : gb;
        else if (mode == LINE1D_ENDS) phi[i] = 0.0;
        else if (mode == LINE1D_LINE) phi[i] = u;
        else phi[i] += u;
    }
}

// ---------------------------------------------------------------- kernel spectra
__global__ void kernel_fill_kernel(const KernelFill a)
{
    const int64_t total = (int64_t)a.np * (a.Mb + 1) * (a.Mc + 1);
    const double inv4pi = 1.0 / (4.0 * 3.14159265358979323846);
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total;
         i += (int64_t)gridDim.x * blockDim.x) {
        int tb, tc;
        int64_t r;
        if (a.tr) {
            tb = (int)(i % (a.Mb + 1));
            r = i / (a.Mb + 1);
            tc = (int)(r % (a.Mc + 1));
            r /= (a.Mc + 1);
        } else {
            tc = (int)(i % (a.Mc + 1));
            r = i / (a.Mc + 1);
            tb = (int)(r % (a.Mb + 1));
            r /= (a.Mb + 1);
        }
        const int p = (int)r;
        const double da = (a.p0 + p + 1) * a.ha, db = tb * a.hb, dc = tc * a.hc;
        const double r2 = da * da + db * db + dc * dc;
        double g;
        if (a.d == 3) g = -inv4pi / sqrt(r2);
        else g = inv4pi * log(r2);   // log(r)/(2 pi) = log(r^2)/(4 pi)
        a.k[i] = g;
    }
}

// ---------------------------------------------------------------- FP64 batched GEMM (plan set-up only)
constexpr int GT = 32;
__global__ void gemm_kernel(int m, int n, int k, const double *A, int64_t lda, int64_t sA,
                            const double *B, int64_t ldb, int64_t sB, double *C, int64_t ldc, int64_t sC)
{
    __shared__ double As[GT][GT + 1], Bs[GT][GT + 1];
    const int b = blockIdx.z;
    A += b * sA; B += b * sB; C += b * sC;
    const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;   // 16 x 16 threads, 2 x 2 outputs each
    const int row0 = blockIdx.y * GT, col0 = blockIdx.x * GT;
    double acc[2][2] = {{0, 0}, {0, 0}};
    for (int k0 = 0; k0 < k; k0 += GT) {
        for (int f = threadIdx.x; f < GT * GT; f += 256) {
            const int i = f / GT, j = f % GT;
            As[i][j] = (row0 + i < m && k0 + j < k) ? A[(int64_t)(row0 + i) * lda + k0 + j] : 0.0;
            Bs[i][j] = (k0 + i < k && col0 + j < n) ? B[(int64_t)(k0 + i) * ldb + col0 + j] : 0.0;
        }
        __syncthreads();
        for (int kk = 0; kk < GT; ++kk) {
            const double a0 = As[ty][kk], a1 = As[ty + 16][kk];
            const double b0 = Bs[kk][tx], b1 = Bs[kk][tx + 16];
            acc[0][0] = fma(a0, b0, acc[0][0]);
            acc[0][1] = fma(a0, b1, acc[0][1]);
            acc[1][0] = fma(a1, b0, acc[1][0]);
            acc[1][1] = fma(a1, b1, acc[1][1]);
        }
        __syncthreads();
    }
    for (int i = 0; i < 2; ++i)
        for (int j = 0; j < 2; ++j) {
            const int r = row0 + ty + 16 * i, c = col0 + tx + 16 * j;
            if (r < m && c < n) C[(int64_t)r * ldc + c] = acc[i][j];
        }
}

template <int L>
size_t smem_lines() { return 2 * sizeof(double2) * LineCfg<L>::LB * L + 32 * (L / 2); }   // + the twiddles
template <int L>
size_t smem_face()
{
    // two buffers of TC x L complex; L a power of two: also the staged half of the next
    // slice and the FFT's L / 2 twiddles of 32 bytes (used in double-float only; one
    // size for both, the FP64 pass leaves them unused)
    return 2 * sizeof(double2) * FaceCfg<L>::TC * L +
           (((L & (L - 1)) == 0) ? sizeof(double2) * FaceCfg<L>::TC * (L / 2) + 32 * (L / 2) : 0);
}

template <class R, int L>
cudaError_t attrs_len_r()
{
    cudaError_t e;
    const int sm = (int)smem_lines<L>();
    if ((e = cudaFuncSetAttribute(rfft_kernel<R, L>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm))) return e;
    if ((e = cudaFuncSetAttribute(face_kernel<R, L>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)smem_face<L>())))
        return e;
    if ((e = cudaFuncSetAttribute(face_invb_kernel<R, L>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)smem_invb<L>())))
        return e;
    return cudaFuncSetAttribute(face_c2r_kernel<R, L>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)smem_c2r<L>());
}
template <int L>
cudaError_t attrs_len()
{
    cudaError_t e = attrs_len_r<double, L>();
    if (e) return e;
    return attrs_len_r<ddr, L>();
}

#define IDP_LEN_SWITCH(LEN, ...)              \
    switch (LEN) {                             \
    case 16: { constexpr int L = 16; __VA_ARGS__; }   \
    case 32: { constexpr int L = 32; __VA_ARGS__; }   \
    case 48: { constexpr int L = 48; __VA_ARGS__; }   \
    case 64: { constexpr int L = 64; __VA_ARGS__; }   \
    case 96: { constexpr int L = 96; __VA_ARGS__; }   \
    case 128: { constexpr int L = 128; __VA_ARGS__; } \
    case 192: { constexpr int L = 192; __VA_ARGS__; } \
    case 256: { constexpr int L = 256; __VA_ARGS__; } \
    case 384: { constexpr int L = 384; __VA_ARGS__; } \
    case 512: { constexpr int L = 512; __VA_ARGS__; } \
    case 768: { constexpr int L = 768; __VA_ARGS__; } \
    case 1024: { constexpr int L = 1024; __VA_ARGS__; } \
    default: return cudaErrorInvalidValue;     \
    }

}  // namespace

cudaError_t boundary_set_attributes()
{
    cudaError_t e;
    if ((e = attrs_len<16>())) return e;
    if ((e = attrs_len<32>())) return e;
    if ((e = attrs_len<48>())) return e;
    if ((e = attrs_len<64>())) return e;
    if ((e = attrs_len<96>())) return e;
    if ((e = attrs_len<128>())) return e;
    if ((e = attrs_len<192>())) return e;
    if ((e = attrs_len<256>())) return e;
    if ((e = attrs_len<384>())) return e;
    if ((e = attrs_len<512>())) return e;
    if ((e = attrs_len<768>())) return e;
    return attrs_len<1024>();
}

int face_columns_per_block(int L)
{
    IDP_LEN_SWITCH(L, return FaceCfg<L>::TC;)
}

int face_blocks_per_sm(int L)
{
    int nb = 1;
    IDP_LEN_SWITCH(L, {
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, face_kernel<double, L>, NT, smem_face<L>()) !=
            cudaSuccess)
            nb = 1;
        return nb > 0 ? nb : 1;
    })
}

cudaError_t launch_rfft_pass(const RfftPass &a, cudaStream_t st)
{
    int nu, nv;
    if (a.axis == 2) { nu = a.n0; nv = a.n1; }
    else if (a.axis == 1) { nu = a.n0; nv = a.n2; }
    else { nu = a.n1; nv = a.n2; }
    IDP_LEN_SWITCH(a.P ? a.P : a.M, {
        dim3 grid((nv + LineCfg<L>::LB - 1) / LineCfg<L>::LB, nu);
        if (a.dd) rfft_kernel<ddr, L><<<grid, RfftThreads<ddr, L>::value, smem_lines<L>(), st>>>(a);
        else rfft_kernel<double, L><<<grid, RfftThreads<double, L>::value, smem_lines<L>(), st>>>(a);
        return cudaGetLastError();
    })
}

cudaError_t launch_face_pass(const FacePass &a, int nchunk, cudaStream_t st)
{
    IDP_LEN_SWITCH(2 * (a.Pb ? a.Pb : a.Mb), {
        dim3 grid((a.nc + FaceCfg<L>::TC - 1) / FaceCfg<L>::TC, nchunk);
        if (a.dd) face_kernel<ddr, L><<<grid, NT, smem_face<L>(), st>>>(a);
        else face_kernel<double, L><<<grid, NT, smem_face<L>(), st>>>(a);
        return cudaGetLastError();
    })
}

cudaError_t launch_face_pass_2d(const FacePass2D &a, cudaStream_t st)
{
    face2d_kernel<<<(a.nm + 127) / 128, 128, 0, st>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_face_inv_b(const FaceInvB &a, cudaStream_t st)
{
    IDP_LEN_SWITCH(2 * (a.Pb ? a.Pb : a.Mb), {
        dim3 grid((a.nc + InvbCfg<L>::TC - 1) / InvbCfg<L>::TC, 2);
        if (a.dd) face_invb_kernel<ddr, L><<<grid, NT, smem_invb<L>(), st>>>(a);
        else face_invb_kernel<double, L><<<grid, NT, smem_invb<L>(), st>>>(a);
        return cudaGetLastError();
    })
}

cudaError_t launch_face_c2r(const FaceC2R &a, cudaStream_t st)
{
    IDP_LEN_SWITCH(a.Pc ? a.Pc : a.Mc, {
        dim3 grid((a.nrows + C2rCfg<L>::LB - 1) / C2rCfg<L>::LB, 2);
        if (a.dd) face_c2r_kernel<ddr, L><<<grid, NT, smem_c2r<L>(), st>>>(a);
        else face_c2r_kernel<double, L><<<grid, NT, smem_c2r<L>(), st>>>(a);
        return cudaGetLastError();
    })
}

cudaError_t launch_line1d(const double *rho, double *phi, int M, double h, int mode, cudaStream_t st)
{
    line1d_kernel<<<1, L1_NT, 0, st>>>(rho, phi, M, h, mode);
    return cudaGetLastError();
}

cudaError_t launch_kernel_fill(const KernelFill &a, cudaStream_t st)
{
    kernel_fill_kernel<<<1024, 256, 0, st>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_gemm_batched(int m, int n, int k, const double *A, int64_t lda, int64_t sA,
                                const double *B, int64_t ldb, int64_t sB, double *C, int64_t ldc,
                                int64_t sC, int batch, cudaStream_t st)
{
    dim3 grid((n + GT - 1) / GT, (m + GT - 1) / GT, batch);
    gemm_kernel<<<grid, 256, 0, st>>>(m, n, k, A, lda, sA, B, ldb, sB, C, ldc, sC);
    return cudaGetLastError();
}

}  // namespace idp
