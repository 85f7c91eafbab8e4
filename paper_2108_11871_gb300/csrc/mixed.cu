// Mixed-precision sine-transform pass on the 5th-generation tensor cores.
//
// One pass transforms every line of an array along its contiguous axis:
//     Y[m][L] = 4 * sum_k S[m][k] X[L][k],   S[m][k] = sin(pi (m+1)(k+1) / M),
// with lines L = p*Q + q read from a strided view and the result written with
// the transformed axis outermost (the pass rotates the axes; three passes of
// a 3-D transform, two of a 2-D one, return to the original layout).
//
// Precision, two variants:
//  * BF16X3: X and S are split into three BF16 pieces each (x = x0 + x1 + x2,
//    |x_i| ~ 2^-8i |x|); the six products with i + j <= 2 are accumulated by
//    tcgen05.mma (kind::f16, BF16 x BF16 -> FP32) in one TMEM accumulator.  The
//    dropped products are below 2^-24 relative, so the error is set by the FP32
//    accumulation.
//  * TF32X3: two TF32 pieces each (x = x0 + x1, |x1| <= 2^-11 |x|, ~22 bits
//    kept); the three products hi*hi, hi*lo, lo*hi by tcgen05.mma kind::tf32
//    (FP32 accumulation); the dropped lo*lo and the rounding of lo are ~2^-22
//    relative.
// The eigenvalue scaling and the additions of the last pass are done in FP64.
//
// Block: 512 threads, a tile of 128 lines x NTN modes (NTN = 64 or 128), K in
// blocks of 64 (BF16) or 32 (TF32): 16 KB per operand piece either way.
// Operands live in shared memory in the canonical K-major layout without
// swizzle: 8 x 16-byte core matrices (8 BF16 or 4 TF32 values per row), core
// matrices adjacent along K are LBO = 2048 bytes apart, adjacent along M/N
// SBO = 128 bytes apart; one MMA takes K = 16 (BF16) or 8 (TF32), two core
// matrices along K, in both variants.  The sine
// image of a K block (128 modes) arrives by cp.async while the block loads and
// splits its input; a 64-mode tile addresses its half of the image through the
// descriptor's start address.  FP64 <-> FP32 conversions and the factor 4 are
// integer operations (FP64 issue is scarce on this GPU).
#include <cuda_bf16.h>

#include "dd.cuh"
#include "idp_internal.cuh"

namespace idp {

namespace {

constexpr int MT = 128;            // lines per tile (MMA M)
constexpr int NTILE = 128;         // modes per tile (MMA N)
constexpr int TILE_BYTES = 16384;  // one operand piece: 128 rows x 16 core-matrix columns
constexpr uint32_t LBO = 2048, SBO = 128;

// per variant (0 = BF16X3, 1 = TF32X3): element bytes, K per block, pieces
template <int V>
struct MpCfg {
    static constexpr int ESZ = V ? 4 : 2;
    static constexpr int EPC = 16 / ESZ;                 // elements per core-matrix row
    static constexpr int KB = TILE_BYTES / (MT * ESZ);   // 64 or 32
    static constexpr int PIECES = V ? 2 : 3;
    static constexpr int SMEM_A = 0;
    static constexpr int SMEM_B = PIECES * TILE_BYTES;
    static constexpr int SMEM_BAR = 2 * PIECES * TILE_BYTES;   // mbarrier (8 B) + TMEM address (4 B)
    static constexpr int SMEM_TOTAL = SMEM_BAR + 64;
};
constexpr long long WAIT_CYCLES = 2000000000ll;       // bounded mbarrier polling (~1 s)

__device__ __forceinline__ uint32_t smem_u32(const void *p)
{
    return (uint32_t)__cvta_generic_to_shared(p);
}

// byte offset of element (row r, k) of a 128-row tile (K-major, no swizzle)
template <int V>
__device__ __forceinline__ uint32_t tile_off(int r, int k)
{
    using C = MpCfg<V>;
    return (uint32_t)((k / C::EPC) * LBO + (r >> 3) * SBO + (r & 7) * 16 + (k % C::EPC) * C::ESZ);
}

// shared-memory matrix descriptor: start, LBO, SBO (>> 4), version 1, no swizzle
__device__ __forceinline__ uint64_t make_desc(uint32_t saddr)
{
    uint64_t d = 0;
    d |= (uint64_t)((saddr >> 4) & 0x3FFF);
    d |= (uint64_t)((LBO >> 4) & 0x3FFF) << 16;
    d |= (uint64_t)((SBO >> 4) & 0x3FFF) << 32;
    d |= (uint64_t)1 << 46;
    return d;
}

// instruction descriptor (D = F32, A = B = BF16 for kind::f16 or TF32 for
// kind::tf32, K-major, M = 128, N = NTN): built in the kernel from the tile width

// x rounded to TF32 (11 significant bits, to nearest, ties to even), by integer
// operations; the tensor cores read these FP32 containers unchanged
__device__ __forceinline__ float tf32_rn(float x)
{
    const uint32_t u = __float_as_uint(x);
    return __uint_as_float((u + 0xFFFu + ((u >> 13) & 1u)) & 0xFFFFE000u);
}

// x = hi + lo (two floats) -> two TF32 pieces; hi - a is exact in FP32
__device__ __forceinline__ void split2(float hi, float lo, float &a, float &b)
{
    a = tf32_rn(hi);
    b = tf32_rn((hi - a) + lo);
}

// x = hi + lo (two floats, |lo| <= 2^-24 |hi|) -> three BF16 pieces.  The
// residuals hi - a and r1 - b are exact in FP32; lo enters below 2^-16 |x|.
__device__ __forceinline__ void split3(float hi, float lo, unsigned short &a, unsigned short &b,
                                       unsigned short &c)
{
    const __nv_bfloat16 ba = __float2bfloat16_rn(hi);
    const float r1 = (hi - __bfloat162float(ba)) + lo;
    const __nv_bfloat16 bb = __float2bfloat16_rn(r1);
    const float r2 = r1 - __bfloat162float(bb);
    const __nv_bfloat16 bc = __float2bfloat16_rn(r2);
    a = __bfloat16_as_ushort(ba);
    b = __bfloat16_as_ushort(bb);
    c = __bfloat16_as_ushort(bc);
}

__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity, long long limit)
{
    const long long t0 = clock64();
    while (clock64() - t0 < limit) {
        uint32_t done;
        asm volatile(
            "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
            : "=r"(done)
            : "r"(bar), "r"(parity)
            : "memory");
        if (done) return true;
    }
    return false;
}

constexpr int NTHR = 512;
constexpr int GPT = MT * (TILE_BYTES / MT / 16) / NTHR;   // 16-byte core-matrix rows of the A tile per thread (2)

__device__ __forceinline__ void cp_async16(uint32_t dst, const void *src)
{
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(dst), "l"(src) : "memory");
}

template <int NTN, int V>
__global__ void __launch_bounds__(NTHR) mp_pass_kernel(const MpPass a)
{
    static_assert(NTN == 64 || NTN == 128, "tile of 64 or 128 modes");
    using C = MpCfg<V>;
    constexpr int KB = C::KB, PIECES = C::PIECES, SMEM_A = C::SMEM_A, SMEM_B = C::SMEM_B, SMEM_BAR = C::SMEM_BAR;
    constexpr int EPC = C::EPC;
    // D = F32 (bit 4); A, B = BF16 (1) for kind::f16 or TF32 (2) for kind::tf32
    constexpr uint32_t FMT = V ? 2u : 1u;
    constexpr uint32_t IDESC_N = (1u << 4) | (FMT << 7) | (FMT << 10) | ((uint32_t)(NTN >> 3) << 17) |
                                 ((uint32_t)(MT >> 4) << 24);
    extern __shared__ __align__(128) unsigned char sm[];
    const int t = threadIdx.x;
    const int warp = t >> 5, lane = t & 31;
    const int64_t nlines = (int64_t)a.P * a.Q;
    const int64_t L0 = (int64_t)blockIdx.x * MT;
    const int m0 = blockIdx.y * NTN;
    const int img_tile = m0 / NTILE;                                   // 128-mode image tile
    const uint32_t b_sub = (uint32_t)(((m0 - img_tile * NTILE) >> 3) * SBO);   // byte offset of the half
    const int nkb = (a.n + KB - 1) / KB;
    const uint32_t bar = smem_u32(sm + SMEM_BAR);
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(sm + SMEM_BAR + 8);
    __shared__ int s_fail;

    if (t == 0) {
        s_fail = 0;
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(bar) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(
                         smem_u32(tmem_slot)),
                     "r"(NTN)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
    const uint32_t tmem = *tmem_slot;

    for (int kb = 0; kb < nkb; ++kb) {
        // B pieces: the pre-split sine image of this K block, copied asynchronously
        {
            const unsigned char *src = reinterpret_cast<const unsigned char *>(a.bimg) +
                                       ((int64_t)img_tile * nkb + kb) * (PIECES * TILE_BYTES);
            const uint32_t dst = smem_u32(sm + SMEM_B);
            for (int e = t; e < PIECES * TILE_BYTES / 16; e += NTHR) cp_async16(dst + 16 * e, src + 16 * e);
            asm volatile("cp.async.commit_group;\n" ::: "memory");
        }
        // A pieces: 128 lines x KB k of the input, split into pieces; a thread
        // takes GPT groups of EPC consecutive k of one line (one 16-byte
        // core-matrix row each; consecutive lanes take consecutive lines, so a
        // warp's stores fill 512 contiguous bytes), all loads issued before any
        // is used
        double xv[GPT][EPC];
#pragma unroll
        for (int g = 0; g < GPT; ++g) {
            const int e = t + g * NTHR;
            const int r = e & (MT - 1), g8 = e / MT;   // rows fastest: conflict-free 16-byte stores
            const int64_t L = L0 + r;
            const int kg0 = kb * KB + g8 * EPC;
            const bool row_ok = L < nlines;
            int64_t base = 0;
            if (row_ok) {
                const int64_t p = L / a.Q, q = L - p * a.Q;
                base = p * a.is_p + q * a.is_q;
            }
#pragma unroll
            for (int j = 0; j < EPC; ++j) {
                const int kg = kg0 + j;
                double x = 0.0;
                if (row_ok && kg < a.n) {
                    const int64_t off = base + (int64_t)kg * a.is_k;
                    if (a.in_f64) x = reinterpret_cast<const double *>(a.in)[off];
                    else x = __longlong_as_double((long long)__float_as_int(reinterpret_cast<const float *>(a.in)[off]));
                }
                xv[g][j] = x;
            }
        }
#pragma unroll
        for (int g = 0; g < GPT; ++g) {
            const int e = t + g * NTHR;
            const int r = e & (MT - 1), g8 = e / MT;   // rows fastest: conflict-free 16-byte stores
            float hi[EPC], lo[EPC];
#pragma unroll
            for (int j = 0; j < EPC; ++j) {
                if (a.in_f64) {
                    const ddr h2 = dd_from_bits(xv[g][j]);   // integer split, no FP64 instruction
                    hi[j] = h2.hi;
                    lo[j] = h2.lo;
                } else {
                    hi[j] = __int_as_float((int)__double_as_longlong(xv[g][j]));
                    lo[j] = 0.f;
                }
            }
            const uint32_t o = tile_off<V>(r, g8 * EPC);
            if constexpr (V == 1) {
                float4 va, vb;
                split2(hi[0], lo[0], va.x, vb.x);
                split2(hi[1], lo[1], va.y, vb.y);
                split2(hi[2], lo[2], va.z, vb.z);
                split2(hi[3], lo[3], va.w, vb.w);
                *reinterpret_cast<float4 *>(sm + SMEM_A + 0 * TILE_BYTES + o) = va;
                *reinterpret_cast<float4 *>(sm + SMEM_A + 1 * TILE_BYTES + o) = vb;
            } else {
                unsigned short pa[8], pb[8], pc[8];
#pragma unroll
                for (int j = 0; j < 8; ++j) split3(hi[j], lo[j], pa[j], pb[j], pc[j]);
                uint4 va, vb, vc;
                va.x = pa[0] | ((uint32_t)pa[1] << 16); va.y = pa[2] | ((uint32_t)pa[3] << 16);
                va.z = pa[4] | ((uint32_t)pa[5] << 16); va.w = pa[6] | ((uint32_t)pa[7] << 16);
                vb.x = pb[0] | ((uint32_t)pb[1] << 16); vb.y = pb[2] | ((uint32_t)pb[3] << 16);
                vb.z = pb[4] | ((uint32_t)pb[5] << 16); vb.w = pb[6] | ((uint32_t)pb[7] << 16);
                vc.x = pc[0] | ((uint32_t)pc[1] << 16); vc.y = pc[2] | ((uint32_t)pc[3] << 16);
                vc.z = pc[4] | ((uint32_t)pc[5] << 16); vc.w = pc[6] | ((uint32_t)pc[7] << 16);
                *reinterpret_cast<uint4 *>(sm + SMEM_A + 0 * TILE_BYTES + o) = va;
                *reinterpret_cast<uint4 *>(sm + SMEM_A + 1 * TILE_BYTES + o) = vb;
                *reinterpret_cast<uint4 *>(sm + SMEM_A + 2 * TILE_BYTES + o) = vc;
            }
        }
        asm volatile("cp.async.wait_group 0;\n" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
        __syncthreads();
        if (t == 0 && !a.stall_test) {
            asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
            // products (i, j) with i + j <= 2 (BF16X3) or <= 1 (TF32X3); one
            // MMA per two core matrices along K
            constexpr int NPR = V ? 3 : 6;
            const int pa[6] = {0, 0, 1, 0, 1, 2};
            const int pb[6] = {0, 1, 0, 2, 1, 0};
            for (int pr = 0; pr < NPR; ++pr) {
                for (int ks = 0; ks < KB / (2 * EPC); ++ks) {
                    const uint64_t ad = make_desc(smem_u32(sm + SMEM_A + pa[pr] * TILE_BYTES) + ks * 2 * LBO);
                    const uint64_t bd =
                        make_desc(smem_u32(sm + SMEM_B + pb[pr] * TILE_BYTES) + ks * 2 * LBO + b_sub);
                    const uint32_t acc = (kb > 0 || pr > 0 || ks > 0) ? 1u : 0u;
                    if constexpr (V == 1)
                        asm volatile(
                            "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
                            " tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem),
                            "l"(ad), "l"(bd), "r"(IDESC_N), "r"(acc)
                            : "memory");
                    else
                        asm volatile(
                            "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
                            " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem),
                            "l"(ad), "l"(bd), "r"(IDESC_N), "r"(acc)
                            : "memory");
                }
            }
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(
                             bar)
                         : "memory");
        }
        // every thread waits for the products (they read the shared memory we refill next)
        // (stall_test: no products were issued, so this wait runs out on purpose)
        if (!mbar_wait(bar, (uint32_t)(kb & 1), a.stall_test ? WAIT_CYCLES / 400 : WAIT_CYCLES)) s_fail = 1;
        asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
        __syncthreads();
        if (s_fail) break;
    }

    if (!s_fail) {
        // epilogue: warp w reads TMEM lane quadrant w % 4 (lines 32*(w%4) ..),
        // columns [NTN/4 * (w / 4), NTN/4 * (w / 4) + NTN/4), 16 at a time
        const int quad = warp & 3;
        const int64_t L = L0 + 32 * quad + lane;
        const bool live = L < nlines;
        int64_t p = 0, q = 0;
        if (live) { p = L / a.Q; q = L - p * a.Q; }
        constexpr int CPW = NTN / 4;
        for (int c0 = CPW * (warp >> 2); c0 < CPW * (warp >> 2) + CPW; c0 += 16) {
            uint32_t v[16];
            const uint32_t taddr = tmem + ((uint32_t)(32 * quad) << 16) + (uint32_t)c0;
            asm volatile(
                "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, "
                "[%16];\n"
                : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]),
                  "=r"(v[7]), "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]),
                  "=r"(v[14]), "=r"(v[15])
                : "r"(taddr));
            asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
            if (!live) continue;
#pragma unroll
            for (int j = 0; j < 16; ++j) {
                const int m = m0 + c0 + j;
                if (m >= a.n) break;
                // 4 * the FP32 sum, exact in FP32; widened to FP64 by bits
                const float y4 = __fmul_rn(4.0f, __uint_as_float(v[j]));
                const int64_t oo = (int64_t)m * a.os_m + p * a.os_p + q * a.os_q;
                if (a.out_f64) {
                    const double y = f2d_bits(y4);
                    double r = y;
                    if (a.tab) {
                        const double tv = a.tab[(int64_t)m * a.ts_m + p * a.ts_p + q * a.ts_q];
                        r = a.add ? fma(tv, y, a.add[(int64_t)m * a.as_m + p * a.as_p + q * a.as_q]) : tv * y;
                    } else if (a.add) {
                        r = y + a.add[(int64_t)m * a.as_m + p * a.as_p + q * a.as_q];
                    }
                    reinterpret_cast<double *>(a.out)[oo] = r;
                } else {
                    reinterpret_cast<float *>(a.out)[oo] = y4;
                }
            }
        }
    } else if (t == 0 && a.err) {
        atomicExch(a.err, 1);
    }
    asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
    __syncthreads();
    if (warp == 0) {
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem), "r"(NTN)
                     : "memory");
    }
}

}  // namespace

cudaError_t mp_set_attributes()
{
    cudaError_t e;
    if ((e = cudaFuncSetAttribute(mp_pass_kernel<128, 0>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  MpCfg<0>::SMEM_TOTAL)) != cudaSuccess ||
        (e = cudaFuncSetAttribute(mp_pass_kernel<64, 0>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  MpCfg<0>::SMEM_TOTAL)) != cudaSuccess ||
        (e = cudaFuncSetAttribute(mp_pass_kernel<128, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  MpCfg<1>::SMEM_TOTAL)) != cudaSuccess)
        return e;
    return cudaFuncSetAttribute(mp_pass_kernel<64, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                MpCfg<1>::SMEM_TOTAL);
}

template <int V>
cudaError_t launch_mp_v(const MpPass &a, cudaStream_t st)
{
    const int64_t lines = (int64_t)a.P * a.Q;
    const unsigned tiles = (unsigned)((lines + MT - 1) / MT);
    // 64-mode tiles double the blocks of a launch that fills the GPU less than twice
    if (a.modes_per_tile == 64 || (a.modes_per_tile == 0 && tiles * ((a.n + NTILE - 1) / NTILE) < 2 * 152)) {
        mp_pass_kernel<64, V><<<dim3(tiles, (unsigned)((a.n + 63) / 64)), NTHR, MpCfg<V>::SMEM_TOTAL, st>>>(a);
    } else {
        mp_pass_kernel<128, V>
            <<<dim3(tiles, (unsigned)((a.n + NTILE - 1) / NTILE)), NTHR, MpCfg<V>::SMEM_TOTAL, st>>>(a);
    }
    return cudaGetLastError();
}

cudaError_t launch_mp_pass(const MpPass &a, cudaStream_t st)
{
    return a.variant ? launch_mp_v<1>(a, st) : launch_mp_v<0>(a, st);
}

}  // namespace idp
