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
//    |x_i| ~ 2^-8i |x|, from x rounded to FP32); the six products with i + j <= 2 are accumulated by
//    tcgen05.mma (kind::f16, BF16 x BF16 -> FP32) in one TMEM accumulator.  The
//    dropped products are below 2^-24 relative, so the error is set by the FP32
//    accumulation.
//  * TF32X3: two TF32 pieces each (x = x0 + x1, |x1| <= 2^-11 |x|, ~22 bits
//    kept); the three products hi*hi, hi*lo, lo*hi by tcgen05.mma kind::tf32
//    (FP32 accumulation); the dropped lo*lo and the rounding of lo are ~2^-22
//    relative.
// The eigenvalue scaling and the additions of the last pass are done in FP64.
//
// Work: tiles of 128 lines x NTN modes (NTN = 128 for n <= 128, else 256, so
// that the input of a line tile is split once per 256 modes), K in stages of
// KB = 32 (BF16) or 16 (TF32) values: 8 KB per operand piece per 128 rows either
// way.  One persistent block per SM takes tiles blockIdx.x, blockIdx.x +
// gridDim.x, ... (mode tile fastest, so that the mode tiles of one line tile run
// at the same time on neighbouring SMs and share its input through L2), with
// specialised warps:
//   warps 0-15  producers: warp w owns lines 8w .. 8w+7 of a tile.  FP32 input
//               (the padded intermediates): they read the stage's values from the
//               input ring; FP64 input (node arrays whose row strides are not
//               multiples of 16 bytes, which no tensor map can describe): they load
//               them, a line of the stage per warp instruction and an 8 x 8 shuffle
//               transpose (BF16X3), the loads of the next two stages in flight while
//               a stage is split.  They split the values into pieces, store them in
//               the K-major core-matrix layout (the eight lanes of a k group write 128
//               contiguous bytes) and arrive on the stage's A barrier;
//   warp 16     copies the stage's pre-split sine image (one contiguous block per
//               (mode tile, K stage)) with one bulk asynchronous copy that
//               completes on the stage's B barrier;
//   warp 17     owns the tensor memory; one thread waits for both barriers of a
//               stage, issues its products into the tile's accumulator, commits
//               them to the stage's empty barrier (the producers' signal to refill
//               it), and after a tile's last stage commits to the accumulator's
//               full barrier;
//   warp 18     FP32 input: brings each stage's 128 lines x KB values with one 2-D
//               tensor copy (128- or 64-byte swizzle) into a ring of input slots,
//               refilled once the producer warps have read a slot;
//   warps 19-   epilogue (8 warps for FP32 input, 4 for FP64): wait for a full
//               accumulator, read it (warp w: TMEM lanes 32 (w % 4) .., half
//               (w - 19) / 4 of the columns), write the lines and release it.
// The operand stages form a ring (NS = 2-3 deep), the input slots another (NR = 2-6),
// and the accumulator is double-buffered (2 x NTN TMEM columns), so the loads, the
// products and the epilogue of consecutive tiles overlap.  Operands live in shared
// memory in the canonical K-major layout without swizzle: 8 x 16-byte core matrices
// (8 BF16 or 4 TF32 values per row), adjacent along M/N 128 bytes apart (SBO),
// adjacent along K one core column apart (LBO: 2048 bytes for the 128 rows of A, 16
// NTN bytes for the NTN rows of B); one MMA takes K = 16 (BF16) or 8 (TF32), two core
// matrices along K, in both variants.  FP64 <-> FP32 conversions and the factor 4 are
// integer operations (FP64 issue is scarce on this GPU).
//
// Every wait is bounded (clock64); a wait that runs out sets the block's failure
// flag, the other roles leave their loops at their next check, the block waits
// (bounded) for its own products and copies still in flight, frees its tensor
// memory and records the failure in *err.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cudaTypedefs.h>

#include "dd.cuh"
#include "idp_internal.cuh"

namespace idp {

namespace {

constexpr int MT = 128;            // lines per tile (MMA M)
constexpr int PIECE_BYTES = 8192;  // one operand piece of one stage per 128 rows: 128 x 64 bytes
constexpr uint32_t SBO = 128;      // core matrices adjacent along M / N
constexpr uint32_t LBO_A = 2048;   // core matrices adjacent along K, 128 rows
constexpr int NPROD = 512;         // producer threads (warps 0-15)
constexpr int WARP_COPY = 16, WARP_MMA = 17, WARP_LOAD = 18, WARP_EPI = 19;
constexpr int SMEM_LIMIT = 227 * 1024;

// per variant (0 = BF16X3, 1 = TF32X3), tile width and input type (IN64: FP64
// input, loaded by the producers; FP32 input: by tensor copies into an input ring):
// element bytes, K per stage, pieces, ring depths, epilogue warps
template <int V, int NTN, int IN64>
struct MpCfg {
    static constexpr int ESZ = V ? 4 : 2;
    static constexpr int EPC = 16 / ESZ;                  // elements per core-matrix row
    static constexpr int KB = PIECE_BYTES / (MT * ESZ);   // 32 or 16
    static constexpr int PIECES = V ? 2 : 3;
    static constexpr int A_BYTES = PIECES * PIECE_BYTES;  // A operand of one stage
    static constexpr int BP_BYTES = PIECE_BYTES * NTN / MT;   // one piece of B
    static constexpr int B_BYTES = PIECES * BP_BYTES;
    static constexpr uint32_t LBO_B = 16u * NTN;
    static constexpr int STAGE = A_BYTES + B_BYTES;
    // operand ring depth: three stages where they fit beside the input ring
    static constexpr int NS = (IN64 || STAGE <= 49152) ? (3 * STAGE <= 220 * 1024 ? 3 : 2) : 2;
    // input ring (FP32 input): one stage is the 128 lines x KB values of a tile, as
    // the tensor copy writes it (rows of KB * 4 = 128 or 64 bytes, 16-byte chunks
    // swizzled by the row so that eight rows read at one offset hit distinct banks)
    static constexpr int RAW_SLOT = IN64 ? 0 : MT * KB * 4;
    static constexpr int NR_FIT = IN64 ? 0 : (SMEM_LIMIT - 2048 - NS * STAGE) / RAW_SLOT;
    static constexpr int NR = NR_FIT > 6 ? 6 : NR_FIT;
    static_assert(IN64 || NR >= 2, "at least two input stages");
    static constexpr int NEPI = IN64 ? 4 : 8;             // epilogue warps
    static constexpr int NTHR = (WARP_EPI + NEPI) * 32;   // 736 or 864
    static constexpr int SMEM_IN = NS * STAGE;
    static constexpr int SMEM_BAR = SMEM_IN + NR * RAW_SLOT;
    // barriers: A, B, empty per operand stage; full, empty per input stage; acc full/free x2; drain
    static constexpr int NBAR = 3 * NS + 2 * NR + 5;
    static constexpr int SMEM_TOTAL = SMEM_BAR + 8 * NBAR + 16 + 1024;   // + TMEM slot + alignment
    static_assert(SMEM_TOTAL <= SMEM_LIMIT, "shared memory");
};
constexpr long long WAIT_CYCLES = 2000000000ll;       // bounded mbarrier polling (~1 s)

__device__ __forceinline__ uint32_t smem_u32(const void *p)
{
    return (uint32_t)__cvta_generic_to_shared(p);
}

// byte offset of element (row r, k) of a 128-row A piece (K-major, no swizzle)
template <int ESZ>
__device__ __forceinline__ uint32_t tile_off(int r, int k)
{
    constexpr int EPC = 16 / ESZ;
    return (uint32_t)((k / EPC) * LBO_A + (r >> 3) * SBO + (r & 7) * 16 + (k % EPC) * ESZ);
}

// shared-memory matrix descriptor: start, LBO, SBO (>> 4), version 1, no swizzle
__device__ __forceinline__ uint64_t make_desc(uint32_t saddr, uint32_t lbo)
{
    uint64_t d = 0;
    d |= (uint64_t)((saddr >> 4) & 0x3FFF);
    d |= (uint64_t)((lbo >> 4) & 0x3FFF) << 16;
    d |= (uint64_t)((SBO >> 4) & 0x3FFF) << 32;
    d |= (uint64_t)1 << 46;
    return d;
}

// FP64 -> FP32, rounded to nearest (ties away), by integer operations on the
// bits (conversions would run on the scarce FP64 pipe); |x| < 2^-126 gives 0.
// 24 bits are all that the pieces below keep of an input value.
__device__ __forceinline__ float f32_of_f64_bits(double x)
{
    const unsigned long long b = (unsigned long long)__double_as_longlong(x);
    const unsigned int hiw = (unsigned int)(b >> 32), low = (unsigned int)b;
    const int e = (int)((hiw >> 20) & 0x7FF) - 1023 + 127;
    if (e <= 0) return 0.f;
    unsigned int f = (hiw & 0x80000000u) | ((unsigned int)e << 23) | ((hiw & 0xFFFFFu) << 3) | (low >> 29);
    f += (low >> 28) & 1u;   // the carry of a round-up moves into the exponent, as it should
    return __uint_as_float(f);
}

// two floats -> packed BF16 pair, rounded to nearest even: lo in the low half
__device__ __forceinline__ uint32_t bf16x2_rn(float lo, float hi)
{
    uint32_t d;
    asm("cvt.rn.bf16x2.f32 %0, %1, %2;\n" : "=r"(d) : "f"(hi), "f"(lo));
    return d;
}
__device__ __forceinline__ float bf16_lo(uint32_t d) { return __uint_as_float(d << 16); }
__device__ __forceinline__ float bf16_hi(uint32_t d) { return __uint_as_float(d & 0xFFFF0000u); }

// x (two values at a time) -> three BF16 pieces x = a + b + c; the residuals
// x - a and r - b are exact in FP32
__device__ __forceinline__ void split3_pair(float x0, float x1, uint32_t &a, uint32_t &b, uint32_t &c)
{
    a = bf16x2_rn(x0, x1);
    const float r0 = x0 - bf16_lo(a), r1 = x1 - bf16_hi(a);
    b = bf16x2_rn(r0, r1);
    c = bf16x2_rn(r0 - bf16_lo(b), r1 - bf16_hi(b));
}

// x rounded to TF32 (to nearest, ties away); the tensor cores read the FP32 container
__device__ __forceinline__ float tf32_rna(float x)
{
    uint32_t d;
    asm("cvt.rna.tf32.f32 %0, %1;\n" : "=r"(d) : "f"(x));
    return __uint_as_float(d);
}
// x -> two TF32 pieces x = a + b (~22 bits); x - a is exact in FP32
__device__ __forceinline__ void split2(float x, float &a, float &b)
{
    a = tf32_rna(x);
    b = tf32_rna(x - a);
}

// mbarrier helpers (shared::cta addresses)
__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(bar), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint32_t bar)
{
    asm volatile("{\n .reg .b64 st;\n mbarrier.arrive.shared::cta.b64 st, [%0];\n}\n" ::"r"(bar) : "memory");
}
__device__ __forceinline__ void mbar_arrive_tx(uint32_t bar, uint32_t bytes)
{
    asm volatile("{\n .reg .b64 st;\n mbarrier.arrive.expect_tx.shared::cta.b64 st, [%0], %1;\n}\n" ::"r"(bar),
                 "r"(bytes)
                 : "memory");
}
// true once the phase of parity `parity` has completed; false after `limit` cycles
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity, long long limit)
{
    const long long t0 = clock64();
    while (true) {
        uint32_t done;
        asm volatile(
            "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
            : "=r"(done)
            : "r"(bar), "r"(parity)
            : "memory");
        if (done) return true;
        if (clock64() - t0 >= limit) return false;
    }
}
// one tensor copy global -> shared of the box at (x, y) that completes on `bar`
__device__ __forceinline__ void tma_load_2d(uint32_t dst, const CUtensorMap *map, int x, int y, uint32_t bar)
{
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], "
        "[%4];\n" ::"r"(dst),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(bar)
        : "memory");
}
// one bulk asynchronous copy global -> shared that completes on `bar`
__device__ __forceinline__ void bulk_g2s(uint32_t dst, const void *src, uint32_t bytes, uint32_t bar)
{
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];\n" ::"r"(
                     dst),
                 "l"(src), "r"(bytes), "r"(bar)
                 : "memory");
}
__device__ __forceinline__ void mma_commit(uint32_t bar)
{
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(bar)
                 : "memory");
}

template <int NTN, int V, int IN64>
__global__ void __launch_bounds__(MpCfg<V, NTN, IN64>::NTHR, 1)
    mp_pass_kernel(const MpPass a, const __grid_constant__ CUtensorMap in_map)
{
    static_assert(NTN == 128 || NTN == 256, "tile of 128 or 256 modes");
    using C = MpCfg<V, NTN, IN64>;
    constexpr int KB = C::KB, NS = C::NS, NR = C::NR, EPC = C::EPC, NEPI = C::NEPI;
    // D = F32 (bit 4); A, B = BF16 (1) for kind::f16 or TF32 (2) for kind::tf32
    constexpr uint32_t FMT = V ? 2u : 1u;
    constexpr uint32_t IDESC_N = (1u << 4) | (FMT << 7) | (FMT << 10) | ((uint32_t)(NTN >> 3) << 17) |
                                 ((uint32_t)(MT >> 4) << 24);
    extern __shared__ unsigned char sm_raw[];
    unsigned char *sm = sm_raw + ((1024u - (smem_u32(sm_raw) & 1023u)) & 1023u);
    const int t = threadIdx.x;
    const int warp = t >> 5, lane = t & 31;
    const int ntm = (a.n + NTN - 1) / NTN;               // mode tiles
    const int64_t nlines = (int64_t)a.P * a.Q;
    const int ntiles = (int)((nlines + MT - 1) / MT) * ntm;
    const int nkb = (a.n + KB - 1) / KB;
    const uint32_t bar0 = smem_u32(sm + C::SMEM_BAR);
    auto bar_a = [&](int s) { return bar0 + 8u * (uint32_t)s; };
    auto bar_b = [&](int s) { return bar0 + 8u * (uint32_t)(NS + s); };
    auto bar_e = [&](int s) { return bar0 + 8u * (uint32_t)(2 * NS + s); };
    auto bar_in = [&](int r) { return bar0 + 8u * (uint32_t)(3 * NS + r); };
    auto bar_ine = [&](int r) { return bar0 + 8u * (uint32_t)(3 * NS + NR + r); };
    auto bar_full = [&](int b) { return bar0 + 8u * (uint32_t)(3 * NS + 2 * NR + b); };
    auto bar_free = [&](int b) { return bar0 + 8u * (uint32_t)(3 * NS + 2 * NR + 2 + b); };
    const uint32_t bar_drain = bar0 + 8u * (3 * NS + 2 * NR + 4);
    auto raw_slot = [&](int r) { return sm + C::SMEM_IN + r * C::RAW_SLOT; };
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(sm + C::SMEM_BAR + 8 * C::NBAR);
    volatile __shared__ int s_fail;
    const long long limit = a.stall_test ? WAIT_CYCLES / 400 : WAIT_CYCLES;

    if (t == 0) {
        s_fail = 0;
        for (int s = 0; s < NS; ++s) {
            mbar_init(bar_a(s), NPROD / 32);   // one arrival per producer warp
            mbar_init(bar_b(s), 1);
            mbar_init(bar_e(s), 1);
        }
        for (int r = 0; r < NR; ++r) {
            mbar_init(bar_in(r), 1);
            mbar_init(bar_ine(r), NPROD / 32);
        }
        for (int b = 0; b < 2; ++b) {
            mbar_init(bar_full(b), 1);
            mbar_init(bar_free(b), NEPI);
        }
        mbar_init(bar_drain, 1);
        asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    }
    if (warp == WARP_MMA) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(
                         smem_u32(tmem_slot)),
                     "r"(2 * NTN)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
    const uint32_t tmem = *tmem_slot;

    int mma_issued = 0;
    constexpr int NARM = NS > NR ? NS : NR;
    int armed[NARM];   // copies issued per stage slot (copy and load warps)
#pragma unroll
    for (int s = 0; s < NARM; ++s) armed[s] = 0;

    if (warp < NPROD / 32) {
        // ---- producers of the input pieces: warp w owns lines 8w .. 8w+7 of a tile,
        //      lane: line r = 8w + (lane & 7), k group g8 = lane >> 3 (EPC consecutive k,
        //      one 16-byte core-matrix row per piece); the eight lanes of a k group
        //      write 128 contiguous bytes of a piece, so their stores hit distinct banks
        const int r = 8 * warp + (lane & 7), g8 = lane >> 3;
        const uint32_t oo = tile_off<C::ESZ>(r, g8 * EPC);
        int sc = 0;
        // FP64 input: loaded here, the next two stages in flight while one is split.
        // BF16X3 (KB = 32): load j of a warp reads line 8w + j of the tile, lane l its
        // value kb KB + l (a line's 256 bytes of the stage per warp instruction); the
        // eight lanes of a k group then exchange their values by shuffles (an 8 x 8
        // transpose) so that each holds its own line's EPC consecutive values.
        // TF32X3: each thread loads its own EPC values.
        int cur_lt = -1;
        bool rvalid = false;     // this thread's line (TF32X3), or line 8w of the tile (BF16X3)
        int64_t rbase = 0;       // its offset in the input
        int jwrap = 8;           // BF16X3: lines 8w + j, j >= jwrap, are in the next p (Q >= 8)
        int jlive = 8;           // BF16X3: lines 8w + j, j < jlive, exist
        int64_t pjump = 0;       // the extra offset of those lines: is_p - Q is_q
        auto load64 = [&](int tile, int kb, unsigned long long (&raw)[EPC]) {
            const int lt = tile / ntm;
            if (lt != cur_lt) {
                cur_lt = lt;
                const int64_t L = (int64_t)lt * MT + (V ? r : 8 * warp);
                rvalid = L < nlines;
                if (rvalid) {
                    const int64_t p = L / a.Q, q = L - p * a.Q;
                    rbase = p * a.is_p + q * a.is_q;
                    jwrap = (int)min((int64_t)8, (int64_t)a.Q - q);
                    jlive = (int)min((int64_t)8, nlines - L);
                    pjump = a.is_p - (int64_t)a.Q * a.is_q;
                }
            }
            if constexpr (V == 0) {
                const int k = kb * KB + lane;
                const double *src = reinterpret_cast<const double *>(a.in) + rbase + k;
#pragma unroll
                for (int j = 0; j < EPC; ++j) {
                    int64_t off = (int64_t)j * a.is_q + (j >= jwrap ? pjump : 0);
                    if (a.Q < 8) {   // the eight lines may span more than two p (small grids)
                        const int64_t Lj = (int64_t)cur_lt * MT + 8 * warp + j;
                        off = (Lj / a.Q) * a.is_p + (Lj % a.Q) * a.is_q - rbase;
                    }
                    raw[j] = (rvalid && j < jlive && k < a.n) ? (unsigned long long)__double_as_longlong(src[off])
                                                               : 0ull;
                }
            } else {
                const int kg0 = kb * KB + g8 * EPC;
                const double *src = reinterpret_cast<const double *>(a.in) + rbase + kg0;
#pragma unroll
                for (int e = 0; e < EPC; ++e)
                    raw[e] = (rvalid && kg0 + e < a.n) ? (unsigned long long)__double_as_longlong(src[e]) : 0ull;
            }
        };
        int ltile = blockIdx.x, lkb = 0;   // next stage to load (FP64 input)
        auto advance = [&](int &tl, int &k) {
            if (++k == nkb) {
                k = 0;
                tl += gridDim.x;
            }
        };
        unsigned long long q0[EPC], q1[EPC];
        if constexpr (IN64) {
            if (ltile < ntiles) load64(ltile, lkb, q0);
            advance(ltile, lkb);
            if (ltile < ntiles) load64(ltile, lkb, q1);
            advance(ltile, lkb);
        }
        // one stage: its values x (from q, or from the input ring), split, stored
        auto step = [&](int tile, int kb, unsigned long long (&q)[EPC]) -> bool {
            const int s = sc % NS;
            float x[EPC];
            if constexpr (IN64) {
#pragma unroll
                for (int e = 0; e < EPC; ++e) x[e] = f32_of_f64_bits(__longlong_as_double((long long)q[e]));
                if constexpr (V == 0) {
                    // x[j] is line 8w + j at k = kb KB + lane; after the transpose of the
                    // eight lanes' values, x[e] is line 8w + (lane & 7) at kb KB + 8 g8 + e
                    const int ai = lane & 7;
#pragma unroll
                    for (int d = 4; d >= 1; d >>= 1) {
#pragma unroll
                        for (int i = 0; i < 8; ++i) {
                            if (i & d) continue;
                            const bool up = (ai & d) != 0;
                            const float send = up ? x[i] : x[i | d];
                            const float got = __shfl_xor_sync(0xffffffffu, send, d);
                            if (up) x[i] = got;
                            else x[i | d] = got;
                        }
                    }
                }
                if (ltile < ntiles) load64(ltile, lkb, q);
                advance(ltile, lkb);
            } else {
                const int ri = sc % NR;
                if (!mbar_wait(bar_in(ri), (uint32_t)((sc / NR) & 1), limit)) s_fail = 1;
                if (s_fail) return false;
                // the tensor copy's 128-byte (BF16X3) or 64-byte (TF32X3) rows with the
                // 16-byte chunk c of row r at chunk c ^ (r % 8), or c ^ ((r / 2) % 4)
                const unsigned char *row = raw_slot(ri) + r * (KB * 4);
#pragma unroll
                for (int v = 0; v < EPC / 4; ++v) {
                    const int c = g8 * (EPC / 4) + v;
                    const int pc = V ? (c ^ ((r >> 1) & 3)) : (c ^ (r & 7));
                    const float4 f = *reinterpret_cast<const float4 *>(row + 16 * pc);
                    x[4 * v] = f.x; x[4 * v + 1] = f.y; x[4 * v + 2] = f.z; x[4 * v + 3] = f.w;
                }
                // past the line's end: the padding of the FP32 rows is written by no one
                const int kg0 = kb * KB + g8 * EPC;
#pragma unroll
                for (int e = 0; e < EPC; ++e)
                    if (kg0 + e >= a.n) x[e] = 0.f;
                // the input slot may be refilled once every producer warp has read it
                __syncwarp();
                if (lane == 0) mbar_arrive(bar_ine(ri));
            }
            if (sc >= NS && !mbar_wait(bar_e(s), (uint32_t)(((sc / NS) - 1) & 1), limit)) s_fail = 1;
            if (s_fail) return false;
            unsigned char *A = sm + s * C::STAGE;
            if constexpr (V == 1) {
                float4 va, vb;
                split2(x[0], va.x, vb.x);
                split2(x[1], va.y, vb.y);
                split2(x[2], va.z, vb.z);
                split2(x[3], va.w, vb.w);
                *reinterpret_cast<float4 *>(A + 0 * PIECE_BYTES + oo) = va;
                *reinterpret_cast<float4 *>(A + 1 * PIECE_BYTES + oo) = vb;
            } else {
                uint4 va, vb, vc;
                split3_pair(x[0], x[1], va.x, vb.x, vc.x);
                split3_pair(x[2], x[3], va.y, vb.y, vc.y);
                split3_pair(x[4], x[5], va.z, vb.z, vc.z);
                split3_pair(x[6], x[7], va.w, vb.w, vc.w);
                *reinterpret_cast<uint4 *>(A + 0 * PIECE_BYTES + oo) = va;
                *reinterpret_cast<uint4 *>(A + 1 * PIECE_BYTES + oo) = vb;
                *reinterpret_cast<uint4 *>(A + 2 * PIECE_BYTES + oo) = vc;
            }
            // the tensor cores read the pieces through the async proxy; one arrival
            // per warp (hundreds of arrivals on one barrier word would serialise)
            asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
            __syncwarp();
            if (lane == 0) mbar_arrive(bar_a(s));
            ++sc;
            return true;
        };
        // the two register sets are used in turn (a copy from one to the other
        // would wait for its loads)
        int tile = blockIdx.x, kb = 0;
        bool go = true;
        while (go && tile < ntiles && !s_fail) {
            go = step(tile, kb, q0);
            advance(tile, kb);
            if (go && tile < ntiles && !s_fail) {
                go = step(tile, kb, q1);
                advance(tile, kb);
            }
        }
    } else if (warp == WARP_LOAD) {
        // ---- FP32 input: one tensor copy per stage (the tile's 128 lines x KB values;
        //      lines past the last and values past the padded row read as zero)
        if constexpr (!IN64) if (lane == 0) {
            asm volatile("prefetch.tensormap [%0];\n" ::"l"(reinterpret_cast<uint64_t>(&in_map)) : "memory");
            int sc = 0;
            for (int tile = blockIdx.x; tile < ntiles && !s_fail; tile += gridDim.x) {
                const int y = (tile / ntm) * MT;
                for (int kb = 0; kb < nkb; ++kb, ++sc) {
                    const int ri = sc % NR;
                    if (sc >= NR && !mbar_wait(bar_ine(ri), (uint32_t)(((sc / NR) - 1) & 1), limit)) s_fail = 1;
                    if (s_fail) break;
                    mbar_arrive_tx(bar_in(ri), (uint32_t)C::RAW_SLOT);
                    tma_load_2d(smem_u32(raw_slot(ri)), &in_map, kb * KB, y, bar_in(ri));
                    ++armed[ri];
                }
            }
        }
    } else if (warp == WARP_COPY) {
        // ---- the sine image: one bulk copy per stage ----
        if (lane == 0) {
            int sc = 0;
            for (int tile = blockIdx.x; tile < ntiles && !s_fail; tile += gridDim.x) {
                const int mt = tile % ntm;
                for (int kb = 0; kb < nkb; ++kb, ++sc) {
                    const int s = sc % NS;
                    if (sc >= NS && !mbar_wait(bar_e(s), (uint32_t)(((sc / NS) - 1) & 1), limit)) s_fail = 1;
                    if (s_fail) break;
                    const unsigned char *src = reinterpret_cast<const unsigned char *>(a.bimg) +
                                               ((int64_t)mt * nkb + kb) * C::B_BYTES;
                    mbar_arrive_tx(bar_b(s), (uint32_t)C::B_BYTES);
                    bulk_g2s(smem_u32(sm + s * C::STAGE + C::A_BYTES), src, (uint32_t)C::B_BYTES, bar_b(s));
                    ++armed[s];
                }
            }
        }
    } else if (warp == WARP_MMA) {
        // ---- the products ----
        if (lane == 0) {
            int sc = 0, ac = 0;
            constexpr int NPR = V ? 3 : 6;
            const int pa[6] = {0, 0, 1, 0, 1, 2};
            const int pb[6] = {0, 1, 0, 2, 1, 0};
            for (int tile = blockIdx.x; tile < ntiles && !s_fail; tile += gridDim.x, ++ac) {
                const int buf = ac & 1;
                // the epilogue must have emptied this accumulator (two tiles ago)
                if (ac >= 2 && !mbar_wait(bar_free(buf), (uint32_t)(((ac >> 1) - 1) & 1), limit)) s_fail = 1;
                if (s_fail) break;
                asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
                const uint32_t d = tmem + (uint32_t)(buf * NTN);
                for (int kb = 0; kb < nkb; ++kb, ++sc) {
                    const int s = sc % NS;
                    const uint32_t ph = (uint32_t)((sc / NS) & 1);
                    if (!mbar_wait(bar_a(s), ph, limit) || !mbar_wait(bar_b(s), ph, limit)) s_fail = 1;
                    if (s_fail) break;
                    asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
                    if (a.stall_test) continue;   // test hook: no products, so the waits run out
                    // products (i, j) with i + j <= 2 (BF16X3) or <= 1 (TF32X3); one
                    // MMA per two core matrices along K
                    const uint32_t sa = smem_u32(sm + s * C::STAGE), sb = sa + (uint32_t)C::A_BYTES;
#pragma unroll
                    for (int pr = 0; pr < NPR; ++pr) {
#pragma unroll
                        for (int ks = 0; ks < KB / (2 * EPC); ++ks) {
                            const uint64_t ad = make_desc(sa + pa[pr] * PIECE_BYTES + ks * 2 * LBO_A, LBO_A);
                            const uint64_t bd = make_desc(sb + pb[pr] * C::BP_BYTES + ks * 2 * C::LBO_B, C::LBO_B);
                            const uint32_t acc = (kb > 0 || pr > 0 || ks > 0) ? 1u : 0u;
                            if constexpr (V == 1)
                                asm volatile(
                                    "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
                                    " tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(d),
                                    "l"(ad), "l"(bd), "r"(IDESC_N), "r"(acc)
                                    : "memory");
                            else
                                asm volatile(
                                    "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
                                    " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(d),
                                    "l"(ad), "l"(bd), "r"(IDESC_N), "r"(acc)
                                    : "memory");
                        }
                    }
                    mma_issued = 1;
                    mma_commit(bar_e(s));   // the stage is free once these products have read it
                }
                if (s_fail) break;
                if (!a.stall_test) mma_commit(bar_full(buf));   // the tile's accumulator is complete
            }
        }
    } else {
        // ---- epilogue: warp w reads TMEM lane quadrant w % 4 (lines 32 (w % 4) ..),
        //      half (w - WARP_EPI) / 4 of the columns
        constexpr int CPW = NTN / (NEPI / 4);   // columns per epilogue warp
        const int quad = warp & 3, half = (warp - WARP_EPI) >> 2;
        const int emode = (a.tab ? 1 : 0) | (a.add ? 2 : 0);   // FP64 operands of the epilogue
        int ac = 0;
        for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x, ++ac) {
            const int buf = ac & 1;
            // a warp-uniform decision: the TMEM loads below are warp-collective
            bool ok = !s_fail;
            if (ok) ok = mbar_wait(bar_full(buf), (uint32_t)((ac >> 1) & 1), limit);
            ok = __all_sync(0xffffffffu, ok) != 0;
            if (!ok) {
                s_fail = 1;
                break;
            }
            asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
            const int64_t L = (int64_t)(tile / ntm) * MT + 32 * quad + lane;
            const int m0 = (tile % ntm) * NTN;
            const bool live = L < nlines;
            int64_t ob = 0, tb = 0, ab = 0;   // this line's offsets in out, tab, add
            if (live) {
                const int64_t p = L / a.Q, q = L - p * a.Q;
                ob = p * a.os_p + q * a.os_q;
                tb = p * a.ts_p + q * a.ts_q;
                ab = p * a.as_p + q * a.as_q;
            }
            const int cols = min(NTN, ((a.n - m0 + 15) / 16) * 16);
            for (int c0 = half * CPW; c0 < min(cols, (half + 1) * CPW); c0 += 16) {
                uint32_t v[16];
                const uint32_t taddr = tmem + ((uint32_t)(32 * quad) << 16) + (uint32_t)(buf * NTN + c0);
                asm volatile(
                    "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, "
                    "[%16];\n"
                    : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]),
                      "=r"(v[7]), "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]),
                      "=r"(v[14]), "=r"(v[15])
                    : "r"(taddr));
                asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
                if (!live) continue;
                const int mc = m0 + c0;
                const int nj = min(16, a.n - mc);
                if (a.out_f64) {
                    double *o = reinterpret_cast<double *>(a.out) + ob + (int64_t)mc * a.os_m;
                    // 4 * the FP32 sum, exact in FP32, widened to FP64 by bits; the FP64
                    // operands, if any, in groups of 8 modes whose loads go out before
                    // any store (the stores could alias them as far as the compiler
                    // knows, and would otherwise put one load latency on every value).
                    // One loop per operand case: a select between the cases would run
                    // their FP64 arithmetic on every value.
                    if (emode == 0) {
#pragma unroll
                        for (int j = 0; j < 16; ++j) {
                            if (j >= nj) break;
                            o[(int64_t)j * a.os_m] = f2d_bits(__fmul_rn(4.0f, __uint_as_float(v[j])));
                        }
                    } else {
                        const double *tp = a.tab ? a.tab + tb + (int64_t)mc * a.ts_m : nullptr;
                        const double *ap = a.add ? a.add + ab + (int64_t)mc * a.as_m : nullptr;
#pragma unroll
                        for (int h = 0; h < 16; h += 8) {
                            double tv[8], av[8];
#pragma unroll
                            for (int j = 0; j < 8; ++j) {
                                tv[j] = (emode & 1) && h + j < nj ? tp[(int64_t)(h + j) * a.ts_m] : 1.0;
                                av[j] = (emode & 2) && h + j < nj ? ap[(int64_t)(h + j) * a.as_m] : 0.0;
                            }
                            if (emode == 1) {
#pragma unroll
                                for (int j = 0; j < 8; ++j) {
                                    if (h + j >= nj) break;
                                    o[(int64_t)(h + j) * a.os_m] =
                                        tv[j] * f2d_bits(__fmul_rn(4.0f, __uint_as_float(v[h + j])));
                                }
                            } else if (emode == 2) {
#pragma unroll
                                for (int j = 0; j < 8; ++j) {
                                    if (h + j >= nj) break;
                                    o[(int64_t)(h + j) * a.os_m] =
                                        f2d_bits(__fmul_rn(4.0f, __uint_as_float(v[h + j]))) + av[j];
                                }
                            } else {
#pragma unroll
                                for (int j = 0; j < 8; ++j) {
                                    if (h + j >= nj) break;
                                    o[(int64_t)(h + j) * a.os_m] =
                                        fma(tv[j], f2d_bits(__fmul_rn(4.0f, __uint_as_float(v[h + j]))), av[j]);
                                }
                            }
                        }
                    }
                } else {
                    float *o = reinterpret_cast<float *>(a.out) + ob + (int64_t)mc * a.os_m;
#pragma unroll
                    for (int j = 0; j < 16; ++j) {
                        if (j >= nj) break;
                        o[(int64_t)j * a.os_m] = __fmul_rn(4.0f, __uint_as_float(v[j]));
                    }
                }
            }
            // the accumulator may be reused once every warp of the epilogue has read it
            asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
            __syncwarp();
            if (lane == 0) mbar_arrive(bar_free(buf));
        }
    }

    // ---- teardown: after a failure, wait (bounded) for this block's own products
    //      and copies still in flight before the tensor memory is freed and the
    //      shared memory released
    __syncthreads();
    const bool failed = s_fail != 0;
    if (failed) {
        if (warp == WARP_MMA && lane == 0 && mma_issued) {
            mma_commit(bar_drain);   // arrives once every product issued so far has completed
            mbar_wait(bar_drain, 0, WAIT_CYCLES);
        }
        if (warp == WARP_COPY && lane == 0) {
#pragma unroll
            for (int s = 0; s < NS; ++s)
                if (armed[s] > 0) mbar_wait(bar_b(s), (uint32_t)((armed[s] - 1) & 1), WAIT_CYCLES);
        }
        if (warp == WARP_LOAD && lane == 0) {
#pragma unroll
            for (int r = 0; r < NR; ++r)
                if (armed[r] > 0) mbar_wait(bar_in(r), (uint32_t)((armed[r] - 1) & 1), WAIT_CYCLES);
        }
        if (t == 0 && a.err) atomicExch(a.err, 1);
    }
    asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
    __syncthreads();
    if (warp == WARP_MMA) {
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem), "r"(2 * NTN)
                     : "memory");
    }
}

int g_num_sms = 0;
PFN_cuTensorMapEncodeTiled_v12000 g_encode = nullptr;

template <int V, int NTN, int IN64>
cudaError_t launch_mp_t(const MpPass &a, cudaStream_t st)
{
    using C = MpCfg<V, NTN, IN64>;
    const int64_t lines = (int64_t)a.P * a.Q;
    const int64_t tiles = ((lines + MT - 1) / MT) * ((a.n + NTN - 1) / NTN);
    if (tiles >= (1ll << 31)) return cudaErrorInvalidValue;
    CUtensorMap map;
    memset(&map, 0, sizeof(map));
    if (!IN64) {
        // FP32 input: lines at a uniform stride (is_p = Q is_q), rows of pad4(n) values
        if (!g_encode) return cudaErrorInitializationError;
        const cuuint64_t dim[2] = {(cuuint64_t)((a.n + 3) & ~3), (cuuint64_t)lines};
        const cuuint64_t stride[1] = {(cuuint64_t)a.is_q * 4u};
        const cuuint32_t box[2] = {(cuuint32_t)C::KB, (cuuint32_t)MT};
        const cuuint32_t estr[2] = {1, 1};
        const CUresult r = g_encode(&map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<void *>(a.in), dim, stride,
                                    box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                                    V ? CU_TENSOR_MAP_SWIZZLE_64B : CU_TENSOR_MAP_SWIZZLE_128B,
                                    CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
        if (r != CUDA_SUCCESS) return cudaErrorInvalidValue;
    }
    const int sms = g_num_sms > 0 ? g_num_sms : 148;
    const unsigned grid = (unsigned)(tiles < sms ? tiles : sms);
    mp_pass_kernel<NTN, V, IN64><<<grid, C::NTHR, C::SMEM_TOTAL, st>>>(a, map);
    return cudaGetLastError();
}

template <int V, int NTN, int IN64>
cudaError_t mp_attr()
{
    return cudaFuncSetAttribute(mp_pass_kernel<NTN, V, IN64>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                MpCfg<V, NTN, IN64>::SMEM_TOTAL);
}

}  // namespace

cudaError_t mp_set_attributes()
{
    cudaError_t e;
    if ((e = mp_attr<0, 128, 0>()) != cudaSuccess || (e = mp_attr<0, 128, 1>()) != cudaSuccess ||
        (e = mp_attr<0, 256, 0>()) != cudaSuccess || (e = mp_attr<0, 256, 1>()) != cudaSuccess ||
        (e = mp_attr<1, 128, 0>()) != cudaSuccess || (e = mp_attr<1, 128, 1>()) != cudaSuccess ||
        (e = mp_attr<1, 256, 0>()) != cudaSuccess || (e = mp_attr<1, 256, 1>()) != cudaSuccess)
        return e;
    if (!g_encode) {
        void *fn = nullptr;
        cudaDriverEntryPointQueryResult q;
        if ((e = cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q)) !=
            cudaSuccess)
            return e;
        if (q != cudaDriverEntryPointSuccess || !fn) return cudaErrorNotSupported;
        g_encode = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
    }
    int dev = 0;
    if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
    return cudaDeviceGetAttribute(&g_num_sms, cudaDevAttrMultiProcessorCount, dev);
}

int mp_stage_k(int variant) { return variant ? MpCfg<1, 128, 0>::KB : MpCfg<0, 128, 0>::KB; }
int mp_tile_modes(int n) { return n <= 128 ? 128 : 256; }

cudaError_t launch_mp_pass(const MpPass &a, cudaStream_t st)
{
    // the input is read along a contiguous axis; FP32 input: 16-byte aligned lines
    // padded to whole 16-byte vectors, at one stride (is_p = Q is_q, or P = 1)
    if (a.is_k != 1) return cudaErrorInvalidValue;
    if (!a.in_f64 && (!a.in_vec4 || (reinterpret_cast<uintptr_t>(a.in) & 15u) || (a.is_q & 3) ||
                      (a.P > 1 && a.is_p != (int64_t)a.Q * a.is_q)))
        return cudaErrorInvalidValue;
    const bool w128 = mp_tile_modes(a.n) == 128;
    if (a.variant) {
        if (w128) return a.in_f64 ? launch_mp_t<1, 128, 1>(a, st) : launch_mp_t<1, 128, 0>(a, st);
        return a.in_f64 ? launch_mp_t<1, 256, 1>(a, st) : launch_mp_t<1, 256, 0>(a, st);
    }
    if (w128) return a.in_f64 ? launch_mp_t<0, 128, 1>(a, st) : launch_mp_t<0, 128, 0>(a, st);
    return a.in_f64 ? launch_mp_t<0, 256, 1>(a, st) : launch_mp_t<0, 256, 0>(a, st);
}

}  // namespace idp
