// Internal declarations shared by the CUDA translation units of libidp.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace idp {

// One twiddle factor w = c + i s stored for the FMA butterfly
//   A = a + w b,  B = a - w b
// with the ratio form w b = m ((P - r Q) + i (Q + r P)) (real part scaled by
// mre, imaginary by mim), where (P, Q) = (b.re, b.im) if |c| >= |s| and
// (b.im, b.re) otherwise; |r| <= 1 in both cases.
struct Tw {
    double r, mre, mim;
    int swap, pad;
};

// Tables for one complex FFT length L (power of two): forward and inverse
// twiddles e^{-+2 pi i j / L}, j < L/2, and the real-transform post/pre
// twiddles e^{-i pi k / L}, k <= L (cos, sin pairs).
struct TwD;
struct ddc;
struct ddr;
struct FftTables {
    int L;
    const Tw *fwd;      // device, L/2 entries
    const Tw *inv;      // device, L/2 entries
    const double2 *half; // device, L+1 entries: (cos(pi k/L), -sin(pi k/L))
    const Tw *halfr;     // device, L+1 entries: the same in ratio form
    const TwD *fwdd;    // double-float forms of the three tables
    const TwD *invd;
    const ddc *halfd;
};

// Strided 3-D view in units of elements: element (i0,i1,i2) at base + i0*s0 + i1*s1 + i2*s2.
struct View3 {
    double *p;
    int64_t s0, s1, s2;
};

// One sine-transform pass along `axis` of an interior-index box n0 x n1 x n2
// (every extent along `axis` equals M-1).  Each line x -> U with U = 4 * S x,
// S_{k,i} = sin(pi k i / M); then the epilogue
//     out = (tab ? tab * U : U) + (add ? add : 0)
// with tab laid out densely over the box and `add` a strided view.
struct DstPass {
    View3 in, out, add;
    const double *tab;
    int n0, n1, n2;
    int axis;
    int M;
    const Tw *tw;          // twiddles for the complex FFT of length M/2
    const double2 *half;   // half-step twiddles for length M/2 (e^{-i pi k/(M/2)})
    const Tw *halfr;       // the same in ratio form
    const double *sin2;    // 2 sin(pi j / M), j = 0..M/2
    // double-float variant (dd = 1): arithmetic on the FP32 pipe; in/out/add
    // may hold FP64 values or double-float pairs (in_dd / out_dd / add_dd)
    int dd;
    int in_dd, out_dd, add_dd;
    const ddr *tabd;       // tab as double-float pairs (if not null, used instead of tab)
    const TwD *twd;
    const ddc *halfd;
    const ddr *sin2d;
    int lines;   // lines per block: 0 = by size (8 for launches of < 2 blocks per SM), 8 = always 8,
                 // -8 = 8 lines on 128 threads (M = 128), 32 (M = 128), 16 (M = 256)
    const void *sinm;      // lengths without an FFT: the sine matrix S[i][e] = sin(pi (i+1)(e+1)/M),
                           // e fastest, FP64 (dd = 0) or double-float pairs (dd = 1): direct sums
};

// Programmatic dependent launch: a kernel launched with launch_pdl lets the next
// launch of its stream be placed on the GPU while it runs (pdl_enter at its start),
// and waits for the previous launch to complete and flush before it reads
// anything (also in pdl_enter).  For a kernel launched otherwise both are no-ops.
__device__ __forceinline__ void pdl_enter()
{
    asm volatile("griddepcontrol.launch_dependents;\n" ::: "memory");
    asm volatile("griddepcontrol.wait;\n" ::: "memory");
}
template <class Kern, class... Args>
cudaError_t launch_pdl(Kern kern, dim3 grid, dim3 block, size_t smem, cudaStream_t st, Args... args)
{
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kern, args...);
}

cudaError_t launch_dst_pass(const DstPass &a, cudaStream_t st);
cudaError_t dst_set_attributes();
cudaError_t boundary_set_attributes();

// ---- mixed-precision sine pass on the tensor cores (mixed.cu) ---------------
// Y[m][p][q] = 4 sum_k S[m][k] X[p][q][k] for every line (p, q), S_{m,k} =
// sin(pi (m+1)(k+1)/M), k, m < n = M-1.  Input/output elements are FP64 or
// FP32; on FP64 output the epilogue out = tab * Y (+ add) is applied in FP64.
struct MpPass {
    const void *in; int in_f64;
    int64_t is_p, is_q, is_k;
    void *out; int out_f64;
    int64_t os_m, os_p, os_q;
    int P, Q, n;
    int variant;                // 0: BF16X3, 1: TF32X3
    const void *bimg;           // pieces of S: [mode tile][k stage][piece][W rows x KB k] (W =
                                // mp_tile_modes(n), KB = mp_stage_k(variant); BF16: 3 pieces, TF32: 2)
    const double *tab; int64_t ts_m, ts_p, ts_q;
    const double *add; int64_t as_m, as_p, as_q;
    int *err;                   // set to 1 if a wait on the tensor cores timed out
    int stall_test;             // test hook: issue no products, so the bounded wait expires
    int in_vec4;                // FP32 input whose lines start on 16-byte boundaries and are padded to
                                // whole 16-byte vectors (is_k = 1, is_q a multiple of 4, is_p = Q is_q
                                // or P = 1): required for FP32 input, which a 2-D tensor map describes
                                // (FP64 input needs is_k = 1 only)
};
cudaError_t launch_mp_pass(const MpPass &a, cudaStream_t st);
cudaError_t mp_set_attributes();
int mp_stage_k(int variant);    // k values per stage of the sine image (32 BF16, 16 TF32)
int mp_tile_modes(int n);       // modes per tile (and image tile) for n modes: 128 or 256

// ---- boundary values (section 4) ------------------------------------------

// Stage 1: real FFT of length 2P (P >= M) of each zero-padded line of interior
// data along `axis`; output P+1 complex values per line, stored at out view
// (complex units).
struct RfftPass {
    const double *in; int64_t is0, is1, is2;     // real input, interior coords
    double2 *out; int64_t os0, os1, os2;          // complex output; `axis` coordinate = frequency m
    int n0, n1, n2;                               // interior box (extent along axis = M-1)
    int axis, M;
    int P;                                        // complex FFT length (0: M)
    FftTables t;                                  // tables for complex length P
    int dd;                                       // 1: double-float arithmetic, output as pairs
    const int *lineflag;   // optional: lineflag[u * nv + v] != 0 iff line (u, v) has a non-zero value
    // stage 1a (axis 2) only, optional: the pass also makes the support flags of
    // its input, zero on entry: rows row2[i0 * n1 + i1] (every entry written),
    // row1[i0 * n2 + i2], slices sl0[i0], sl1[i1], sl2[i2] (set to 1 where non-zero)
    int *fl_row2, *fl_row1, *fl_sl0, *fl_sl1, *fl_sl2;
    double *copy;          // optional: the input is also copied here (same strides)
};
cudaError_t launch_rfft_pass(const RfftPass &a, cudaStream_t st);

// Stage 2 (3-D): for each face axis a, FFT of length 2Pb (Pb >= Mb) along b of
// the stage-1 data of every slice p, times the kernel spectra, summed over p.
struct FacePass {
    const double2 *D;          // stage-1 data
    int64_t sp, sb, sc;        // strides (complex units) of slice p, axis b, frequency c
    int np;                    // number of slices (M_a - 1)
    int Mb;                    // panels along b (data at positions 1..Mb-1)
    int nc;                    // number of frequencies along c (P_c + 1)
    const double *khat;        // [np][nc][Pb+1] real kernel spectra for distance (p+1) h_a (frequency
                               // along b fastest: the threads of a block read consecutive ones)
    double2 *part;             // partial sums [nchunk][2][2Pb][nc]
    int pchunk;                // slices per chunk
    FftTables t;               // tables for complex length 2Pb
    int dd;                    // 1: double-float (D, part as pairs; khatd used)
    const ddr *khatd;          // kernel spectra as double-float pairs
    const int *sliceflag;      // optional: sliceflag[p] != 0 iff slice p has a non-zero value
    int Pb;                    // half the FFT length along b (0: Mb)
};
cudaError_t launch_face_pass(const FacePass &a, int nchunk, cudaStream_t st);
int face_columns_per_block(int L);   // frequencies c per block of the face pass
int face_blocks_per_sm(int L);       // resident blocks per SM of the face pass

// 2-D contraction: part[0/1][m] = sum_p khat[p or np-1-p][m] * T[p][m]
struct FacePass2D {
    const double2 *T; int64_t sp, sm;
    int np, nm;
    const double *khat;        // [np][nm]
    double2 *acc;              // [2][nm]
};
cudaError_t launch_face_pass_2d(const FacePass2D &a, cudaStream_t st);

// Stage 3a (3-D): sum the partials and inverse FFT along b (length 2Pb); keep
// rows 0..Mb.
struct FaceInvB {
    const double2 *part; int nchunk;
    int Mb, nc;
    double2 *out;              // [2][Mb+1][nc]
    FftTables t;               // length 2Pb
    int dd;
    int Pb;                    // 0: Mb
};
cudaError_t launch_face_inv_b(const FaceInvB &a, cudaStream_t st);

// Stage 3b: inverse real FFT of length 2Pc (Pc >= Mc) of each row (Pc+1
// Hermitian coefficients) and scatter the first Mc+1 values into the face nodes
// of up to two node arrays.  Row r of face f (lo/hi) maps to nodes
// base_f + r*row_stride + j*col_stride.
struct FaceC2R {
    const double2 *in;         // [2][nrows][Pc+1]
    int nrows, Mc;
    double *dst0, *dst1;       // node arrays (dst1 may be null)
    int64_t base[2];           // node offset of row 0, col 0 for lo / hi
    int64_t row_stride, col_stride;
    // ownership: skip rows r with skip_row_lo/hi set (edge already owned by a
    // lower face axis) and columns with col in {0, Mc} if skip_cols is set.
    int skip_row_edges, skip_col_edges;
    FftTables t;               // length Pc
    int dd;
    int Pc;                    // 0: Mc
};
cudaError_t launch_face_c2r(const FaceC2R &a, cudaStream_t st);

// d = 1 (section 5): g at the two end nodes from rho (node array, M + 1 values)
// and the straight line through them; see line1d_kernel for the modes
enum { LINE1D_ENDS = 0, LINE1D_LINE = 1, LINE1D_ADD = 2 };
cudaError_t launch_line1d(const double *rho, double *phi, int M, double h, int mode, cudaStream_t st);

// Cyclic-kernel samples k[p][tb][tc] = G(sqrt(((p0+p+1) h_a)^2 + (tb h_b)^2 + (tc h_c)^2)),
// tb = 0..Mb, tc = 0..Mc (2-D: Mc = 0).
struct KernelFill {
    double *k;                 // [np][Mb+1][Mc+1], or [np][Mc+1][Mb+1] if tr
    int d, np, Mb, Mc;
    double ha, hb, hc;
    int p0;
    int tr;
};
cudaError_t launch_kernel_fill(const KernelFill &a, cudaStream_t st);
// batched C[b] = A[b] * B[b] (FP64), row-major, strides in elements
cudaError_t launch_gemm_batched(int m, int n, int k, const double *A, int64_t lda, int64_t sA,
                                const double *B, int64_t ldb, int64_t sB, double *C, int64_t ldc,
                                int64_t sC, int batch, cudaStream_t st);

// ---- stencils (section 5) -------------------------------------------------
struct Grid3 {
    int d;                     // 2 or 3 (2-D grids use n0 = 1, axes 1,2)
    int n0, n1, n2;            // node counts (n0 = 1 for d = 2)
    double h0, h1, h2;
};
// Stencil weights computed once on the host: wf/we = L4 face/edge weights,
// a = 6th-order pair coefficients (see stencil.cu).
struct StencilCoef {
    double wf[3];
    double we[3][3];
    double a[3][3];
};
StencilCoef make_stencil_coef(const Grid3 &g);
// gtilde on the boundary-adjacent layers, split into parts Q0 (3-D), Q1, Q2 (see stencil.cu)
cudaError_t launch_gtilde_planes(const Grid3 &g, const StencilCoef &c, const double *U, double *Q0, double *Q1,
                                 double *Q2, cudaStream_t st);
// out = tab * (4^d S gtilde) (+ add) from the transformed, combined parts; if out2
// is given, also out2 = (tab2 (- tab unless fold)) * (4^d S gtilde) + add2; with
// ascale, add and add2 are multiplied by ascale first
cudaError_t launch_gtilde_expand(const Grid3 &g, const double *Q0, const double *Q1, const double *Q2,
                                 const double *sin4, const double *tab, const double *add, double *out,
                                 cudaStream_t st, const double *tab2 = nullptr, const double *add2 = nullptr,
                                 double *out2 = nullptr, int fold = 0, const double *ascale = nullptr);
// (a, b) -> (a + b, a - b) for the pairs of transformed layers at the two faces of
// an axis: part i holds [2][nl][pl_i] (pl_i = 0: absent)
cudaError_t launch_layers_combine(double *P0, int64_t pl0, double *P1, int64_t pl1, double *P2, int64_t pl2,
                                  int nl, cudaStream_t st);
cudaError_t launch_gtilde_scatter(const Grid3 &g, const double *Q0, const double *Q1, const double *Q2,
                                  double *out, cudaStream_t st);
// W_s = sum_{r != s} a_sr (u(+e_r) + u(-e_r) - 2u) on nodes; W is 3 node arrays (2 for d = 2).
cudaError_t launch_rhs6_w(const Grid3 &g, const StencilCoef &c, const double *U, double *W, cudaStream_t st);
// R on the core (indices 2..M-2) into dense interior `R`, then extrapolation to the layers 1, M-1.
cudaError_t launch_rhs6_core(const Grid3 &g, const double *W, double *R, cudaStream_t st);
cudaError_t launch_rhs6_extrap(const Grid3 &g, double *R, cudaStream_t st);
// y = double-float pairs of x (set-up only)
cudaError_t launch_to_dd(const double *x, ddr *y, int64_t n, cudaStream_t st);
// tabc = sc / lambda_c(k) and tab4 = sc / Lambda4(k) on the dense mode grid;
// lc / ld hold the per-axis 1-D eigenvalues, axis s at offset off_s (axis 0 at 0).
// tabR (optional) = tab4 * Lambda_R / Lambda4 + tab4 with Lambda_R the symbol of
// the 6th-order right-hand side.
cudaError_t launch_eigen_tables(const Grid3 &g, const double *lc, const double *ld, int64_t off1,
                                int64_t off2, double sc, double *tabc, double *tab4, double *tabR, cudaStream_t st);
// The 6th-order right-hand side in spectral form (stencil.cu): kind 0: W of the
// odd continuation of u1 on the nodes within 7 of a face; kind 1: R at the
// extrapolation taps into the dense interior array Rt; kind 2: the layers of
// E = R - R_spec (E0 [2][2][n1][n2] (3-D), E1 [2][2][n0][n2], E2 [2][2][n0][n1]).
cudaError_t launch_rhs6_spectral(const Grid3 &g, const StencilCoef &c, const double *U, double *W, double *Rt,
                                 double *E0, double *E1, double *E2, int kind, cudaStream_t st);
// out += tab * (4^d S E) from the transformed layers of E
cudaError_t launch_rhs6_e_expand(const Grid3 &g, const double *E0, const double *E1, const double *E2,
                                 const double *sin4, const double *sin4b, const double *tab, double *out,
                                 cudaStream_t st);
// x *= Lambda_R (per mode) and out += E on its layers: the stage output of R
cudaError_t launch_rhs6_symbol(const Grid3 &g, const double *ld, int64_t off1, int64_t off2, double *x,
                               cudaStream_t st);
// dst[i0*d0 + i1*d1 + i2] = src[i0*s0 + i1*s1 + i2] over the box e0 x e1 x e2
// (innermost axis contiguous on both sides): the copies between the caller's
// grid and a padded grid
cudaError_t launch_box_copy(const double *src, int64_t s0, int64_t s1, double *dst, int64_t d0, int64_t d1,
                            int e0, int e1, int e2, cudaStream_t st);
// Validation of rho (node array n0 x n1 x n2, inactive axes of extent 1): bit 1
// of *word for a NaN or infinite value on an interior node, bit 2 for a non-zero
// value on an interior node within k layers of the boundary (of an active axis)
cudaError_t launch_validate_rho(const double *rho, int n0, int n1, int n2, int act0, int act1, int act2, int k,
                                int *word, cudaStream_t st);
cudaError_t launch_rhs6_e_scatter(const Grid3 &g, const double *E0, const double *E1, const double *E2,
                                  double *out, cudaStream_t st);

}  // namespace idp
