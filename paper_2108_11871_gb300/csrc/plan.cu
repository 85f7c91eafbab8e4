// C ABI of the infinite-domain Poisson solver: plans, workspace, tables and
// the order of the stages of one solve (section 2: phi = phi* + phi_H).
#include <cmath>
#include <cstdio>
#include <cstring>
#include <map>
#include <atomic>
#include <mutex>
#include <new>
#include <algorithm>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "dd.cuh"
#include "idp_internal.cuh"
#include "../../include/idp.h"

using namespace idp;

namespace {

thread_local char g_cuda_err[256] = "";

int cuda_fail(cudaError_t e, const char *what)
{
    snprintf(g_cuda_err, sizeof(g_cuda_err), "%s: %s", what, cudaGetErrorString(e));
    return IDP_ECUDA;
}

#define IDP_CK(call)                                       \
    do {                                                   \
        cudaError_t e_ = (call);                           \
        if (e_ != cudaSuccess) return cuda_fail(e_, #call); \
    } while (0)

bool is_pow2(int64_t x) { return x > 0 && (x & (x - 1)) == 0; }
// panel counts with a transform kernel: 2^a in [16, 512] or 3 * 2^a in [48, 384]
bool supported_panels(int64_t M)
{
    return M >= 16 && M <= 512 && (is_pow2(M) || (M >= 48 && M % 3 == 0 && is_pow2(M / 3)));
}

// panel counts whose sine transform runs as an FFT here
bool has_fft_dst(int64_t M) { return supported_panels(M); }

// half the length of the zero-padded boundary convolutions for M panels: the
// smallest complex FFT length here that is >= M (M itself where it has one)
int conv_half(int64_t M)
{
    const int lens[12] = {16, 32, 48, 64, 96, 128, 192, 256, 384, 512, 768, 1024};
    for (int L : lens)
        if (L >= M) return L;
    return 0;
}

// the smallest supported panel count >= M (0 if there is none)
int64_t padded_panels(int64_t M)
{
    for (int64_t m = M < 16 ? 16 : M; m <= 512; ++m)
        if (supported_panels(m)) return m;
    return 0;
}

// host tables ----------------------------------------------------------------
// sin(pi m / L) and cos(pi m / L) with the integer argument reduced to [0, 2L).
double sinpi_frac(int64_t m, int64_t L)
{
    m %= 2 * L;
    if (m < 0) m += 2 * L;
    return std::sin(M_PI * (double)m / (double)L);
}
double cospi_frac(int64_t m, int64_t L)
{
    m %= 2 * L;
    if (m < 0) m += 2 * L;
    return std::cos(M_PI * (double)m / (double)L);
}

Tw make_tw(double c, double s)
{
    Tw t;
    if (std::fabs(c) >= std::fabs(s)) {
        t.r = s / c; t.mre = c; t.mim = c; t.swap = 0;
    } else {
        t.r = c / s; t.mre = -s; t.mim = s; t.swap = 1;
    }
    t.pad = 0;
    return t;
}

struct DevFft {
    Tw *fwd = nullptr, *inv = nullptr;
    double2 *half = nullptr;
    Tw *halfr = nullptr;
    TwD *fwdd = nullptr, *invd = nullptr;   // double-float forms
    ddc *halfd = nullptr;
    FftTables view(int L) const { return FftTables{L, fwd, inv, half, halfr, fwdd, invd, halfd}; }
};

// double-float pair of a double (host): hi = nearest float, lo = nearest float of the rest
ddr host_dd(double x)
{
    ddr r;
    r.hi = (float)x;
    r.lo = (float)(x - (double)r.hi);
    return r;
}
TwD make_twd(const Tw &t)
{
    TwD d;
    d.r = host_dd(t.r);
    d.mre = host_dd(t.mre);
    d.mim = host_dd(t.mim);
    d.swap = t.swap;
    d.pad = 0;
    return d;
}

std::mutex g_attr_mu;
std::atomic<uint64_t> g_serial{1};
std::vector<int> g_attr_done;

int ensure_attributes(int dev)
{
    std::lock_guard<std::mutex> lk(g_attr_mu);
    for (int d : g_attr_done)
        if (d == dev) return IDP_OK;
    IDP_CK(dst_set_attributes());
    IDP_CK(boundary_set_attributes());
    IDP_CK(mp_set_attributes());
    g_attr_done.push_back(dev);
    return IDP_OK;
}

}  // namespace

struct BatchCache {
    std::vector<uint64_t> serials;
    std::vector<const double *> rho;
    std::vector<double *> phi;
    cudaGraphExec_t exec = nullptr;
    std::vector<cudaEvent_t> joins;
    cudaEvent_t fork = nullptr;
};

struct idp_plan_s {
    int d = 0, order = 0, dev = 0;
    uint64_t serial = 0;                 // unique per plan (keys the batch graph cache)
    uint64_t version = 0;                // bumped when an option changes the queued work
    cudaStream_t bst = nullptr;          // this plan's branch stream in a batched graph
    BatchCache *batch = nullptr;         // batched graph owned by this plan (first of its batch)
    int n[3] = {1, 1, 1};      // internal node counts (2-D: n[0] = 1)
    int M[3] = {0, 0, 0};
    int P[3] = {0, 0, 0};      // half the length of the boundary convolutions along each axis (P >= M)
    int ni[3] = {1, 1, 1};     // interior extents
    int act[3] = {0, 0, 0};
    double h[3] = {1, 1, 1};
    int64_t nodes = 0, nint = 0;
    // automatic padding (section 2: the domain is extended by a few panels so that
    // every panel count suits the transforms): the caller's node counts, the offset
    // of the caller's node 0 in the grid solved on, the caller's node count, and
    // the padded copies of rho and phi
    int padded = 0;
    int un[3] = {1, 1, 1}, uoff[3] = {0, 0, 0};
    int64_t unodes = 0;
    double *rho_pad = nullptr, *phi_pad = nullptr;
    int64_t ns[3] = {0, 0, 0};  // node strides
    int64_t is[3] = {0, 0, 0};  // interior strides
    Grid3 grid{};
    StencilCoef coef{};

    std::map<int, DevFft> fft;        // by complex length
    std::map<int, double *> sin2;     // by M: 2 sin(pi j / M), j = 0..M/2
    std::map<int, ddr *> sin2d;       // double-float form
    std::map<int, double *> sinm;     // by M (lengths without an FFT): sine matrices for direct sums
    std::map<int, ddr *> sinmd;       // double-float form
    int exact = 0;                    // created by idp_create_plan_exact
    std::vector<void *> allocs;
    static constexpr size_t GUARD = 256;              // keeps the buffers 256-byte aligned
    static constexpr unsigned char GUARD_BYTE = 0xA5;
    std::vector<std::pair<char *, size_t>> guarded;   // allocation base, payload bytes
    int64_t bytes = 0;

    double *A = nullptr, *B = nullptr, *C = nullptr, *U = nullptr, *W = nullptr;
    double *tabc = nullptr, *tab4 = nullptr;
    double *tabc2 = nullptr;   // -2 * tabc (forward transform of rho continued from T0)
    double *Q0 = nullptr, *Q1 = nullptr, *Q2 = nullptr, *sin4 = nullptr;   // gtilde parts
    double *tabR = nullptr;    // tab4 * Lambda_R / Lambda4 + tab4 (R_spec's smoothing solve plus u1)
    double *E0 = nullptr, *E1 = nullptr, *E2 = nullptr, *sin4b = nullptr;   // layers of E = R - R_spec
    double *ld = nullptr;      // per-axis eigenvalues of D2_s (axis s at ldoff[s])
    int64_t ldoff[3] = {0, 0, 0};
    int *flags = nullptr;        // support flags of rho: rows along axes 2 and 1, slices of axes 0, 1, 2
    int64_t nflags = 0;
    int *row2 = nullptr, *row1 = nullptr, *sl[3] = {nullptr, nullptr, nullptr};
    double2 *T0 = nullptr, *T1 = nullptr, *part = nullptr, *F = nullptr;
    double *khat[3] = {nullptr, nullptr, nullptr};
    ddr *khatd[3] = {nullptr, nullptr, nullptr};   // double-float copies (precision DF32)
    int64_t khat_n[3] = {0, 0, 0};
    int nchunk[3] = {1, 1, 1}, pchunk[3] = {1, 1, 1};
    int dst_lines = 0;                // lines per block of the full-volume sine passes (0 = default)

    // mixed precision (IDP_KEY_PRECISION = 1): sine passes on the tensor cores
    int mixed = 0;
    int stall_test = 0;               // IDP_KEY_STALL_TEST: next tensor-core pass waits in vain
    int mixed_path = 0;               // mixed precision: 0 = tensor-core matrix pass, 1 = df32 FFT pass
    int mixed_bdd = 0;                // IDP_KEY_MIXED_BOUNDARY_DF32: tensor-core modes, 3-D boundary in double-float
    int64_t part_cap = 0;             // capacity (complex) of the partial face sums of one axis
    int64_t f_cap = 0;                // capacity (complex) of the face spectra of one axis
    int tuned = 0;
    std::map<int, void *> mp_img;     // by M: BF16 pieces of the sine matrix
    float *t32[2][2] = {{nullptr, nullptr}, {nullptr, nullptr}};   // [stream][ping/pong]
    int *d_err = nullptr;
    int validate = 0;                 // IDP_KEY_VALIDATE: margin k (0: off)
    int *d_val = nullptr;             // validation word (bit 1: NaN/inf, bit 2: support too close)

    // per-launch timing (idp_profile_solve)
    int profiling = 0;
    std::vector<cudaEvent_t> ev;
    std::vector<int> ev_kind;
    int ev_used = 0;
    int64_t launches = 0;      // kernel launches queued by the last enqueue

    // staging for idp_solve_host
    double *h_rho = nullptr, *h_phi = nullptr;

    // CUDA graph of one solve for a fixed (rho, phi)
    int use_graph = 1;
    int nvtx = 0;                     // IDP_KEY_NVTX: NVTX ranges around launches and stages
    cudaStream_t cap = nullptr;
    cudaStream_t side = nullptr;          // second stream of a solve (forward transform of rho)
    cudaEvent_t fork = nullptr, join = nullptr;
    // 3-D faces: axes 0 and 1 run on their own streams beside axis 2 (each axis
    // with its own partial sums and face spectra)
    cudaStream_t fst[2] = {nullptr, nullptr};
    cudaEvent_t fev[3] = {nullptr, nullptr, nullptr};   // T0 ready; axis 0 done; axis 1 done
    // host-buffer solves (page-locked buffers, captured into their own graph): the
    // first row transform reads rho from the host buffer (through its device view)
    // and the kernels that write phi write the host buffer directly, so that the
    // upload and the download overlap their work
    const double *hio_rho = nullptr;   // host rho of the solve being queued (null: none)
    const double *hio_view = nullptr;  // its device view
    cudaGraphExec_t hexec = nullptr;
    const double *hg_rho = nullptr;
    double *hg_phi = nullptr;
    uint64_t hg_version = ~0ull;
    cudaGraphExec_t gexec = nullptr;
    const double *g_rho = nullptr;
    double *g_phi = nullptr;
    cudaStream_t last = nullptr;
    int last_valid = 0;

    template <class T>
    int alloc(T **p, int64_t count)
    {
        // every buffer sits between two guard regions of GUARD bytes filled with
        // GUARD_BYTE; idp_plan_check_guards reports one that was overwritten (an
        // out-of-bounds write), in place of a memory checker
        void *q = nullptr;
        const size_t b = (size_t)count * sizeof(T);
        const size_t payload = b > 0 ? b : 16;
        cudaError_t e = cudaMalloc(&q, payload + 2 * GUARD);
        if (e != cudaSuccess) {
            cuda_fail(e, "cudaMalloc");
            return IDP_ENOMEM;
        }
        char *c = static_cast<char *>(q);
        e = cudaMemset(c, GUARD_BYTE, GUARD);
        if (e == cudaSuccess) e = cudaMemset(c + GUARD + payload, GUARD_BYTE, GUARD);
        allocs.push_back(q);
        guarded.emplace_back(c, payload);
        if (e != cudaSuccess) return cuda_fail(e, "cudaMemset (guards)");
        bytes += (int64_t)b;
        *p = (T *)(c + GUARD);
        return IDP_OK;
    }
};

namespace {

// NVTX range names of the IDP_KERNEL_* families
const char *kernel_range(int kind)
{
    switch (kind) {
    case IDP_KERNEL_DST: return "idp:dst";
    case IDP_KERNEL_RFFT: return "idp:rfft";
    case IDP_KERNEL_FACE: return "idp:face";
    case IDP_KERNEL_FACE_INVB: return "idp:face_invb";
    case IDP_KERNEL_FACE_C2R: return "idp:face_c2r";
    case IDP_KERNEL_GTILDE: return "idp:gtilde";
    case IDP_KERNEL_RHS6_W: return "idp:rhs6_w";
    case IDP_KERNEL_RHS6_CORE: return "idp:rhs6_core";
    case IDP_KERNEL_RHS6_EXTRAP: return "idp:rhs6_extrap";
    case IDP_KERNEL_GTILDE_EXPAND: return "idp:gtilde_expand";
    case IDP_KERNEL_DST_PARTS: return "idp:dst_layers";
    case IDP_KERNEL_MIXED: return "idp:mixed";
    case IDP_KERNEL_RHS6_EXPAND: return "idp:rhs6_expand";
    case IDP_KERNEL_LINE1D: return "idp:line1d";
    case IDP_KERNEL_PAD: return "idp:pad";
    case IDP_KERNEL_VALIDATE: return "idp:validate";
    default: return "idp:kernel";
    }
}

// An NVTX range over a stage of a solve (IDP_KEY_NVTX), closed at the end of scope.
struct Range {
    bool on;
    Range(idp_plan p, const char *name) : on(p->nvtx != 0)
    {
        if (on) nvtxRangePushA(name);
    }
    ~Range()
    {
        if (on) nvtxRangePop();
    }
};

// Marks one kernel launch: counts it, with IDP_KEY_NVTX encloses it in an NVTX
// range named after its family and, while profiling, brackets it with CUDA events
// recorded on the launch stream.
struct Mark {
    idp_plan p;
    cudaStream_t st;
    int idx = -1;
    Range r;
    Mark(idp_plan p_, int kind, cudaStream_t st_) : p(p_), st(st_), r(p_, kernel_range(kind))
    {
        ++p->launches;
        if (p->profiling && p->ev_used + 2 <= (int)p->ev.size()) {
            idx = p->ev_used;
            p->ev_used += 2;
            p->ev_kind.push_back(kind);
            cudaEventRecord(p->ev[idx], st);
        }
    }
    ~Mark()
    {
        if (idx >= 0) cudaEventRecord(p->ev[idx + 1], st);
    }
};

int get_fft(idp_plan p, int L, FftTables *out)
{
    auto it = p->fft.find(L);
    if (it != p->fft.end()) {
        *out = it->second.view(L);
        return IDP_OK;
    }
    DevFft t;
    std::vector<Tw> fw(L / 2), iv(L / 2);
    for (int j = 0; j < L / 2; ++j) {
        const double c = cospi_frac(2 * j, L), s = sinpi_frac(2 * j, L);
        fw[j] = make_tw(c, -s);
        iv[j] = make_tw(c, s);
    }
    std::vector<double2> hf(L + 1);
    std::vector<Tw> hr(L + 1);
    for (int k = 0; k <= L; ++k) {
        hf[k] = make_double2(cospi_frac(k, L), -sinpi_frac(k, L));
        hr[k] = make_tw(hf[k].x, hf[k].y);
    }
    std::vector<TwD> fwd2(L / 2), ivd2(L / 2);
    std::vector<ddc> hfd(L + 1);
    for (int j = 0; j < L / 2; ++j) {
        fwd2[j] = make_twd(fw[j]);
        ivd2[j] = make_twd(iv[j]);
    }
    for (int k = 0; k <= L; ++k) {
        hfd[k].re = host_dd(hf[k].x);
        hfd[k].im = host_dd(hf[k].y);
    }
    int rc;
    if ((rc = p->alloc(&t.fwd, L / 2)) || (rc = p->alloc(&t.inv, L / 2)) || (rc = p->alloc(&t.half, L + 1)) ||
        (rc = p->alloc(&t.halfr, L + 1)) ||
        (rc = p->alloc(&t.fwdd, L / 2)) || (rc = p->alloc(&t.invd, L / 2)) || (rc = p->alloc(&t.halfd, L + 1)))
        return rc;
    IDP_CK(cudaMemcpy(t.fwd, fw.data(), sizeof(Tw) * (L / 2), cudaMemcpyHostToDevice));
    IDP_CK(cudaMemcpy(t.inv, iv.data(), sizeof(Tw) * (L / 2), cudaMemcpyHostToDevice));
    IDP_CK(cudaMemcpy(t.half, hf.data(), sizeof(double2) * (L + 1), cudaMemcpyHostToDevice));
    IDP_CK(cudaMemcpy(t.halfr, hr.data(), sizeof(Tw) * (L + 1), cudaMemcpyHostToDevice));
    IDP_CK(cudaMemcpy(t.fwdd, fwd2.data(), sizeof(TwD) * (L / 2), cudaMemcpyHostToDevice));
    IDP_CK(cudaMemcpy(t.invd, ivd2.data(), sizeof(TwD) * (L / 2), cudaMemcpyHostToDevice));
    IDP_CK(cudaMemcpy(t.halfd, hfd.data(), sizeof(ddc) * (L + 1), cudaMemcpyHostToDevice));
    p->fft[L] = t;
    *out = t.view(L);
    return IDP_OK;
}

int get_sin2(idp_plan p, int M, const double **out)
{
    auto it = p->sin2.find(M);
    if (it != p->sin2.end()) {
        *out = it->second;
        return IDP_OK;
    }
    std::vector<double> s(M / 2 + 1);
    std::vector<ddr> sd(M / 2 + 1);
    for (int j = 0; j <= M / 2; ++j) {
        s[j] = 2.0 * sinpi_frac(j, M);
        sd[j] = host_dd(s[j]);
    }
    double *d = nullptr;
    ddr *dd = nullptr;
    int rc;
    if ((rc = p->alloc(&d, M / 2 + 1)) || (rc = p->alloc(&dd, M / 2 + 1))) return rc;
    IDP_CK(cudaMemcpy(d, s.data(), sizeof(double) * (M / 2 + 1), cudaMemcpyHostToDevice));
    IDP_CK(cudaMemcpy(dd, sd.data(), sizeof(ddr) * (M / 2 + 1), cudaMemcpyHostToDevice));
    p->sin2[M] = d;
    p->sin2d[M] = dd;
    *out = d;
    return IDP_OK;
}

// sine matrix S[i][e] = sin(pi (i+1)(e+1) / M), i, e < M - 1, e fastest, for the
// direct sums of the lengths without an FFT; FP64 and double-float forms
int get_sinm(idp_plan p, int M, const void **out, int dd)
{
    auto it = p->sinm.find(M);
    if (it == p->sinm.end()) {
        const int N = M - 1;
        std::vector<double> s((size_t)N * N);
        std::vector<ddr> sd((size_t)N * N);
        for (int i = 0; i < N; ++i)
            for (int e = 0; e < N; ++e) {
                s[(size_t)i * N + e] = sinpi_frac((int64_t)(i + 1) * (e + 1), M);
                sd[(size_t)i * N + e] = host_dd(s[(size_t)i * N + e]);
            }
        double *d = nullptr;
        ddr *d2 = nullptr;
        int rc;
        if ((rc = p->alloc(&d, (int64_t)N * N)) || (rc = p->alloc(&d2, (int64_t)N * N))) return rc;
        IDP_CK(cudaMemcpy(d, s.data(), sizeof(double) * s.size(), cudaMemcpyHostToDevice));
        IDP_CK(cudaMemcpy(d2, sd.data(), sizeof(ddr) * sd.size(), cudaMemcpyHostToDevice));
        p->sinm[M] = d;
        p->sinmd[M] = d2;
    }
    *out = dd ? (const void *)p->sinmd[M] : (const void *)p->sinm[M];
    return IDP_OK;
}

View3 node_interior(idp_plan p, const double *base)
{
    int64_t off = 0;
    for (int s = 0; s < 3; ++s)
        if (p->act[s]) off += p->ns[s];
    return View3{const_cast<double *>(base) + off, p->ns[0], p->ns[1], p->ns[2]};
}
View3 dense(idp_plan p, const double *base) { return View3{const_cast<double *>(base), p->is[0], p->is[1], p->is[2]}; }

uint16_t bf16_bits(float f)
{
    uint32_t u;
    std::memcpy(&u, &f, 4);
    u += 0x7FFFu + ((u >> 16) & 1u);   // round to nearest even (finite values)
    return (uint16_t)(u >> 16);
}
double bf16_value(uint16_t b)
{
    const uint32_t u = (uint32_t)b << 16;
    float f;
    std::memcpy(&f, &u, 4);
    return (double)f;
}

// FP32 bits rounded to TF32 (11 significant bits, to nearest, ties to even)
uint32_t tf32_bits(float x)
{
    uint32_t u;
    std::memcpy(&u, &x, 4);
    return (u + 0xFFFu + ((u >> 13) & 1u)) & 0xFFFFE000u;
}
double tf32_value(uint32_t u)
{
    float f;
    std::memcpy(&f, &u, 4);
    return (double)f;
}

// TF32 pieces of S (variant 1): [mode tile][k stage][2][W rows m x KB k] FP32
// containers (W = mp_tile_modes(n), KB = mp_stage_k(1)), element (r, c) at byte
// (c/4)*(16 W) + (r/8)*128 + (r%8)*16 + (c%4)*4
int get_mp_image_tf32(idp_plan p, int M, const void **out)
{
    const int KB = mp_stage_k(1);
    const int n = M - 1, W = mp_tile_modes(n), nt = (n + W - 1) / W, nkb = (n + KB - 1) / KB;
    const size_t tile = (size_t)W * KB;
    std::vector<uint32_t> img((size_t)nt * nkb * 2 * tile, 0);
    for (int t = 0; t < nt; ++t)
        for (int kb = 0; kb < nkb; ++kb)
            for (int r = 0; r < W; ++r)
                for (int c = 0; c < KB; ++c) {
                    const int m = t * W + r, k = kb * KB + c;
                    const double s = (m < n && k < n) ? sinpi_frac((int64_t)(m + 1) * (k + 1), M) : 0.0;
                    const uint32_t a = tf32_bits((float)s);
                    const uint32_t b = tf32_bits((float)(s - tf32_value(a)));
                    const size_t off = ((size_t)(c / 4) * (16 * W) + (r / 8) * 128 + (r % 8) * 16 + (c % 4) * 4) / 4;
                    const size_t base = (((size_t)t * nkb + kb) * 2) * tile;
                    img[base + off] = a;
                    img[base + tile + off] = b;
                }
    uint32_t *d;
    int rc = p->alloc(&d, (int64_t)img.size());
    if (rc) return rc;
    IDP_CK(cudaMemcpy(d, img.data(), img.size() * sizeof(uint32_t), cudaMemcpyHostToDevice));
    *out = d;
    return IDP_OK;
}

int64_t pad4(int64_t x) { return (x + 3) & ~(int64_t)3; }
// floats of one FP32 intermediate of the tensor-core transforms (the larger of the
// two padded layouts)
int64_t t32_count(idp_plan p)
{
    const int64_t n0 = p->ni[0], n1 = p->ni[1], n2 = p->ni[2];
    if (p->d == 3) return std::max(n2 * n0 * pad4(n1), n1 * n2 * pad4(n0));
    return n2 * pad4(n1);
}

// the tensor-core pass variant of the plan's precision (0: BF16X3, 1: TF32X3)
int mp_variant(idp_plan p) { return p->mixed == IDP_PRECISION_MIXED_TF32X3 ? 1 : 0; }
bool tensor_mode(idp_plan p)
{
    return p->mixed == IDP_PRECISION_MIXED_BF16X3 || p->mixed == IDP_PRECISION_MIXED_TF32X3;
}
// the 3-D boundary convolutions (and so T0) in double-float arithmetic: precision
// DF32, or a tensor-core mode with IDP_KEY_MIXED_BOUNDARY_DF32
int boundary_dd(idp_plan p)
{
    return p->d == 3 && (p->mixed == IDP_PRECISION_DF32 || (tensor_mode(p) && p->mixed_bdd)) ? 1 : 0;
}

// Pieces of S_{m,k} = sin(pi (m+1)(k+1)/M) for a tensor-core variant, laid out
// as the kernel's shared-memory tiles, one contiguous block per (mode tile,
// K stage).  BF16 (variant 0): [mode tile][k stage][3][W rows m x KB k] with
// W = mp_tile_modes(n), KB = mp_stage_k(0), element (r, c) at byte
// (c/8)*(16 W) + (r/8)*128 + (r%8)*16 + (c%8)*2.  Cached per (M, variant).
int get_mp_image(idp_plan p, int M, int variant, const void **out)
{
    const int key = M + (variant << 24);
    auto it = p->mp_img.find(key);
    if (it != p->mp_img.end()) {
        *out = it->second;
        return IDP_OK;
    }
    if (variant) {
        int rc = get_mp_image_tf32(p, M, out);
        if (!rc) p->mp_img[key] = const_cast<void *>(*out);
        return rc;
    }
    const int KB = mp_stage_k(0);
    const int n = M - 1, W = mp_tile_modes(n), nt = (n + W - 1) / W, nkb = (n + KB - 1) / KB;
    const size_t tile = (size_t)W * KB;
    std::vector<uint16_t> img((size_t)nt * nkb * 3 * tile, 0);
    for (int t = 0; t < nt; ++t)
        for (int kb = 0; kb < nkb; ++kb)
            for (int r = 0; r < W; ++r)
                for (int c = 0; c < KB; ++c) {
                    const int m = t * W + r, k = kb * KB + c;
                    const double s = (m < n && k < n) ? sinpi_frac((int64_t)(m + 1) * (k + 1), M) : 0.0;
                    const uint16_t a = bf16_bits((float)s);
                    const double r1 = s - bf16_value(a);
                    const uint16_t b = bf16_bits((float)r1);
                    const double r2 = r1 - bf16_value(b);
                    const uint16_t cc = bf16_bits((float)r2);
                    const size_t off = ((size_t)(c / 8) * (16 * W) + (r / 8) * 128 + (r % 8) * 16 + (c % 8) * 2) / 2;
                    const size_t base = (((size_t)t * nkb + kb) * 3) * tile;
                    img[base + off] = a;
                    img[base + tile + off] = b;
                    img[base + 2 * tile + off] = cc;
                }
    uint16_t *d;
    int rc = p->alloc(&d, (int64_t)img.size());
    if (rc) return rc;
    IDP_CK(cudaMemcpy(d, img.data(), img.size() * sizeof(uint16_t), cudaMemcpyHostToDevice));
    p->mp_img[key] = d;
    *out = d;
    return IDP_OK;
}

// Sine transform of all active axes with the tensor-core pass (mixed.cu).
// The passes rotate the axes: (a,b,c) -> (c',a,b) -> (b',c',a) -> (a',b',c').
int transform_mixed(idp_plan p, View3 in, View3 out, const double *tab, View3 add, int sidx, cudaStream_t st)
{
    const int n0 = p->ni[0], n1 = p->ni[1], n2 = p->ni[2];
    float *ta = p->t32[sidx][0], *tb = p->t32[sidx][1];
    std::vector<MpPass> ps;
    MpPass a{};
    a.err = p->d_err;
    a.variant = mp_variant(p);
    // the FP32 intermediates keep their contiguous (next pass's k) axis padded to
    // whole 16-byte vectors, so that the next pass loads its lines as vectors
    const int64_t n0p = pad4(n0), n1p = pad4(n1);
    if (p->d == 3) {
        a.in = in.p; a.in_f64 = 1; a.is_p = in.s0; a.is_q = in.s1; a.is_k = in.s2;
        a.out = ta; a.out_f64 = 0; a.os_m = (int64_t)n0 * n1p; a.os_p = n1p; a.os_q = 1;
        a.P = n0; a.Q = n1; a.n = n2;
        ps.push_back(a);
        a.in = ta; a.in_f64 = 0; a.in_vec4 = 1; a.is_p = (int64_t)n0 * n1p; a.is_q = n1p; a.is_k = 1;
        a.out = tb; a.os_m = (int64_t)n2 * n0p; a.os_p = n0p; a.os_q = 1;
        a.P = n2; a.Q = n0; a.n = n1;
        ps.push_back(a);
        a.in = tb; a.is_p = (int64_t)n2 * n0p; a.is_q = n0p; a.is_k = 1;
        a.P = n1; a.Q = n2; a.n = n0;
    } else {
        a.in = in.p; a.in_f64 = 1; a.is_p = 0; a.is_q = in.s1; a.is_k = in.s2;
        a.out = ta; a.out_f64 = 0; a.os_m = n1p; a.os_p = 0; a.os_q = 1;
        a.P = 1; a.Q = n1; a.n = n2;
        ps.push_back(a);
        a.in = ta; a.in_f64 = 0; a.in_vec4 = 1; a.is_p = 0; a.is_q = n1p; a.is_k = 1;
        a.P = 1; a.Q = n2; a.n = n1;
    }
    // last pass: FP64 output in the original layout with the epilogue
    const int s0 = p->d == 3 ? 0 : 1;   // output axis of the modes
    const int64_t os[3] = {out.s0, out.s1, out.s2}, as[3] = {add.s0, add.s1, add.s2};
    const int64_t ts[3] = {p->is[0], p->is[1], p->is[2]};
    a.out = out.p; a.out_f64 = 1;
    a.os_m = os[s0]; a.os_p = p->d == 3 ? os[1] : 0; a.os_q = os[2];
    a.tab = tab; a.ts_m = ts[s0]; a.ts_p = p->d == 3 ? ts[1] : 0; a.ts_q = ts[2];
    a.add = add.p; a.as_m = as[s0]; a.as_p = p->d == 3 ? as[1] : 0; a.as_q = as[2];
    ps.push_back(a);
    // pass i transforms axis 2, 1, 0 (3-D) / 2, 1 (2-D) of the original array
    const int axes3[3] = {2, 1, 0}, axes2[2] = {2, 1};
    if (p->stall_test) {
        ps[0].stall_test = 1;
        p->stall_test = 0;
    }
    for (size_t i = 0; i < ps.size(); ++i) {
        const int ax = p->d == 3 ? axes3[i] : axes2[i];
        int rc = get_mp_image(p, p->M[ax], ps[i].variant, &ps[i].bimg);
        if (rc) return rc;
        Mark mk(p, IDP_KERNEL_MIXED, st);
        IDP_CK(launch_mp_pass(ps[i], st));
    }
    return IDP_OK;
}

// one full sine transform (all active axes); `first` pass reads `in`, the
// last pass applies the epilogue (tab, add) and writes `out`; intermediate
// passes run in place on `work`.
// allow_reduced = false: FP64 passes in every precision mode except that
// fp64_only = false lets the tensor-core modes run them as double-float passes
// (the transform producing u1: FP64-class there, never the tensor cores)
int transform(idp_plan p, View3 in, double *work, View3 out, const double *tab, View3 add, bool forward,
              cudaStream_t st, bool allow_reduced = true, bool skip_axis2 = false, int in_dd0 = 0,
              bool fp64_only = true)
{
    Range rg(p, forward ? "idp:sine transform (forward)" : "idp:sine transform (inverse)");
    if (tensor_mode(p) && allow_reduced && p->mixed_path == 0)
        return transform_mixed(p, in, out, tab, add, st == p->side ? 1 : 0, st);
    // df32 passes: precision DF32, or precision MIXED when the autotuner found the
    // double-float FFT faster than the matrix pass (it is also more accurate), or the
    // double-float transform of u1 in the tensor-core modes
    const bool dd = ((p->mixed == IDP_PRECISION_DF32 || (tensor_mode(p) && p->mixed_path == 1)) && allow_reduced) ||
                    (tensor_mode(p) && !allow_reduced && !fp64_only);
    int axes[3], na = 0;
    if (forward) {
        for (int s = skip_axis2 ? 1 : 2; s >= 0; --s)
            if (p->act[s]) axes[na++] = s;
    } else {
        for (int s = 0; s < 3; ++s)
            if (p->act[s]) axes[na++] = s;
    }
    for (int q = 0; q < na; ++q) {
        const int s = axes[q];
        DstPass a{};
        a.lines = p->dst_lines;
        a.in = (q == 0) ? in : dense(p, work);
        a.out = (q == na - 1) ? out : dense(p, work);
        a.add = (q == na - 1) ? add : View3{nullptr, 0, 0, 0};
        a.tab = (q == na - 1) ? tab : nullptr;
        a.n0 = p->ni[0]; a.n1 = p->ni[1]; a.n2 = p->ni[2];
        a.axis = s;
        a.M = p->M[s];
        FftTables t{};
        int rc;
        if (has_fft_dst(p->M[s])) {
            if ((rc = get_fft(p, p->M[s] / 2, &t))) return rc;
            a.tw = t.fwd;
            a.half = t.half;
            a.halfr = t.halfr;
            if ((rc = get_sin2(p, p->M[s], &a.sin2))) return rc;
        } else if ((rc = get_sinm(p, p->M[s], &a.sinm, dd ? 1 : 0))) {   // direct sums
            return rc;
        }
        if (dd) {
            // double-float arithmetic; intermediate passes keep double-float pairs
            a.dd = 1;
            a.in_dd = (q == 0) ? in_dd0 : 1;
            a.out_dd = (q == na - 1) ? 0 : 1;
            a.add_dd = 0;
            a.twd = t.fwdd;
            a.halfd = t.halfd;
            if (has_fft_dst(p->M[s])) a.sin2d = p->sin2d[p->M[s]];
        }
        Mark mk(p, IDP_KERNEL_DST, st);
        IDP_CK(launch_dst_pass(a, st));
    }
    return IDP_OK;
}

// in-place sine passes over a dense box b0 x b1 x b2 along axis 2, then axis 1
// (if M1 > 0), with panel counts M2 / M1
int dst_box(idp_plan p, double *x, int b0, int b1, int b2, int M2, int M1, cudaStream_t st)
{
    const int axes[2] = {2, 1};
    const int Ms[2] = {M2, M1};
    for (int q = 0; q < 2; ++q) {
        if (Ms[q] <= 0) continue;
        DstPass a{};
        const View3 v{x, (int64_t)b1 * b2, b2, 1};
        a.in = v; a.out = v; a.add = View3{nullptr, 0, 0, 0}; a.tab = nullptr;
        a.n0 = b0; a.n1 = b1; a.n2 = b2;
        a.axis = axes[q];
        a.M = Ms[q];
        FftTables t{};
        int rc;
        const bool ddm = p->mixed == IDP_PRECISION_DF32 || tensor_mode(p);
        if (has_fft_dst(Ms[q])) {
            if ((rc = get_fft(p, Ms[q] / 2, &t))) return rc;
            a.tw = t.fwd;
            a.half = t.half;
            a.halfr = t.halfr;
            if ((rc = get_sin2(p, Ms[q], &a.sin2))) return rc;
        } else if ((rc = get_sinm(p, Ms[q], &a.sinm, ddm ? 1 : 0))) {   // direct sums
            return rc;
        }
        if (ddm) {
            a.dd = 1;
            a.twd = t.fwdd;
            a.halfd = t.halfd;
            if (has_fft_dst(Ms[q])) a.sin2d = p->sin2d[Ms[q]];
        }
        Mark mk(p, IDP_KERNEL_DST_PARTS, st);
        IDP_CK(launch_dst_pass(a, st));
    }
    return IDP_OK;
}

// gtilde parts Q0, Q1, Q2 and their (d-1)-dimensional sine transforms
int gtilde_parts(idp_plan p, bool transform_parts, cudaStream_t st)
{
    {
        Mark mk(p, IDP_KERNEL_GTILDE, st);
        IDP_CK(launch_gtilde_planes(p->grid, p->coef, p->U, p->Q0, p->Q1, p->Q2, st));
    }
    if (!transform_parts) return IDP_OK;
    int rc;
    const int n0 = p->ni[0], n1 = p->ni[1], n2 = p->ni[2];
    if (p->d == 3 && n0 == n1 && n1 == n2) {
        // equal shapes: the three parts form one box of 6 layers
        if ((rc = dst_box(p, p->Q0, 6, n1, n2, p->M[2], p->M[1], st))) return rc;
    } else if (p->d == 3) {
        if ((rc = dst_box(p, p->Q0, 2, n1, n2, p->M[2], p->M[1], st))) return rc;
        if ((rc = dst_box(p, p->Q1, 2, n0, n2, p->M[2], p->M[0], st))) return rc;
        if ((rc = dst_box(p, p->Q2, 2, n0, n1, p->M[1], p->M[0], st))) return rc;
    } else {
        if ((rc = dst_box(p, p->Q1, 2, 1, n2, p->M[2], 0, st))) return rc;
        if ((rc = dst_box(p, p->Q2, 2, 1, n1, p->M[1], 0, st))) return rc;
    }
    Mark mk(p, IDP_KERNEL_GTILDE, st);
    IDP_CK(launch_layers_combine(p->Q0, p->d == 3 ? (int64_t)n1 * n2 : 0, p->Q1, (int64_t)n0 * n2, p->Q2,
                                 (int64_t)n0 * n1, 1, st));
    return IDP_OK;
}

// (d-1)-dimensional sine transforms of the layers of E (two per face)
int e_layers(idp_plan p, cudaStream_t st)
{
    int rc;
    const int n0 = p->ni[0], n1 = p->ni[1], n2 = p->ni[2];
    if (p->d == 3 && n0 == n1 && n1 == n2) {
        if ((rc = dst_box(p, p->E0, 12, n1, n2, p->M[2], p->M[1], st))) return rc;
    } else if (p->d == 3) {
        if ((rc = dst_box(p, p->E0, 4, n1, n2, p->M[2], p->M[1], st))) return rc;
        if ((rc = dst_box(p, p->E1, 4, n0, n2, p->M[2], p->M[0], st))) return rc;
        if ((rc = dst_box(p, p->E2, 4, n0, n1, p->M[1], p->M[0], st))) return rc;
    } else {
        if ((rc = dst_box(p, p->E1, 4, 1, n2, p->M[2], 0, st))) return rc;
        if ((rc = dst_box(p, p->E2, 4, 1, n1, p->M[1], 0, st))) return rc;
    }
    Mark mk(p, IDP_KERNEL_RHS6_EXPAND, st);
    IDP_CK(launch_layers_combine(p->E0, p->d == 3 ? (int64_t)n1 * n2 : 0, p->E1, (int64_t)n0 * n2, p->E2,
                                 (int64_t)n0 * n1, 2, st));
    return IDP_OK;
}

// Forward transform of rho scaled by 1/lambda_c into A, starting from the
// boundary stage 1a output: T0 = 2 * (real FFT of the zero-padded rows along
// axis 2), whose imaginary part at m = 1..M2-1 is -2 times the sine sums of
// the rows, i.e. -1/2 of the first sine pass (4 S).  The remaining passes run
// on that data and the factor -2 is in tabc2.
int transform_rho_from_T0(idp_plan p, cudaStream_t st)
{
    const View3 none{nullptr, 0, 0, 0};
    const int64_t row = 2 * (int64_t)(p->P[2] + 1);   // doubles per T0 row
    const View3 im{reinterpret_cast<double *>(p->T0) + 3, (int64_t)p->ni[1] * row, row, 2};
    const int dd = boundary_dd(p);   // T0 holds pairs
    return transform(p, im, p->A, dense(p, p->A), p->tabc2, none, true, st, true, true, dd);
}

// boundary values g into the boundary nodes of dst0 (and dst1 if not null).
// rho_src (optional): the node array that the first row transform reads instead
// of rho, copying its interior into rho for the later stages (a page-locked host
// buffer, through its device view: the upload then runs inside that pass)
int boundary(idp_plan p, const double *rho, double *dst0, double *dst1, cudaStream_t st,
             bool fork_rho = false, const double *rho_src = nullptr)
{
    Range rg(p, "idp:boundary values g");
    const View3 r = node_interior(p, rho);
    int rc;
    FftTables t;
    // double-float arithmetic for the 3-D convolutions in precision DF32 (and, on
    // request, in the tensor-core modes)
    const int dd = boundary_dd(p);
    // support flags of rho: set by the first row transform
    IDP_CK(cudaMemsetAsync(p->flags, 0, sizeof(int) * p->nflags, st));
    // stage 1a: along axis 2 -> T0[i0][i1][m2]; stage 1b: along axis 1 -> T1[i0][i2][m1]
    RfftPass a2{}, a1{};
    a2.in = rho_src ? node_interior(p, rho_src).p : r.p;
    a2.copy = rho_src ? r.p : nullptr;
    a2.is0 = r.s0; a2.is1 = r.s1; a2.is2 = r.s2;
    a2.out = p->T0;
    a2.os2 = 1; a2.os1 = p->P[2] + 1; a2.os0 = (int64_t)p->ni[1] * (p->P[2] + 1);
    a2.n0 = p->ni[0]; a2.n1 = p->ni[1]; a2.n2 = p->ni[2];
    a2.axis = 2; a2.M = p->M[2]; a2.P = p->P[2];
    if ((rc = get_fft(p, p->P[2], &t))) return rc;
    a2.t = t;
    a2.dd = dd;
    // the pass along axis 2 reads every value of rho once: it also marks which
    // rows and slices are non-zero (zero ones are skipped below; their
    // contributions are exactly zero)
    a2.fl_row2 = p->row2; a2.fl_row1 = p->row1;
    a2.fl_sl0 = p->sl[0]; a2.fl_sl1 = p->sl[1]; a2.fl_sl2 = p->sl[2];
    a1.in = r.p; a1.is0 = r.s0; a1.is1 = r.s1; a1.is2 = r.s2;
    a1.out = p->T1;
    a1.os1 = 1; a1.os2 = p->P[1] + 1; a1.os0 = (int64_t)p->ni[2] * (p->P[1] + 1);
    a1.n0 = p->ni[0]; a1.n1 = p->ni[1]; a1.n2 = p->ni[2];
    a1.axis = 1; a1.M = p->M[1]; a1.P = p->P[1];
    if ((rc = get_fft(p, p->P[1], &t))) return rc;
    a1.t = t;
    a1.dd = dd;
    a1.lineflag = p->row1;
    {
        Mark mk(p, IDP_KERNEL_RFFT, st);
        IDP_CK(launch_rfft_pass(a2, st));
    }
    if (fork_rho) {
        // the rest of the forward transform of rho runs beside the boundary stages
        IDP_CK(cudaEventRecord(p->fork, st));
        IDP_CK(cudaStreamWaitEvent(p->side, p->fork, 0));
        if ((rc = transform_rho_from_T0(p, p->side))) return rc;
        IDP_CK(cudaEventRecord(p->join, p->side));
    }
    // the faces of axes 0 and 1 read only T0: with fork_rho they start on their
    // own streams while the rest runs on st
    const bool conc = fork_rho && p->d == 3;
    if (conc) {
        IDP_CK(cudaEventRecord(p->fev[0], st));
        for (int i = 0; i < 2; ++i) IDP_CK(cudaStreamWaitEvent(p->fst[i], p->fev[0], 0));
    }
    {
        Mark mk(p, IDP_KERNEL_RFFT, st);
        IDP_CK(launch_rfft_pass(a1, st));
    }
    if (p->d == 2) {
        // faces of axis 1 (rows i1 = 0, M1; data along axis 2) and of axis 2
        for (int face = 1; face <= 2; ++face) {
            FacePass2D a{};
            const int other = face == 1 ? 2 : 1;
            if (face == 1) { a.T = p->T0; a.sp = p->P[2] + 1; a.sm = 1; }
            else { a.T = p->T1; a.sp = p->P[1] + 1; a.sm = 1; }
            a.np = p->ni[face];
            a.nm = p->P[other] + 1;
            a.khat = p->khat[face];
            a.acc = p->F;
            {
                Mark mk(p, IDP_KERNEL_FACE, st);
                IDP_CK(launch_face_pass_2d(a, st));
            }
            FaceC2R c{};
            c.in = p->F; c.nrows = 1; c.Mc = p->M[other]; c.Pc = p->P[other];
            c.dst0 = dst0; c.dst1 = dst1;
            c.base[0] = 0; c.base[1] = (int64_t)p->M[face] * p->ns[face];
            c.row_stride = 0; c.col_stride = p->ns[other];
            c.skip_row_edges = 0; c.skip_col_edges = (face == 2);
            if ((rc = get_fft(p, p->P[other], &t))) return rc;
            c.t = t;
            Mark mk(p, IDP_KERNEL_FACE_C2R, st);
            IDP_CK(launch_face_c2r(c, st));
        }
        return IDP_OK;
    }
    // 3-D: faces of axis a; b < c the other axes; data and strides per face
    for (int a_ = 0; a_ < 3; ++a_) {
        const int b = a_ == 0 ? 1 : 0;
        const int c = a_ == 2 ? 1 : 2;
        cudaStream_t sa = (conc && a_ < 2) ? p->fst[a_] : st;
        double2 *part = p->part + a_ * p->part_cap, *F = p->F + a_ * p->f_cap;
        FacePass f{};
        if (a_ == 0) { f.D = p->T0; f.sp = (int64_t)p->ni[1] * (p->P[2] + 1); f.sb = p->P[2] + 1; f.sc = 1; }
        else if (a_ == 1) { f.D = p->T0; f.sp = p->P[2] + 1; f.sb = (int64_t)p->ni[1] * (p->P[2] + 1); f.sc = 1; }
        else { f.D = p->T1; f.sp = p->P[1] + 1; f.sb = (int64_t)p->ni[2] * (p->P[1] + 1); f.sc = 1; }
        f.np = p->ni[a_];
        f.Mb = p->M[b];
        f.Pb = p->P[b];
        f.nc = p->P[c] + 1;
        f.khat = p->khat[a_];
        f.part = part;
        f.pchunk = p->pchunk[a_];
        if ((rc = get_fft(p, 2 * p->P[b], &t))) return rc;
        f.t = t;
        f.dd = dd;
        f.khatd = p->khatd[a_];
        f.sliceflag = p->sl[a_];
        {
            Mark mk(p, IDP_KERNEL_FACE, sa);
            IDP_CK(launch_face_pass(f, p->nchunk[a_], sa));
        }
        FaceInvB ib{};
        ib.part = part; ib.nchunk = p->nchunk[a_];
        ib.Mb = p->M[b]; ib.Pb = p->P[b]; ib.nc = f.nc; ib.out = F; ib.t = t;
        ib.dd = dd;
        {
            Mark mk(p, IDP_KERNEL_FACE_INVB, sa);
            IDP_CK(launch_face_inv_b(ib, sa));
        }
        FaceC2R cr{};
        cr.in = F; cr.nrows = p->M[b] + 1; cr.Mc = p->M[c]; cr.Pc = p->P[c];
        cr.dst0 = dst0; cr.dst1 = dst1;
        cr.base[0] = 0; cr.base[1] = (int64_t)p->M[a_] * p->ns[a_];
        cr.row_stride = p->ns[b]; cr.col_stride = p->ns[c];
        cr.skip_row_edges = (a_ >= 1);
        cr.skip_col_edges = (a_ == 2);
        if ((rc = get_fft(p, p->P[c], &t))) return rc;
        cr.t = t;
        cr.dd = dd;
        Mark mk(p, IDP_KERNEL_FACE_C2R, sa);
        IDP_CK(launch_face_c2r(cr, sa));
    }
    if (conc)
        for (int i = 0; i < 2; ++i) {
            IDP_CK(cudaEventRecord(p->fev[1 + i], p->fst[i]));
            IDP_CK(cudaStreamWaitEvent(st, p->fev[1 + i], 0));
        }
    return IDP_OK;
}

enum { RUN_PHI = 0 };

// Queue the stages of one solve.  stop: 0 = full solve into phi; otherwise an
// IDP_STAGE_* value whose result is written to `out`.
// d = 1 (section 5): phi* by one forward and one inverse sine pass, then g at
// the two ends and the straight line through them added inside
int enqueue_1d(idp_plan p, const double *rho, double *phi, int stop, cudaStream_t st)
{
    const View3 none{nullptr, 0, 0, 0};
    const size_t node_bytes = sizeof(double) * p->nodes;
    const int M = p->M[2];
    if (stop == 0 && p->hio_rho)
        IDP_CK(cudaMemcpyAsync(p->h_rho, p->hio_rho, node_bytes, cudaMemcpyHostToDevice, st));
    if (stop == IDP_STAGE_BOUNDARY || stop == IDP_STAGE_U1) {
        Mark mk(p, IDP_KERNEL_LINE1D, st);
        IDP_CK(launch_line1d(rho, phi, M, p->h[2], stop == IDP_STAGE_BOUNDARY ? LINE1D_ENDS : LINE1D_LINE, st));
        return IDP_OK;
    }
    if (stop != 0 && stop != IDP_STAGE_PHISTAR) return IDP_ESUPPORT;
    int rc;
    if (stop == IDP_STAGE_PHISTAR) IDP_CK(cudaMemsetAsync(phi, 0, node_bytes, st));
    if ((rc = transform(p, node_interior(p, rho), p->A, dense(p, p->A), p->tabc, none, true, st))) return rc;
    if ((rc = transform(p, dense(p, p->A), p->A, node_interior(p, phi), nullptr, none, false, st))) return rc;
    if (stop == IDP_STAGE_PHISTAR) return IDP_OK;
    Mark mk(p, IDP_KERNEL_LINE1D, st);
    IDP_CK(launch_line1d(rho, phi, M, p->h[2], LINE1D_ADD, st));
    return IDP_OK;
}

int enqueue_grid(idp_plan p, const double *rho, double *phi, int stop, cudaStream_t st);

// A padded plan: the interior nodes of the caller's rho go into the padded array
// (the rest of it stays zero: the caller's boundary entries of rho are not used,
// as in an unpadded solve), the solve runs on the padded grid, and phi is read
// back at the caller's nodes.  Full solves only.
int enqueue_padded(idp_plan p, const double *rho, double *phi, int stop, cudaStream_t st)
{
    if (stop != 0) return IDP_ESUPPORT;
    if (p->hio_rho)
        IDP_CK(cudaMemcpyAsync(p->h_rho, p->hio_rho, sizeof(double) * p->unodes, cudaMemcpyHostToDevice, st));
    int lo[3], ext[3];
    for (int s = 0; s < 3; ++s) {
        lo[s] = p->act[s] ? 1 : 0;
        ext[s] = p->act[s] ? p->un[s] - 2 : 1;
    }
    const int64_t u1 = p->un[2], u0 = (int64_t)p->un[1] * p->un[2];
    const int64_t n1 = p->n[2], n0 = (int64_t)p->n[1] * p->n[2];
    const int64_t uo = (int64_t)p->uoff[0] * n0 + (int64_t)p->uoff[1] * n1 + p->uoff[2];
    {
        Mark mk(p, IDP_KERNEL_PAD, st);
        IDP_CK(launch_box_copy(rho + lo[0] * u0 + lo[1] * u1 + lo[2], u0, u1,
                               p->rho_pad + uo + lo[0] * n0 + lo[1] * n1 + lo[2], n0, n1, ext[0], ext[1], ext[2],
                               st));
    }
    const double *hio = p->hio_rho;
    p->hio_rho = nullptr;
    const int rc = enqueue_grid(p, p->rho_pad, p->phi_pad, 0, st);
    p->hio_rho = hio;
    if (rc) return rc;
    Mark mk(p, IDP_KERNEL_PAD, st);
    IDP_CK(launch_box_copy(p->phi_pad + uo, n0, n1, phi, u0, u1, p->un[0], p->un[1], p->un[2], st));
    return IDP_OK;
}

int enqueue(idp_plan p, const double *rho, double *phi, int stop, cudaStream_t st)
{
    Range rg(p, stop ? "idp:stage" : "idp:solve");
    if (p->validate) {
        // validation mode: the caller's rho is checked first (in a host-buffer
        // solve it goes up in one copy, and the check reads the copy)
        const double *hio = p->hio_rho;
        if (hio) {
            IDP_CK(cudaMemcpyAsync(p->h_rho, hio, sizeof(double) * p->unodes, cudaMemcpyHostToDevice, st));
            p->hio_rho = nullptr;
        }
        {
            Mark mk(p, IDP_KERNEL_VALIDATE, st);
            IDP_CK(launch_validate_rho(rho, p->un[0], p->un[1], p->un[2], p->act[0], p->act[1], p->act[2],
                                       p->validate, p->d_val, st));
        }
        const int rc = p->padded ? enqueue_padded(p, rho, phi, stop, st) : enqueue_grid(p, rho, phi, stop, st);
        p->hio_rho = hio;
        return rc;
    }
    if (p->padded) return enqueue_padded(p, rho, phi, stop, st);
    return enqueue_grid(p, rho, phi, stop, st);
}

// one solve (or stage) on the plan's own grid
int enqueue_grid(idp_plan p, const double *rho, double *phi, int stop, cudaStream_t st)
{
    if (p->d == 1) return enqueue_1d(p, rho, phi, stop, st);
    int rc;
    const View3 none{nullptr, 0, 0, 0};
    const size_t node_bytes = sizeof(double) * p->nodes;
    if (stop == IDP_STAGE_BOUNDARY) {
        IDP_CK(cudaMemsetAsync(phi, 0, node_bytes, st));
        return boundary(p, rho, phi, nullptr, st);
    }
    if (stop == IDP_STAGE_PHISTAR) {
        IDP_CK(cudaMemsetAsync(phi, 0, node_bytes, st));
        if ((rc = transform(p, node_interior(p, rho), p->A, dense(p, p->A), p->tabc, none, true, st))) return rc;
        return transform(p, dense(p, p->A), p->A, node_interior(p, phi), nullptr, none, false, st);
    }
    // 0. the forward transform of rho does not depend on the boundary values:
    //    queue it on the side stream so it overlaps the boundary convolutions
    // (profiling keeps one stream so that every launch is timed on its own)
    const bool overlap_rho = (stop == 0) && !p->profiling;
    // FP64 / df32 transforms: the first pass of the forward transform of rho is
    // the imaginary part of the boundary's first real FFT (see transform_rho_from_T0)
    const bool rho_from_T0 = (stop == 0) && !(tensor_mode(p) && p->mixed_path == 0) &&
                             has_fft_dst(p->M[2]) && p->P[2] == p->M[2];
    // host-buffer solve: the first row transform reads rho from the host buffer
    // and leaves the device copy for the later stages; where rho is needed before
    // it (the tensor-core transform of rho starts at once), rho goes up first
    const double *rho_src = (stop == 0 && p->hio_rho && rho_from_T0) ? p->hio_view : nullptr;
    if (stop == 0 && p->hio_rho && !rho_src)
        IDP_CK(cudaMemcpyAsync(p->h_rho, p->hio_rho, sizeof(double) * p->nodes, cudaMemcpyHostToDevice, st));
    // the tensor-core transform of rho leaves out the eigenvalue factor tabc: the
    // expansion kernels below apply it (an FP64 table read in the epilogue of a
    // tensor-core pass is latency-bound there)
    const bool rho_unscaled = (stop == 0) && !rho_from_T0;
    const double *ascale = rho_unscaled ? p->tabc : nullptr;
    if (overlap_rho && !rho_from_T0) {
        IDP_CK(cudaEventRecord(p->fork, st));
        IDP_CK(cudaStreamWaitEvent(p->side, p->fork, 0));
        if ((rc = transform(p, node_interior(p, rho), p->A, dense(p, p->A), nullptr, none, true, p->side)))
            return rc;
        IDP_CK(cudaEventRecord(p->join, p->side));
    }
    // 1. boundary values: phi boundary and U boundary
    if ((rc = boundary(p, rho, stop == 0 ? phi : p->U, stop == 0 ? p->U : nullptr, st,
                       overlap_rho && rho_from_T0, rho_src)))
        return rc;
    // 2. gtilde on the boundary-adjacent layers, and the transforms of its parts
    if ((rc = gtilde_parts(p, stop != IDP_STAGE_GTILDE, st))) return rc;
    if (stop == IDP_STAGE_GTILDE) {
        IDP_CK(launch_gtilde_scatter(p->grid, p->Q0, p->Q1, p->Q2, phi, st));
        return IDP_OK;
    }
    // 3. the forward transform of rho, scaled by 1/lambda_c (on the side stream
    //    in a full solve, joined before A is first used)
    if (stop == 0 && !overlap_rho) {
        if (rho_from_T0) {
            if ((rc = transform_rho_from_T0(p, st))) return rc;
        } else if ((rc = transform(p, node_interior(p, rho), p->A, dense(p, p->A), nullptr, none, true, st))) {
            return rc;
        }
    }
    if (p->order == 4 && stop == 0) {
        if (overlap_rho) IDP_CK(cudaStreamWaitEvent(st, p->join, 0));
        // A += tab4 * S gtilde; phi = S A inside
        {
            Mark mk(p, IDP_KERNEL_GTILDE_EXPAND, st);
            IDP_CK(launch_gtilde_expand(p->grid, p->Q0, p->Q1, p->Q2, p->sin4, p->tab4, p->A, p->A, st, nullptr,
                                        nullptr, nullptr, 0, ascale));
        }
        return transform(p, dense(p, p->A), p->A, node_interior(p, phi), nullptr, none, false, st);
    }
    // 4. u1 = S B, B = tab4 * S gtilde; in a full solve also C = A + tabR * S gtilde,
    //    the solution coefficients less the layer correction (R_spec's share)
    if (stop == 0 && overlap_rho) IDP_CK(cudaStreamWaitEvent(st, p->join, 0));
    // the final transform takes u1 in C (S C + S B = S (C + B)), in every mode
    {
        Mark mk(p, IDP_KERNEL_GTILDE_EXPAND, st);
        IDP_CK(launch_gtilde_expand(p->grid, p->Q0, p->Q1, p->Q2, p->sin4, p->tab4, nullptr, p->B, st,
                                    p->tabR, p->A, stop == 0 ? p->C : nullptr, 1, ascale));
    }
    // u1 feeds the sixth differences of R, which amplify its rounding by ~1e4-1e7:
    // this inverse transform stays FP64 in the FP64 and DF32 modes, and is a
    // double-float one (48 bits, never the tensor cores) in the tensor-core modes
    if ((rc = transform(p, dense(p, p->B), p->B, node_interior(p, p->U), nullptr, none, false, st, false, false, 0,
                        false)))
        return rc;
    if (stop == IDP_STAGE_U1) {
        IDP_CK(cudaMemcpyAsync(phi, p->U, node_bytes, cudaMemcpyDeviceToDevice, st));
        return IDP_OK;
    }
    // 5. E = R - R_spec on the layers next to the faces: W of the odd continuation
    //    near the faces, R at the extrapolation taps (into A, free now), E
    {
        Mark mk(p, IDP_KERNEL_RHS6_W, st);
        IDP_CK(launch_rhs6_spectral(p->grid, p->coef, p->U, p->W, p->A, p->E0, p->E1, p->E2, 0, st));
    }
    {
        Mark mk(p, IDP_KERNEL_RHS6_CORE, st);
        IDP_CK(launch_rhs6_spectral(p->grid, p->coef, p->U, p->W, p->A, p->E0, p->E1, p->E2, 1, st));
    }
    {
        Mark mk(p, IDP_KERNEL_RHS6_EXTRAP, st);
        IDP_CK(launch_rhs6_spectral(p->grid, p->coef, p->U, p->W, p->A, p->E0, p->E1, p->E2, 2, st));
    }
    if (stop == IDP_STAGE_R) {
        // R = S (Lambda_R b) + E with b the coefficients of u1 (recomputed), as a
        // dense interior array
        {
            Mark mk(p, IDP_KERNEL_GTILDE_EXPAND, st);
            IDP_CK(launch_gtilde_expand(p->grid, p->Q0, p->Q1, p->Q2, p->sin4, p->tab4, nullptr, p->C, st));
        }
        IDP_CK(launch_rhs6_symbol(p->grid, p->ld, p->ldoff[1], p->ldoff[2], p->C, st));
        if ((rc = transform(p, dense(p, p->C), p->C, dense(p, phi), nullptr, none, false, st, false))) return rc;
        IDP_CK(launch_rhs6_e_scatter(p->grid, p->E0, p->E1, p->E2, phi, st));
        return IDP_OK;
    }
    // 6. the layer transforms of E; C += tab4 * S E;  phi = S C + u1 inside
    if ((rc = e_layers(p, st))) return rc;
    {
        Mark mk(p, IDP_KERNEL_RHS6_EXPAND, st);
        IDP_CK(launch_rhs6_e_expand(p->grid, p->E0, p->E1, p->E2, p->sin4, p->sin4b, p->tab4, p->C, st));
    }
    return transform(p, dense(p, p->C), p->C, node_interior(p, phi), nullptr, none, false, st);
}

// the plan's streams and events (graph capture forks and joins through them)
int plan_streams(idp_plan p)
{
    IDP_CK(cudaStreamCreateWithFlags(&p->side, cudaStreamNonBlocking));
    IDP_CK(cudaStreamCreateWithFlags(&p->bst, cudaStreamNonBlocking));
    if (!p->cap) IDP_CK(cudaStreamCreateWithFlags(&p->cap, cudaStreamNonBlocking));
    IDP_CK(cudaEventCreateWithFlags(&p->fork, cudaEventDisableTiming));
    IDP_CK(cudaEventCreateWithFlags(&p->join, cudaEventDisableTiming));
    for (int i = 0; i < 2; ++i) IDP_CK(cudaStreamCreateWithFlags(&p->fst[i], cudaStreamNonBlocking));
    for (int i = 0; i < 3; ++i) IDP_CK(cudaEventCreateWithFlags(&p->fev[i], cudaEventDisableTiming));
    return IDP_OK;
}

// d = 1: the sine-pass tables (made by plan_setup), the coefficient array and
// tabc = (2/M) / lambda_c(k) / 16 with lambda_c(k) = -(pi k / L)^2, L = M h: the
// forward sums scaled by 2/M and divided by the continuum eigenvalue (section 3);
// each sine pass returns 4 S x, hence the 1/16
int plan_setup_1d(idp_plan p)
{
    int rc;
    const int M = p->M[2], N = p->ni[2];
    if ((rc = p->alloc(&p->A, p->nint)) || (rc = p->alloc(&p->tabc, p->nint))) return rc;
    std::vector<double> tc(N);
    const double L = (double)M * p->h[2];
    for (int k = 1; k <= N; ++k) {
        const double w = 3.14159265358979323846 * k / L;
        tc[k - 1] = (2.0 / M) / (-(w * w)) / 16.0;
    }
    IDP_CK(cudaMemcpy(p->tabc, tc.data(), sizeof(double) * N, cudaMemcpyHostToDevice));
    return plan_streams(p);
}

int plan_setup(idp_plan p)
{
    int rc;
    // every table a solve uses is created here, so that solves (and their
    // graph capture) never allocate
    for (int s = 0; s < 3; ++s) {
        if (!p->act[s]) continue;
        FftTables t;
        const double *sn;
        const void *sm_;
        if ((has_fft_dst(p->M[s]) && ((rc = get_fft(p, p->M[s] / 2, &t)) || (rc = get_sin2(p, p->M[s], &sn)))) ||
            (!has_fft_dst(p->M[s]) && (rc = get_sinm(p, p->M[s], &sm_, 0))) ||
            (rc = get_fft(p, p->P[s], &t)) || (rc = get_fft(p, 2 * p->P[s], &t)))
            return rc;
    }
    if (p->padded) {
        if ((rc = p->alloc(&p->rho_pad, p->nodes)) || (rc = p->alloc(&p->phi_pad, p->nodes))) return rc;
        IDP_CK(cudaMemset(p->rho_pad, 0, sizeof(double) * p->nodes));
    }
    if (p->d == 1) return plan_setup_1d(p);
    // workspace
    if ((rc = p->alloc(&p->A, p->nint)) || (rc = p->alloc(&p->B, p->nint)) || (rc = p->alloc(&p->C, p->nint)) ||
        (rc = p->alloc(&p->U, p->nodes)) || (rc = p->alloc(&p->W, 3 * p->nodes)) ||
        (rc = p->alloc(&p->tabc, p->nint)) || (rc = p->alloc(&p->tab4, p->nint)) ||
        (rc = p->alloc(&p->tabc2, p->nint)))
        return rc;
    if ((rc = p->alloc(&p->T0, (int64_t)p->ni[0] * p->ni[1] * (p->P[2] + 1))) ||
        (rc = p->alloc(&p->T1, (int64_t)p->ni[0] * p->ni[2] * (p->P[1] + 1))))
        return rc;
    {
        const int64_t q0 = 2 * (int64_t)p->ni[1] * p->ni[2], q1 = 2 * (int64_t)p->ni[0] * p->ni[2],
                      q2 = 2 * (int64_t)p->ni[0] * p->ni[1];
        if ((rc = p->alloc(&p->Q0, q0 + q1 + q2))) return rc;
        p->Q1 = p->Q0 + q0;
        p->Q2 = p->Q1 + q1;
    }
    {
        const int64_t n0 = p->ni[0], n1 = p->ni[1], n2 = p->ni[2];
        p->nflags = n0 * n1 + n0 * n2 + n0 + n1 + n2;
        if ((rc = p->alloc(&p->flags, p->nflags))) return rc;
        p->row2 = p->flags;
        p->row1 = p->row2 + n0 * n1;
        p->sl[0] = p->row1 + n0 * n2;
        p->sl[1] = p->sl[0] + n0;
        p->sl[2] = p->sl[1] + n1;
    }
    if ((rc = plan_streams(p))) return rc;
    {
        std::vector<double> s4;
        for (int s = 0; s < 3; ++s) {
            if (!p->act[s]) continue;
            for (int k = 0; k < p->ni[s]; ++k) s4.push_back(4.0 * sinpi_frac(k + 1, p->M[s]));
        }
        if ((rc = p->alloc(&p->sin4, (int64_t)s4.size()))) return rc;
        IDP_CK(cudaMemcpy(p->sin4, s4.data(), sizeof(double) * s4.size(), cudaMemcpyHostToDevice));
        std::vector<double> s4b;
        for (int s = 0; s < 3; ++s) {
            if (!p->act[s]) continue;
            for (int k = 0; k < p->ni[s]; ++k) s4b.push_back(4.0 * sinpi_frac(2 * (k + 1), p->M[s]));
        }
        if ((rc = p->alloc(&p->sin4b, (int64_t)s4b.size()))) return rc;
        IDP_CK(cudaMemcpy(p->sin4b, s4b.data(), sizeof(double) * s4b.size(), cudaMemcpyHostToDevice));
    }
    {
        // layers of E (two per face): E0 [2][2][n1][n2] (3-D), E1 [2][2][n0][n2], E2 [2][2][n0][n1]
        const int64_t n0 = p->ni[0], n1 = p->ni[1], n2 = p->ni[2];
        const int64_t e0 = p->d == 3 ? 4 * n1 * n2 : 0, e1 = 4 * n0 * n2, e2 = 4 * n0 * n1;
        if ((rc = p->alloc(&p->E0, e0 + e1 + e2))) return rc;
        p->E1 = p->E0 + e0;
        p->E2 = p->E1 + e1;
        if ((rc = p->alloc(&p->tabR, p->nint))) return rc;
    }
    IDP_CK(cudaMemset(p->U, 0, sizeof(double) * p->nodes));
    IDP_CK(cudaMemset(p->W, 0, sizeof(double) * 3 * p->nodes));

    // eigenvalue tables (sections 3 and 5)
    {
        std::vector<double> lc, ld;
        int64_t off[3] = {0, 0, 0};
        for (int s = 0; s < 3; ++s) {
            off[s] = (int64_t)lc.size();
            if (!p->act[s]) { lc.push_back(0.0); ld.push_back(0.0); continue; }
            const double L = p->M[s] * p->h[s];
            for (int k = 1; k < p->M[s]; ++k) {
                lc.push_back(-(M_PI * M_PI) * (double)k * k / (L * L));
                const double sn = sinpi_frac(k, 2 * p->M[s]);
                ld.push_back(-(4.0 / (p->h[s] * p->h[s])) * sn * sn);
            }
        }
        double *dlc, *dld;
        if ((rc = p->alloc(&dlc, (int64_t)lc.size())) || (rc = p->alloc(&dld, (int64_t)ld.size()))) return rc;
        IDP_CK(cudaMemcpy(dlc, lc.data(), sizeof(double) * lc.size(), cudaMemcpyHostToDevice));
        IDP_CK(cudaMemcpy(dld, ld.data(), sizeof(double) * ld.size(), cudaMemcpyHostToDevice));
        double sc = 1.0;
        int da = 0;
        for (int s = 0; s < 3; ++s)
            if (p->act[s]) { sc *= 2.0 / p->M[s]; ++da; }
        for (int q = 0; q < 2 * da; ++q) sc *= 0.25;   // each sine pass returns 4 S x
        IDP_CK(launch_eigen_tables(p->grid, dlc, dld, off[1], off[2], sc, p->tabc, p->tab4, p->tabR, 0));
        IDP_CK(launch_eigen_tables(p->grid, dlc, dld, off[1], off[2], -2.0 * sc, p->tabc2, p->B, nullptr, 0));
        p->ld = dld;
        for (int s = 0; s < 3; ++s) p->ldoff[s] = off[s];
    }

    // kernel spectra of the boundary convolutions (section 4)
    if (p->d == 2) {
        int64_t fmax = 0;
        for (int face = 1; face <= 2; ++face) {
            const int other = face == 1 ? 2 : 1;
            const int Mb = p->P[other];   // spectra of the cyclic kernel of length 2P
            const int np = p->ni[face];
            if ((rc = p->alloc(&p->khat[face], (int64_t)np * (Mb + 1)))) return rc;
            double *kb, *tb;
            if ((rc = p->alloc(&kb, (int64_t)np * (Mb + 1))) || (rc = p->alloc(&tb, (int64_t)(Mb + 1) * (Mb + 1))))
                return rc;
            KernelFill kf{kb, 2, np, Mb, 0, p->h[face], p->h[other], 0.0, 0, 0};
            IDP_CK(launch_kernel_fill(kf, 0));
            // DCT-I table Cb[t][m] = w_t cos(pi m t / Mb) * h_a h_b / (4 Mb)
            std::vector<double> cb((size_t)(Mb + 1) * (Mb + 1));
            const double sc = p->h[face] * p->h[other] / (4.0 * Mb);
            for (int tt = 0; tt <= Mb; ++tt)
                for (int m = 0; m <= Mb; ++m)
                    cb[(size_t)tt * (Mb + 1) + m] = ((tt == 0 || tt == Mb) ? 1.0 : 2.0) *
                                                    cospi_frac((int64_t)m * tt, Mb) * sc;
            IDP_CK(cudaMemcpy(tb, cb.data(), sizeof(double) * cb.size(), cudaMemcpyHostToDevice));
            IDP_CK(launch_gemm_batched(np, Mb + 1, Mb + 1, kb, Mb + 1, 0, tb, Mb + 1, 0, p->khat[face], Mb + 1, 0,
                                       1, 0));
            fmax = std::max<int64_t>(fmax, 2 * (Mb + 1));
        }
        if ((rc = p->alloc(&p->F, fmax))) return rc;
    } else {
        int64_t pmax = 0, fmax = 0;
        for (int a_ = 0; a_ < 3; ++a_) {
            const int b = a_ == 0 ? 1 : 0;
            const int c = a_ == 2 ? 1 : 2;
            // spectra of the cyclic kernel of length 2P along b and c
            const int Mb = p->P[b], Mc = p->P[c], np = p->ni[a_];
            const int L = 2 * Mb;
            const int TC = face_columns_per_block(L);
            const int tiles = (Mc + 1 + TC - 1) / TC;
            // one wave of resident blocks; fewer chunks = fewer partial sums
            int nsm = 152;
            cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, p->dev);
            const int slots = nsm * face_blocks_per_sm(L);
            int nch = std::max(1, std::min(np, slots / tiles));
            int pch = (np + nch - 1) / nch;
            nch = (np + pch - 1) / pch;
            p->nchunk[a_] = nch;
            p->pchunk[a_] = pch;
            pmax = std::max<int64_t>(pmax, (int64_t)nch * 2 * L * (Mc + 1));
            fmax = std::max<int64_t>(fmax, (int64_t)2 * (Mb + 1) * (Mc + 1));
            const int64_t per = (int64_t)(Mb + 1) * (Mc + 1);
            if ((rc = p->alloc(&p->khat[a_], (int64_t)np * per))) return rc;
            p->khat_n[a_] = (int64_t)np * per;
            // build in slabs of slices to bound the temporaries
            const int slab = std::max(1, (int)std::min<int64_t>(np, (int64_t)(64 << 20) / (per * 8)));
            double *kb, *yb, *tcb, *tbb;
            if ((rc = p->alloc(&kb, (int64_t)slab * per)) || (rc = p->alloc(&yb, (int64_t)slab * per)) ||
                (rc = p->alloc(&tcb, (int64_t)(Mc + 1) * (Mc + 1))) || (rc = p->alloc(&tbb, (int64_t)(Mb + 1) * (Mb + 1))))
                return rc;
            // the spectra are stored transposed, [slice][frequency c][frequency b]:
            //   khat^T = Cc^T K^T Cb^T  with  K^T[t_c][t_b] = G(d_p, t_b h_b, t_c h_c)
            std::vector<double> cct((size_t)(Mc + 1) * (Mc + 1)), cbt((size_t)(Mb + 1) * (Mb + 1));
            const double sc = p->h[0] * p->h[1] * p->h[2] / (8.0 * Mb * Mc);
            for (int m = 0; m <= Mc; ++m)        // Cc^T[m][t] = w_t cos(pi m t / Mc) * sc
                for (int tt = 0; tt <= Mc; ++tt)
                    cct[(size_t)m * (Mc + 1) + tt] = ((tt == 0 || tt == Mc) ? 1.0 : 2.0) *
                                                     cospi_frac((int64_t)m * tt, Mc) * sc;
            for (int tt = 0; tt <= Mb; ++tt)     // Cb^T[t][m] = w_t cos(pi m t / Mb)
                for (int m = 0; m <= Mb; ++m)
                    cbt[(size_t)tt * (Mb + 1) + m] = ((tt == 0 || tt == Mb) ? 1.0 : 2.0) *
                                                     cospi_frac((int64_t)m * tt, Mb);
            IDP_CK(cudaMemcpy(tcb, cct.data(), sizeof(double) * cct.size(), cudaMemcpyHostToDevice));
            IDP_CK(cudaMemcpy(tbb, cbt.data(), sizeof(double) * cbt.size(), cudaMemcpyHostToDevice));
            for (int p0 = 0; p0 < np; p0 += slab) {
                const int cnt = std::min(slab, np - p0);
                KernelFill kf{kb, 3, cnt, Mb, Mc, p->h[a_], p->h[b], p->h[c], p0, 1};
                IDP_CK(launch_kernel_fill(kf, 0));
                // Y^T = Cc^T K^T: rows (frequency c) x cols (t_b)
                IDP_CK(launch_gemm_batched(Mc + 1, Mb + 1, Mc + 1, tcb, Mc + 1, 0, kb, Mb + 1, per, yb, Mb + 1, per,
                                           cnt, 0));
                // khat^T = Y^T Cb^T: rows (frequency c) x cols (frequency b)
                IDP_CK(launch_gemm_batched(Mc + 1, Mb + 1, Mb + 1, yb, Mb + 1, per, tbb, Mb + 1, 0,
                                           p->khat[a_] + (int64_t)p0 * per, Mb + 1, per, cnt, 0));
            }
        }
        if ((rc = p->alloc(&p->part, 3 * pmax)) || (rc = p->alloc(&p->F, 3 * fmax))) return rc;
        p->part_cap = pmax;
        p->f_cap = fmax;
    }
    IDP_CK(cudaDeviceSynchronize());
    return IDP_OK;
}

// Times candidate settings on the plan's own buffers and keeps the fastest:
// the slice chunking of each 3-D face pass, and (precision MIXED) the
// tensor-core matrix pass versus the df32 FFT pass for the reduced-precision
// transforms.  Results depend only on timing, not on the data.
int autotune(idp_plan p)
{
    if (p->d == 1) {   // one line per pass: nothing to choose
        p->tuned = 1;
        return IDP_OK;
    }
    cudaStream_t st = p->cap;
    cudaEvent_t e0, e1;
    IDP_CK(cudaEventCreate(&e0));
    IDP_CK(cudaEventCreate(&e1));
    int rc = IDP_OK;
    auto timed = [&](auto &&fn) -> float {
        float best = 1e30f;
        for (int r = 0; r < 4 && !rc; ++r) {
            cudaEventRecord(e0, st);
            rc = fn();
            cudaEventRecord(e1, st);
            cudaEventSynchronize(e1);
            float ms = 0.f;
            cudaEventElapsedTime(&ms, e0, e1);
            if (r > 0 && ms < best) best = ms;   // first run warms up
        }
        return best;
    };
    if (p->d == 3) {
        for (int a_ = 0; a_ < 3 && !rc; ++a_) {
            const int b = a_ == 0 ? 1 : 0, c = a_ == 2 ? 1 : 2;
            const int np = p->ni[a_], L = 2 * p->P[b], nc = p->P[c] + 1;
            const int n0 = p->nchunk[a_];
            // around the set-up's choice, and the chunk counts that fill whole waves
            // of resident blocks (one column block per chunk: the block count is
            // chunks x column blocks, and a part-filled last wave leaves SMs idle)
            std::vector<int> cands = {std::max(1, n0 / 2), n0, std::min(np, 2 * n0), std::min(np, 4 * n0)};
            {
                int nsm = 152;
                cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, p->dev);
                const int slots = nsm * face_blocks_per_sm(L);
                const int tiles = (nc + face_columns_per_block(L) - 1) / face_columns_per_block(L);
                for (int w = 1; w <= 8; ++w) {
                    const int c = std::min(np, std::max(1, (int)(((int64_t)w * slots + tiles - 1) / tiles)));
                    if (std::find(cands.begin(), cands.end(), c) == cands.end()) cands.push_back(c);
                }
            }
            int best_n = n0, best_p = p->pchunk[a_];
            float best_t = 1e30f;
            for (size_t ci = 0; ci < cands.size() && !rc; ++ci) {
                const int pch = (np + cands[ci] - 1) / cands[ci];
                const int nch = (np + pch - 1) / pch;
                if ((int64_t)nch * 2 * L * nc > p->part_cap) {
                    double2 *np_part;
                    if ((rc = p->alloc(&np_part, 3 * (int64_t)nch * 2 * L * nc))) break;
                    p->part = np_part;
                    p->part_cap = (int64_t)nch * 2 * L * nc;
                }
                FacePass f{};
                if (a_ == 0) { f.D = p->T0; f.sp = (int64_t)p->ni[1] * (p->P[2] + 1); f.sb = p->P[2] + 1; f.sc = 1; }
                else if (a_ == 1) { f.D = p->T0; f.sp = p->P[2] + 1; f.sb = (int64_t)p->ni[1] * (p->P[2] + 1); f.sc = 1; }
                else { f.D = p->T1; f.sp = p->P[1] + 1; f.sb = (int64_t)p->ni[2] * (p->P[1] + 1); f.sc = 1; }
                f.np = np; f.Mb = p->M[b]; f.Pb = p->P[b]; f.nc = nc; f.khat = p->khat[a_]; f.part = p->part;
                f.pchunk = pch;
                FftTables t;
                if ((rc = get_fft(p, L, &t))) break;
                f.t = t;
                // the chunk count sets the work of the face pass and of the
                // partial-sum reduction that follows it: time both
                FaceInvB ib{};
                ib.part = p->part; ib.nchunk = nch; ib.Mb = p->M[b]; ib.Pb = p->P[b]; ib.nc = nc; ib.out = p->F;
                ib.t = t;
                const float ms = timed([&]() -> int {
                    cudaError_t e = launch_face_pass(f, nch, st);
                    if (e == cudaSuccess) e = launch_face_inv_b(ib, st);
                    return e == cudaSuccess ? IDP_OK : cuda_fail(e, "face pass (autotune)");
                });
                if (ms < best_t) { best_t = ms; best_n = nch; best_p = pch; }
            }
            p->nchunk[a_] = best_n;
            p->pchunk[a_] = best_p;
        }
    }
    if (!rc) {
        // block shape of the full-volume sine passes: the default, 8 lines on 256
        // threads, 8 lines on 128 threads (M = 128), 32 lines (M = 128), 16
        // lines (M = 256) or 4 lines on 128 threads (M = 256, 512); shapes that do
        // not apply to a length fall back to the default.  Timed in whole solves: the transform of rho runs beside the
        // boundary stages, so what a shape costs depends on what runs next to it
        // (a shape can win alone and lose in the solve).  The density is a smooth
        // bump over the middle of the box, zero near the boundary.
        std::vector<double> hr((size_t)p->nodes, 0.0);
        for (int i0 = 0; i0 < p->n[0]; ++i0)
            for (int i1 = 0; i1 < p->n[1]; ++i1)
                for (int i2 = 0; i2 < p->n[2]; ++i2) {
                    const int ii[3] = {i0, i1, i2};
                    double r2 = 0.0;
                    for (int s = 0; s < 3; ++s)
                        if (p->act[s]) {
                            const double t = 2.0 * ii[s] / p->M[s] - 1.0;
                            r2 += t * t;
                        }
                    const double q = 1.0 - r2 / 0.36;
                    hr[((size_t)i0 * p->n[1] + i1) * p->n[2] + i2] = q > 0.0 ? q * q * q * q : 0.0;
                }
        double *trho = nullptr, *tphi = nullptr;
        cudaError_t e = cudaMalloc(&trho, sizeof(double) * p->nodes);
        if (e == cudaSuccess) e = cudaMalloc(&tphi, sizeof(double) * p->nodes);
        if (e == cudaSuccess) e = cudaMemcpy(trho, hr.data(), sizeof(double) * p->nodes, cudaMemcpyHostToDevice);
        if (e != cudaSuccess) rc = cuda_fail(e, "autotune buffers");
        const int opts[6] = {0, 8, -8, 32, 16, 4};
        int best = 0;
        float bt = 1e30f;
        for (int i = 0; i < 6 && !rc; ++i) {
            p->dst_lines = opts[i];
            const float t = timed([&]() -> int { return enqueue_grid(p, trho, tphi, 0, st); });
            if (t < bt) { bt = t; best = opts[i]; }
        }
        cudaStreamSynchronize(st);
        if (trho) cudaFree(trho);
        if (tphi) cudaFree(tphi);
        p->dst_lines = best;
    }
    if (!rc && tensor_mode(p)) {
        const View3 none{nullptr, 0, 0, 0};
        float tm[2];
        for (int path = 0; path < 2 && !rc; ++path) {
            p->mixed_path = path;
            tm[path] = timed([&]() -> int {
                return transform(p, dense(p, p->C), p->C, dense(p, p->C), nullptr, none, false, st);
            });
        }
        p->mixed_path = (tm[1] < tm[0]) ? 1 : 0;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    IDP_CK(cudaStreamSynchronize(st));
    p->tuned = 1;
    ++p->version;
    if (p->gexec) {
        cudaGraphExecDestroy(p->gexec);
        p->gexec = nullptr;
    }
    return rc;
}

bool overlap(const void *a, size_t na, const void *b, size_t nb)
{
    const char *x = (const char *)a, *y = (const char *)b;
    return x < y + nb && y < x + na;
}

int run_solve(idp_plan p, const double *rho, double *phi, cudaStream_t st)
{
    p->last = st;
    p->last_valid = 1;
    // a stall test is never baked into a graph, and NVTX ranges recorded while one is
    // captured would not recur on its replays
    if (!p->use_graph || p->stall_test || p->nvtx) {
        p->launches = 0;
        return enqueue(p, rho, phi, 0, st);
    }
    if (!p->gexec || p->g_rho != rho || p->g_phi != phi) {
        if (!p->cap) IDP_CK(cudaStreamCreateWithFlags(&p->cap, cudaStreamNonBlocking));
        IDP_CK(cudaStreamBeginCapture(p->cap, cudaStreamCaptureModeThreadLocal));
        p->launches = 0;
        int rc = enqueue(p, rho, phi, 0, p->cap);
        cudaGraph_t g = nullptr;
        cudaError_t e = cudaStreamEndCapture(p->cap, &g);
        if (rc) {
            if (g) cudaGraphDestroy(g);
            return rc;
        }
        if (e != cudaSuccess) return cuda_fail(e, "cudaStreamEndCapture");
        if (p->gexec) {
            cudaGraphExecDestroy(p->gexec);
            p->gexec = nullptr;
        }
        e = cudaGraphInstantiate(&p->gexec, g, 0);
        cudaGraphDestroy(g);
        if (e != cudaSuccess) return cuda_fail(e, "cudaGraphInstantiate");
        p->g_rho = rho;
        p->g_phi = phi;
    }
    IDP_CK(cudaGraphLaunch(p->gexec, st));
    return IDP_OK;
}

// device view of page-locked (or registered, mapped) host memory: the address at
// which kernels read and write it directly; null for other memory
double *device_view(const void *ptr)
{
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, ptr) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    return at.type == cudaMemoryTypeHost ? static_cast<double *>(at.devicePointer) : nullptr;
}

// a solve from page-locked host buffers: the first row transform reads rho through
// the buffer's device view (leaving a device copy for the later stages), and the
// kernels that produce phi (the boundary values and the last sine pass) write the
// host buffer directly, so that the upload and the download run inside those
// kernels instead of before and after them.  Its own cached graph, keyed by the
// host pointers and the plan's settings.
int run_solve_host(idp_plan p, const double *rho_h, double *phi_h, double *phi_view, cudaStream_t st)
{
    p->last = st;
    p->last_valid = 1;
    if (!p->hexec || p->hg_rho != rho_h || p->hg_phi != phi_h || p->hg_version != p->version) {
        IDP_CK(cudaStreamBeginCapture(p->cap, cudaStreamCaptureModeThreadLocal));
        p->hio_rho = rho_h;
        p->hio_view = device_view(rho_h);
        int rc = enqueue(p, p->h_rho, phi_view, 0, p->cap);
        p->hio_rho = nullptr;
        p->hio_view = nullptr;
        cudaGraph_t g = nullptr;
        cudaError_t e = cudaStreamEndCapture(p->cap, &g);
        if (rc) {
            if (g) cudaGraphDestroy(g);
            return rc;
        }
        if (e != cudaSuccess) return cuda_fail(e, "cudaStreamEndCapture");
        if (p->hexec) {
            cudaGraphExecDestroy(p->hexec);
            p->hexec = nullptr;
        }
        e = cudaGraphInstantiate(&p->hexec, g, 0);
        cudaGraphDestroy(g);
        if (e != cudaSuccess) return cuda_fail(e, "cudaGraphInstantiate");
        p->hg_rho = rho_h;
        p->hg_phi = phi_h;
        p->hg_version = p->version;
    }
    IDP_CK(cudaGraphLaunch(p->hexec, st));
    return IDP_OK;
}

int create_plan(idp_plan *out, int d, const int64_t n[], const double h[], int order, int exact)
{
    if (!out || !n || !h) return IDP_EINVAL;
    *out = nullptr;
    if (d < 1 || d > 3) return IDP_EINVAL;
    if (order != 4 && order != 6) return IDP_EINVAL;
    for (int s = 0; s < d; ++s) {
        if (!(h[s] > 0.0) || !std::isfinite(h[s])) return IDP_EINVAL;
        if (n[s] < (exact ? 8 : 3)) return IDP_EINVAL;
        if (exact ? n[s] - 1 > 512 : !padded_panels(n[s] - 1)) return IDP_ESUPPORT;
    }
    idp_plan p = new (std::nothrow) idp_plan_s();
    if (!p) return IDP_ENOMEM;
    p->d = d;
    p->order = order;
    p->exact = exact;
    p->serial = g_serial.fetch_add(1);
    const int o = 3 - d;
    for (int s = 0; s < d; ++s) {
        // an unsupported panel count is padded to the next supported one, the
        // extra panels split between the two ends (h unchanged); an exact plan
        // solves on the given grid
        const int64_t Mp = exact ? n[s] - 1 : padded_panels(n[s] - 1);
        p->n[s + o] = (int)Mp + 1;
        p->un[s + o] = (int)n[s];
        p->uoff[s + o] = (int)((Mp - (n[s] - 1)) / 2);
        if (Mp != n[s] - 1) p->padded = 1;
        p->h[s + o] = h[s];
        p->act[s + o] = 1;
    }
    p->unodes = (int64_t)p->un[0] * p->un[1] * p->un[2];
    for (int s = 0; s < 3; ++s) {
        p->M[s] = p->n[s] - 1;
        p->P[s] = p->act[s] ? conv_half(p->M[s]) : p->M[s];
        p->ni[s] = p->act[s] ? p->n[s] - 2 : 1;
    }
    p->ns[2] = 1; p->ns[1] = p->n[2]; p->ns[0] = (int64_t)p->n[1] * p->n[2];
    p->is[2] = 1; p->is[1] = p->ni[2]; p->is[0] = (int64_t)p->ni[1] * p->ni[2];
    p->nodes = (int64_t)p->n[0] * p->n[1] * p->n[2];
    p->nint = (int64_t)p->ni[0] * p->ni[1] * p->ni[2];
    p->grid = Grid3{d, p->n[0], p->n[1], p->n[2], p->h[0], p->h[1], p->h[2]};
    p->coef = make_stencil_coef(p->grid);
    int rc;
    cudaError_t e = cudaGetDevice(&p->dev);
    if (e != cudaSuccess) rc = cuda_fail(e, "cudaGetDevice");
    else if (!(rc = ensure_attributes(p->dev))) rc = plan_setup(p);
    if (rc) {
        idp_destroy_plan(p);
        return rc;
    }
    *out = p;
    return IDP_OK;
}

}  // namespace

extern "C" {

int idp_create_plan(idp_plan *out, int d, const int64_t n[], const double h[], int order)
{
    return create_plan(out, d, n, h, order, 0);
}

int idp_create_plan_exact(idp_plan *out, int d, const int64_t n[], const double h[], int order)
{
    return create_plan(out, d, n, h, order, 1);
}

int idp_plan_set(idp_plan p, int key, int64_t value)
{
    if (!p) return IDP_EINVAL;
    if (key == IDP_KEY_USE_GRAPH) {
        p->use_graph = value ? 1 : 0;
        return IDP_OK;
    }
    if (key == IDP_KEY_NVTX) {
        p->nvtx = value ? 1 : 0;
        return IDP_OK;
    }
    if (key == IDP_KEY_AUTOTUNE) {
        if (!value) return IDP_OK;
        return autotune(p);
    }
    if (key == IDP_KEY_DST_SHAPE) {
        if (value != 0 && value != 8 && value != -8 && value != 32 && value != 16 && value != 4) return IDP_EINVAL;
        p->dst_lines = (int)value;
        ++p->version;
        if (p->gexec) {
            cudaGraphExecDestroy(p->gexec);
            p->gexec = nullptr;
        }
        return IDP_OK;
    }
    if (key == IDP_KEY_VALIDATE) {
        if (value < 0 || value > 1 << 20) return IDP_EINVAL;
        if (value && !p->d_val) {
            int rc;
            if ((rc = p->alloc(&p->d_val, 1))) return rc;
            IDP_CK(cudaMemset(p->d_val, 0, sizeof(int)));
        }
        p->validate = (int)value;
        ++p->version;
        if (p->gexec) {
            cudaGraphExecDestroy(p->gexec);
            p->gexec = nullptr;
        }
        return IDP_OK;
    }
    if (key == IDP_KEY_MIXED_BOUNDARY_DF32) {
        if (value != 0 && value != 1) return IDP_EINVAL;
        if (value && p->d == 3 && !p->khatd[0]) {
            int rc;
            for (int a_ = 0; a_ < 3; ++a_) {
                if ((rc = p->alloc(&p->khatd[a_], p->khat_n[a_]))) return rc;
                IDP_CK(launch_to_dd(p->khat[a_], p->khatd[a_], p->khat_n[a_], 0));
            }
            IDP_CK(cudaDeviceSynchronize());
        }
        if (p->mixed_bdd != (int)value) {
            p->mixed_bdd = (int)value;
            ++p->version;
            if (p->gexec) {
                cudaGraphExecDestroy(p->gexec);
                p->gexec = nullptr;
            }
        }
        return IDP_OK;
    }
    if (key == IDP_KEY_GUARD_TEST) {
        // test hook: overwrite (1) or restore (0) the first byte of the guard
        // region in front of the plan's first buffer; the write stays inside
        // that allocation
        if (value != 0 && value != 1) return IDP_EINVAL;
        if (p->guarded.empty()) return IDP_ESUPPORT;
        IDP_CK(cudaDeviceSynchronize());
        IDP_CK(cudaMemset(p->guarded.front().first, value ? 0x5A : idp_plan_s::GUARD_BYTE, 1));
        IDP_CK(cudaDeviceSynchronize());
        return IDP_OK;
    }
    if (key == IDP_KEY_STALL_TEST) {
        if (!tensor_mode(p)) return IDP_EINVAL;
        p->stall_test = value ? 1 : 0;
        ++p->version;
        if (p->gexec) {
            cudaGraphExecDestroy(p->gexec);
            p->gexec = nullptr;
        }
        return IDP_OK;
    }
    if (key == IDP_KEY_PRECISION) {
        if (value != IDP_PRECISION_FP64 && value != IDP_PRECISION_MIXED_BF16X3 && value != IDP_PRECISION_DF32 &&
            value != IDP_PRECISION_MIXED_TF32X3)
            return IDP_EINVAL;
        if (p->d == 1 && value != IDP_PRECISION_FP64) return IDP_ESUPPORT;
        if (value == IDP_PRECISION_MIXED_BF16X3 || value == IDP_PRECISION_MIXED_TF32X3) {
            int rc;
            if (!p->d_err) {
                if ((rc = p->alloc(&p->d_err, 1))) return rc;
                IDP_CK(cudaMemset(p->d_err, 0, sizeof(int)));
            }
            for (int s = 0; s < 2; ++s)
                for (int q = 0; q < 2; ++q)
                    if (!p->t32[s][q] && (rc = p->alloc(&p->t32[s][q], t32_count(p)))) return rc;
            for (int s = 0; s < 3; ++s) {
                const void *img;
                if (p->act[s] &&
                    (rc = get_mp_image(p, p->M[s], value == IDP_PRECISION_MIXED_TF32X3 ? 1 : 0, &img)))
                    return rc;
            }
        }
        if (value == IDP_PRECISION_DF32 && p->d == 3 && !p->khatd[0]) {
            int rc;
            for (int a_ = 0; a_ < 3; ++a_) {
                if ((rc = p->alloc(&p->khatd[a_], p->khat_n[a_]))) return rc;
                IDP_CK(launch_to_dd(p->khat[a_], p->khatd[a_], p->khat_n[a_], 0));
            }
            IDP_CK(cudaDeviceSynchronize());
        }
        if (p->mixed != (int)value) {
            p->mixed = (int)value;
            p->mixed_path = 0;
            ++p->version;
            if (p->gexec) {
                cudaGraphExecDestroy(p->gexec);
                p->gexec = nullptr;
            }
        }
        return IDP_OK;
    }
    return IDP_EINVAL;
}

int idp_solve(idp_plan p, const double *rho, double *phi, void *stream)
{
    if (!p || !rho || !phi) return IDP_EINVAL;
    const size_t b = sizeof(double) * p->unodes;
    if (overlap(rho, b, phi, b)) return IDP_EALIAS;
    return run_solve(p, rho, phi, (cudaStream_t)stream);
}

int idp_solve_host(idp_plan p, const double *rho_host, double *phi_host, void *stream)
{
    if (!p || !rho_host || !phi_host) return IDP_EINVAL;
    const size_t b = sizeof(double) * p->unodes;
    if (overlap(rho_host, b, phi_host, b)) return IDP_EALIAS;
    int rc;
    if (!p->h_rho && ((rc = p->alloc(&p->h_rho, p->unodes)) || (rc = p->alloc(&p->h_phi, p->unodes)))) return rc;
    cudaStream_t st = (cudaStream_t)stream;
    double *phi_view = nullptr;
    if (p->use_graph && !p->stall_test && !p->nvtx && device_view(rho_host) && (phi_view = device_view(phi_host))) {
        // page-locked buffers: phi is written in place by the kernels
        if ((rc = run_solve_host(p, rho_host, phi_host, phi_view, st))) return rc;
    } else {
        IDP_CK(cudaMemcpyAsync(p->h_rho, rho_host, b, cudaMemcpyHostToDevice, st));
        if ((rc = run_solve(p, p->h_rho, p->h_phi, st))) return rc;
        IDP_CK(cudaMemcpyAsync(phi_host, p->h_phi, b, cudaMemcpyDeviceToHost, st));
    }
    IDP_CK(cudaStreamSynchronize(st));
    return IDP_OK;
}

int idp_solve_batched(int count, const idp_plan plans[], const double *const rho[], double *const phi[],
                      void *stream)
{
    if (count < 0 || (count > 0 && (!plans || !rho || !phi))) return IDP_EINVAL;
    for (int i = 0; i < count; ++i) {
        if (!plans[i] || !rho[i] || !phi[i]) return IDP_EINVAL;
        for (int j = 0; j < i; ++j)
            if (plans[j] == plans[i]) return IDP_EINVAL;
    }
    // the problems run concurrently (branches of one graph): an output may
    // overlap no input and no other output, of its own problem or another
    for (int i = 0; i < count; ++i) {
        const size_t bi = sizeof(double) * plans[i]->unodes;
        for (int j = 0; j < count; ++j) {
            const size_t bj = sizeof(double) * plans[j]->unodes;
            if (overlap(phi[i], bi, rho[j], bj)) return IDP_EALIAS;
            if (j != i && overlap(phi[i], bi, phi[j], bj)) return IDP_EALIAS;
        }
    }
    if (count == 0) return IDP_OK;
    cudaStream_t st = (cudaStream_t)stream;
    idp_plan p0 = plans[0];
    bool graphs = true;
    for (int i = 0; i < count; ++i)
        graphs = graphs && plans[i]->use_graph && !plans[i]->nvtx && plans[i]->dev == p0->dev;
    if (!graphs) {
        for (int i = 0; i < count; ++i) {
            int rc = run_solve(plans[i], rho[i], phi[i], st);
            if (rc) return rc;
        }
        return IDP_OK;
    }
    // one CUDA graph: a branch per problem (each with its own two streams), all
    // forked from and joined into the launch stream, so that independent
    // problems of different sizes run concurrently
    BatchCache *bc = p0->batch;
    bool hit = bc && (int)bc->serials.size() == count;
    for (int i = 0; hit && i < count; ++i)
        hit = bc->serials[i] == (plans[i]->serial << 16 ^ plans[i]->version) && bc->rho[i] == rho[i] &&
              bc->phi[i] == phi[i];
    if (!hit) {
        if (!bc) bc = p0->batch = new BatchCache();
        if (bc->exec) {
            cudaGraphExecDestroy(bc->exec);
            bc->exec = nullptr;
        }
        if (!bc->fork) IDP_CK(cudaEventCreateWithFlags(&bc->fork, cudaEventDisableTiming));
        while ((int)bc->joins.size() < count) {
            cudaEvent_t e;
            IDP_CK(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
            bc->joins.push_back(e);
        }
        cudaStream_t origin = p0->cap;
        IDP_CK(cudaStreamBeginCapture(origin, cudaStreamCaptureModeThreadLocal));
        int rc = IDP_OK;
        cudaError_t e = cudaEventRecord(bc->fork, origin);
        for (int i = 0; i < count && !rc && e == cudaSuccess; ++i) {
            idp_plan q = plans[i];
            e = cudaStreamWaitEvent(q->bst, bc->fork, 0);
            if (e != cudaSuccess) break;
            q->launches = 0;
            rc = enqueue(q, rho[i], phi[i], 0, q->bst);
            if (!rc) e = cudaEventRecord(bc->joins[i], q->bst);
            if (!rc && e == cudaSuccess) e = cudaStreamWaitEvent(origin, bc->joins[i], 0);
        }
        cudaGraph_t g = nullptr;
        cudaError_t e2 = cudaStreamEndCapture(origin, &g);
        if (rc || e != cudaSuccess || e2 != cudaSuccess) {
            if (g) cudaGraphDestroy(g);
            if (rc) return rc;
            return cuda_fail(e != cudaSuccess ? e : e2, "batched capture");
        }
        e = cudaGraphInstantiate(&bc->exec, g, 0);
        cudaGraphDestroy(g);
        if (e != cudaSuccess) return cuda_fail(e, "cudaGraphInstantiate");
        bc->serials.assign(count, 0);
        bc->rho.assign(rho, rho + count);
        bc->phi.assign(phi, phi + count);
        for (int i = 0; i < count; ++i) bc->serials[i] = plans[i]->serial << 16 ^ plans[i]->version;
    }
    for (int i = 0; i < count; ++i) {
        plans[i]->last = st;
        plans[i]->last_valid = 1;
    }
    IDP_CK(cudaGraphLaunch(bc->exec, st));
    return IDP_OK;
}

int idp_solve_stage(idp_plan p, int stage, const double *rho, double *out, void *stream)
{
    if (!p || !rho || !out) return IDP_EINVAL;
    if (stage < IDP_STAGE_BOUNDARY || stage > IDP_STAGE_PHI) return IDP_EINVAL;
    if (stage == IDP_STAGE_R && p->order != 6) return IDP_EINVAL;
    const size_t b = sizeof(double) * p->unodes;
    if (overlap(rho, b, out, b)) return IDP_EALIAS;
    p->last = (cudaStream_t)stream;
    p->last_valid = 1;
    return enqueue(p, rho, out, stage == IDP_STAGE_PHI ? 0 : stage, (cudaStream_t)stream);
}

int idp_plan_status(idp_plan p)
{
    if (!p) return IDP_EINVAL;
    if (p->last_valid) IDP_CK(cudaStreamSynchronize(p->last));
    IDP_CK(cudaGetLastError());
    if (p->d_val) {
        int v = 0;
        IDP_CK(cudaMemcpy(&v, p->d_val, sizeof(int), cudaMemcpyDeviceToHost));
        if (v) {
            IDP_CK(cudaMemset(p->d_val, 0, sizeof(int)));   // reported once
            return (v & 1) ? IDP_EINVAL : IDP_ESUPPORT;
        }
    }
    if (p->d_err) {
        int e = 0;
        IDP_CK(cudaMemcpy(&e, p->d_err, sizeof(int), cudaMemcpyDeviceToHost));
        if (e) {
            IDP_CK(cudaMemset(p->d_err, 0, sizeof(int)));   // reported once
            return IDP_ETIMEOUT;
        }
    }
    return IDP_OK;
}

int idp_profile_solve(idp_plan p, const double *rho, double *phi, void *stream, int capacity, int *kinds,
                      float *ms)
{
    if (!p || !rho || !phi || capacity < 0 || (capacity > 0 && (!kinds || !ms))) return IDP_EINVAL;
    const size_t b = sizeof(double) * p->unodes;
    if (overlap(rho, b, phi, b)) return IDP_EALIAS;
    cudaStream_t st = (cudaStream_t)stream;
    while ((int)p->ev.size() < 2 * capacity) {
        cudaEvent_t e;
        IDP_CK(cudaEventCreate(&e));
        p->ev.push_back(e);
    }
    p->profiling = 1;
    p->ev_used = 0;
    p->ev_kind.clear();
    p->launches = 0;
    p->last = st;
    p->last_valid = 1;
    const int rc = enqueue(p, rho, phi, 0, st);
    p->profiling = 0;
    if (rc) return rc;
    IDP_CK(cudaStreamSynchronize(st));
    const int n = (int)p->ev_kind.size();
    for (int i = 0; i < n; ++i) {
        kinds[i] = p->ev_kind[i];
        IDP_CK(cudaEventElapsedTime(&ms[i], p->ev[2 * i], p->ev[2 * i + 1]));
    }
    return n;
}

int idp_plan_check_guards(idp_plan p)
{
    if (!p) return IDP_EINVAL;
    IDP_CK(cudaDeviceSynchronize());
    std::vector<unsigned char> h(idp_plan_s::GUARD);
    for (const auto &g : p->guarded) {
        for (int side = 0; side < 2; ++side) {
            const char *src = side ? g.first + idp_plan_s::GUARD + g.second : g.first;
            IDP_CK(cudaMemcpy(h.data(), src, idp_plan_s::GUARD, cudaMemcpyDeviceToHost));
            for (unsigned char v : h)
                if (v != idp_plan_s::GUARD_BYTE) return IDP_EGUARD;
        }
    }
    return IDP_OK;
}

int idp_plan_grid(idp_plan p, int64_t n_solved[], int64_t offset[])
{
    if (!p || !n_solved || !offset) return IDP_EINVAL;
    const int o = 3 - p->d;
    for (int s = 0; s < p->d; ++s) {
        n_solved[s] = p->n[s + o];
        offset[s] = p->uoff[s + o];
    }
    return IDP_OK;
}

int idp_plan_info(idp_plan p, int64_t *nodes, int64_t *interior, int64_t *workspace_bytes)
{
    if (!p) return IDP_EINVAL;
    if (nodes) *nodes = p->unodes;
    if (interior) *interior = p->nint;
    if (workspace_bytes) *workspace_bytes = p->bytes;
    return IDP_OK;
}

int idp_destroy_plan(idp_plan p)
{
    if (!p) return IDP_EINVAL;
    cudaDeviceSynchronize();
    if (p->gexec) cudaGraphExecDestroy(p->gexec);
    if (p->hexec) cudaGraphExecDestroy(p->hexec);
    if (p->cap) cudaStreamDestroy(p->cap);
    if (p->side) cudaStreamDestroy(p->side);
    if (p->bst) cudaStreamDestroy(p->bst);
    if (p->batch) {
        if (p->batch->exec) cudaGraphExecDestroy(p->batch->exec);
        for (cudaEvent_t e : p->batch->joins) cudaEventDestroy(e);
        if (p->batch->fork) cudaEventDestroy(p->batch->fork);
        delete p->batch;
    }
    if (p->fork) cudaEventDestroy(p->fork);
    if (p->join) cudaEventDestroy(p->join);
    for (int i = 0; i < 2; ++i)
        if (p->fst[i]) cudaStreamDestroy(p->fst[i]);
    for (int i = 0; i < 3; ++i)
        if (p->fev[i]) cudaEventDestroy(p->fev[i]);
    for (cudaEvent_t e : p->ev) cudaEventDestroy(e);
    for (void *q : p->allocs) cudaFree(q);
    delete p;
    return IDP_OK;
}

const char *idp_strerror(int code)
{
    switch (code) {
    case IDP_OK: return "ok";
    case IDP_EINVAL: return "invalid argument";
    case IDP_ENOMEM: return "out of memory";
    case IDP_ECUDA: return "CUDA error";
    case IDP_EALIAS: return "input and output overlap";
    case IDP_ESUPPORT: return "size or option not supported (panel counts must be 2^a in [16, 512] or 3*2^a in [48, 384])";
    case IDP_ETIMEOUT: return "a device-side wait exceeded its iteration limit";
    case IDP_EGUARD: return "a guard region around a workspace buffer was overwritten";
    case IDP_ESCRATCH: return "problem larger than the fixed scratch of idp_rhs6_noalloc (524288 nodes)";
    default: return "unknown error";
    }
}

const char *idp_last_cuda_error(void) { return g_cuda_err; }

int idp_plan_tuning(idp_plan p, int64_t out[9])
{
    if (!p || !out) return IDP_EINVAL;
    out[0] = p->tuned;
    out[1] = p->mixed_path;
    for (int a = 0; a < 3; ++a) {
        out[2 + a] = p->nchunk[a];
        out[5 + a] = p->pchunk[a];
    }
    out[8] = p->dst_lines;
    return IDP_OK;
}

int idp_plan_launches(idp_plan p, int64_t *launches)
{
    if (!p || !launches) return IDP_EINVAL;
    *launches = p->launches;
    return IDP_OK;
}

}  // extern "C"
