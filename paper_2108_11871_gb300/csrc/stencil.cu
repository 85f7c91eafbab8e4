// Grid-function kernels of the harmonic correction (section 5) and the
// eigenvalue tables of the two spectral solves (sections 3 and 5).
//
// Node arrays are n0 x n1 x n2 (C order); 2-D grids use n0 = 1 and the
// axes 1, 2.  Interior arrays are dense over the interior nodes.
#include "dd.cuh"
#include "idp_internal.cuh"

namespace idp {

namespace {

struct Geo {
    int act[3];          // 1 if the axis is active
    int n[3], M[3], ni[3];
    int64_t ns[3], is[3];
    double h[3];
};

__device__ __forceinline__ Geo make_geo(const Grid3 &g)
{
    Geo o;
    o.n[0] = g.n0; o.n[1] = g.n1; o.n[2] = g.n2;
    o.h[0] = g.h0; o.h[1] = g.h1; o.h[2] = g.h2;
    for (int s = 0; s < 3; ++s) {
        o.act[s] = (g.d == 3) || (s > 0);
        o.M[s] = o.n[s] - 1;
        o.ni[s] = o.act[s] ? o.n[s] - 2 : 1;
    }
    o.ns[2] = 1; o.ns[1] = o.n[2]; o.ns[0] = (int64_t)o.n[1] * o.n[2];
    o.is[2] = 1; o.is[1] = o.ni[2]; o.is[0] = (int64_t)o.ni[1] * o.ni[2];
    return o;
}

__device__ __forceinline__ bool on_boundary(const Geo &g, const int j[3])
{
    for (int s = 0; s < 3; ++s)
        if (g.act[s] && (j[s] == 0 || j[s] == g.M[s])) return true;
    return false;
}

// distance of node index j_s from the nearer face of axis s (large for an inactive axis)
__device__ __forceinline__ int face_dist(const Geo &g, int s, int js)
{
    return g.act[s] ? min(js, g.M[s] - js) : (1 << 20);
}

// gtilde = -L4(ghat) at interior node i, ghat = U on boundary nodes and 0 inside
// (eq. harmonic4thOrderNH2D).  L4 weights (host-computed in c): face +-e_s:
// 1/h_s^2 - 2 sum_r c_sr/(h_s^2 h_r^2); edge +-e_s +-e_r: c_sr/(h_s^2 h_r^2),
// c_sr = (h_s^2 + h_r^2)/12.
__device__ __forceinline__ double gtilde_at(const Geo &g, const StencilCoef &c, const double *__restrict__ U,
                                            const int i[3])
{
    double acc = 0.0;
    for (int d0 = -1; d0 <= 1; ++d0) {
        if (d0 != 0 && !g.act[0]) continue;
        for (int d1 = -1; d1 <= 1; ++d1)
            for (int d2 = -1; d2 <= 1; ++d2) {
                const int nz = (d0 != 0) + (d1 != 0) + (d2 != 0);
                if (nz == 0 || nz == 3) continue;
                const int j[3] = {i[0] + d0, i[1] + d1, i[2] + d2};
                if (!on_boundary(g, j)) continue;
                double wgt;
                if (nz == 1) wgt = c.wf[d0 != 0 ? 0 : (d1 != 0 ? 1 : 2)];
                else wgt = c.we[d0 != 0 ? 0 : 1][d2 != 0 ? 2 : 1];
                acc = fma(wgt, U[j[0] * g.ns[0] + j[1] * g.ns[1] + j[2] * g.ns[2]], acc);
            }
    }
    return -acc;
}

// gtilde on the layers next to the boundary, as planes (3-D) or lines (2-D).
// The shell is split by the first axis s whose index is 0 or n_s-1:
//   Q0[side][i1][i2]  (3-D only)      nodes i0 = side ? n0-1 : 0
//   Q1[side][i0][i2]                  i1 = side ? n1-1 : 0, i0 not on the i0 layers
//   Q2[side][i0][i1]                  i2 = side ? n2-1 : 0, i0, i1 not on their layers
// (2-D: axis 0 is inactive, Q1[side][i2] and Q2[side][i1]).  Entries outside a
// part are zero.  Interior indices i_s = node index - 1.
__global__ void gtilde_planes_kernel(const Grid3 gg, const StencilCoef c, const double *__restrict__ U,
                                     double *__restrict__ Q0, double *__restrict__ Q1, double *__restrict__ Q2)
{
    const Geo g = make_geo(gg);
    const int n0 = g.ni[0], n1 = g.ni[1], n2 = g.ni[2];
    const int s0 = g.act[0] ? 2 * n1 * n2 : 0, s1 = 2 * n0 * n2, s2 = 2 * n0 * n1;
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < s0 + s1 + s2; t += gridDim.x * blockDim.x) {
        int part, side, a, b;
        double *dst;
        if (t < s0) {
            part = 0; const int q = t; side = q / (n1 * n2); const int r = q - side * n1 * n2;
            a = r / n2; b = r - a * n2; dst = Q0 + q;
        } else if (t < s0 + s1) {
            part = 1; const int q = t - s0; side = q / (n0 * n2); const int r = q - side * n0 * n2;
            a = r / n2; b = r - a * n2; dst = Q1 + q;
        } else {
            part = 2; const int q = t - s0 - s1; side = q / (n0 * n1); const int r = q - side * n0 * n1;
            a = r / n1; b = r - a * n1; dst = Q2 + q;
        }
        int k[3];   // interior indices
        if (part == 0) { k[0] = side ? n0 - 1 : 0; k[1] = a; k[2] = b; }
        else if (part == 1) { k[0] = a; k[1] = side ? n1 - 1 : 0; k[2] = b; }
        else { k[0] = a; k[1] = b; k[2] = side ? n2 - 1 : 0; }
        bool keep = true;
        if (part >= 1 && g.act[0] && (k[0] == 0 || k[0] == n0 - 1)) keep = false;
        if (part == 2 && (k[1] == 0 || k[1] == n1 - 1)) keep = false;
        double v = 0.0;
        if (keep) {
            const int i[3] = {g.act[0] ? k[0] + 1 : 0, k[1] + 1, k[2] + 1};
            v = gtilde_at(g, c, U, i);
        }
        *dst = v;
    }
}

// Forward sine transform of gtilde from the transformed, combined parts
// (4^{d-1} S of each part, then (a + b, a - b) per pair of faces):
//   val(k) = sum_s sin4_s(k_s) Qs[k_s odd](k_other),  sin4_s(k) = 4 sin(pi (k+1)/M_s).
// out = tab * val (+ add); if out2: out2 = (tab2 (- tab unless fold)) * val + add2.
__global__ void gtilde_expand_kernel(const Grid3 gg, const double *__restrict__ Q0, const double *__restrict__ Q1,
                                     const double *__restrict__ Q2, const double *__restrict__ sin4,
                                     const double *__restrict__ tab, const double *add, double *out,
                                     const double *__restrict__ tab2, const double *__restrict__ add2,
                                     double *__restrict__ out2, int fold, const double *__restrict__ ascale)
{
    const Geo g = make_geo(gg);
    const int k2 = blockIdx.x * blockDim.x + threadIdx.x;
    const int k1 = blockIdx.y * blockDim.y + threadIdx.y;
    const int k0 = blockIdx.z;
    if (k2 >= g.ni[2] || k1 >= g.ni[1]) return;
    const int n0 = g.ni[0], n1 = g.ni[1], n2 = g.ni[2];
    const double *sn0 = sin4, *sn1 = sin4 + (g.act[0] ? n0 : 0), *sn2 = sn1 + n1;
    double v = sn1[k1] * Q1[(int64_t)((k1 & 1) ? n0 + k0 : k0) * n2 + k2];
    v = fma(sn2[k2], Q2[(int64_t)((k2 & 1) ? n0 + k0 : k0) * n1 + k1], v);
    if (g.act[0]) v = fma(sn0[k0], Q0[(int64_t)((k0 & 1) ? n1 + k1 : k1) * n2 + k2], v);
    const int64_t t = k0 * g.is[0] + (int64_t)k1 * g.is[1] + k2;
    const double tb = tab[t];
    // ascale (optional): the addends still need their eigenvalue factor (the
    // tensor-core transform of rho leaves it to this kernel)
    const double sc = ascale ? ascale[t] : 1.0;
    out[t] = add ? fma(tb, v, ascale ? sc * add[t] : add[t]) : tb * v;
    // tab2 holds tabR + tab4 (u1 folded in); without fold, tabR = tab2 - tab4
    if (out2) out2[t] = fma(fold ? tab2[t] : tab2[t] - tb, v, ascale ? sc * add2[t] : add2[t]);
}

// gtilde as a dense interior array from its parts (for the stage output).
__global__ void gtilde_scatter_kernel(const Grid3 gg, const double *__restrict__ Q0, const double *__restrict__ Q1,
                                      const double *__restrict__ Q2, double *__restrict__ out)
{
    const Geo g = make_geo(gg);
    const int k2 = blockIdx.x * blockDim.x + threadIdx.x;
    const int k1 = blockIdx.y * blockDim.y + threadIdx.y;
    const int k0 = blockIdx.z;
    if (k2 >= g.ni[2] || k1 >= g.ni[1]) return;
    const int n0 = g.ni[0], n1 = g.ni[1], n2 = g.ni[2];
    double v = 0.0;
    if (g.act[0] && (k0 == 0 || k0 == n0 - 1)) v = Q0[((int64_t)(k0 ? 1 : 0) * n1 + k1) * n2 + k2];
    else if (k1 == 0 || k1 == n1 - 1) v = Q1[((int64_t)(k1 ? 1 : 0) * n0 + k0) * n2 + k2];
    else if (k2 == 0 || k2 == n2 - 1) v = Q2[((int64_t)(k2 ? 1 : 0) * n0 + k0) * n1 + k1];
    out[k0 * g.is[0] + (int64_t)k1 * g.is[1] + k2] = v;
}

// W_s(j) = sum_{r != s} a_sr (U(j+e_r) + U(j-e_r) - 2 U(j)),
// a_sr = (h_s^4/240 + h_s^2 h_r^2/144) / (h_s^4 h_r^2) (host-computed), at nodes
// with 1 <= j_r <= M_r-1 for r != s.  Then R = sum_s [1 -4 6 -4 1]_s W_s is the
// right-hand side of eqs. 6thOrderRelation2D/3D, the sum over ordered pairs
// of c_sr D2_s D2_s D2_r u.
// odd = 1: u is taken as zero on the boundary nodes (the sine series of the
// interior values, continued oddly).
__device__ __forceinline__ void w_node(const Geo &g, const StencilCoef &c, const double *__restrict__ U,
                                       double *__restrict__ W, const int j[3], bool odd)
{
    const int64_t nodes = (int64_t)g.n[0] * g.n[1] * g.n[2];
    const int64_t t = j[0] * g.ns[0] + (int64_t)j[1] * g.ns[1] + j[2];
    // odd: a node on a face reads as zero; the neighbours along r of a node off
    // the faces lie on a face only through index r
    const bool bnd = odd && on_boundary(g, j);
    const double u0 = bnd ? 0.0 : U[t];
    double e[3];
    bool inner[3];
#pragma unroll
    for (int r = 0; r < 3; ++r) {
        inner[r] = !g.act[r] || (j[r] >= 1 && j[r] <= g.M[r] - 1);
        e[r] = 0.0;
        if (g.act[r] && inner[r] && !bnd) {
            const double up = (odd && j[r] + 1 == g.M[r]) ? 0.0 : U[t + g.ns[r]];
            const double um = (odd && j[r] - 1 == 0) ? 0.0 : U[t - g.ns[r]];
            e[r] = fma(-2.0, u0, up + um);
        }
    }
#pragma unroll
    for (int s = 0; s < 3; ++s) {
        if (!g.act[s]) continue;
        bool ok = true;
#pragma unroll
        for (int r = 0; r < 3; ++r)
            if (r != s && !inner[r]) ok = false;
        if (!ok) continue;
        double w = 0.0;
#pragma unroll
        for (int r = 0; r < 3; ++r)
            if (r != s && g.act[r]) w = fma(c.a[s][r], e[r], w);
        W[(int64_t)s * nodes + t] = w;
    }
}

// all nodes; grid: x = node index 2, y = index 1, z = index 0
__global__ void rhs6_w_kernel(const Grid3 gg, const StencilCoef c, const double *__restrict__ U,
                              double *__restrict__ W)
{
    const Geo g = make_geo(gg);
    const int j2 = blockIdx.x * blockDim.x + threadIdx.x;
    const int j1 = blockIdx.y * blockDim.y + threadIdx.y;
    const int j0 = blockIdx.z;
    if (j2 >= g.n[2] || j1 >= g.n[1]) return;
    const int j[3] = {j0, j1, j2};
    w_node(g, c, U, W, j, false);
}

// The nodes of a box (node indices lo_s .. lo_s + ext_s - 1 on the active axes)
// that lie within tau - 1 of its faces, enumerated as the slabs of axis 0, then
// those of axis 1 between them, then those of axis 2 (axis 2 fastest in each).
// Requires ext_s >= 2 tau on the active axes.
struct Shell {
    int lo[3], ext[3], tau, act0;
    int64_t c0, c1, count;
};

inline Shell make_shell(const Grid3 &g, int lo, int shrink, int tau)
{
    Shell sh{};
    const int n[3] = {g.n0, g.n1, g.n2};
    sh.act0 = g.d == 3;
    for (int s = 0; s < 3; ++s) {
        const bool act = s > 0 || sh.act0;
        sh.lo[s] = act ? lo : 0;
        sh.ext[s] = act ? n[s] - shrink : 1;
    }
    sh.tau = tau;
    const int m0 = sh.act0 ? sh.ext[0] - 2 * tau : 1;
    sh.c0 = sh.act0 ? 2 * (int64_t)tau * sh.ext[1] * sh.ext[2] : 0;
    sh.c1 = (int64_t)m0 * 2 * tau * sh.ext[2];
    sh.count = sh.c0 + sh.c1 + (int64_t)m0 * (sh.ext[1] - 2 * tau) * 2 * tau;
    return sh;
}

__device__ __forceinline__ void shell_node(const Shell &sh, int t, int j[3])
{
    // 32-bit index arithmetic: a shell has at most 513^3 < 2^31 nodes (M_s <= 512)
    const int tau = sh.tau, e0 = sh.ext[0], e1 = sh.ext[1], e2 = sh.ext[2];
    const int c0 = (int)sh.c0, c1 = (int)sh.c1;
    if (t < c0) {
        const int pl = e1 * e2;
        const int q = t / pl, r = t - q * pl;
        j[0] = sh.lo[0] + (q < tau ? q : e0 - 2 * tau + q);
        j[1] = sh.lo[1] + r / e2;
        j[2] = sh.lo[2] + r % e2;
        return;
    }
    t -= c0;
    const int l0 = sh.act0 ? sh.lo[0] + tau : sh.lo[0];
    if (t < c1) {
        const int pl = 2 * tau * e2;
        const int q = t / pl, r = t - q * pl;
        const int a = r / e2;
        j[0] = l0 + q;
        j[1] = sh.lo[1] + (a < tau ? a : e1 - 2 * tau + a);
        j[2] = sh.lo[2] + r - a * e2;
        return;
    }
    t -= c1;
    const int pl = (e1 - 2 * tau) * 2 * tau;
    const int q = t / pl, r = t - q * pl;
    const int a = r / (2 * tau), bb = r - a * 2 * tau;
    j[0] = l0 + q;
    j[1] = sh.lo[1] + tau + a;
    j[2] = sh.lo[2] + (bb < tau ? bb : e2 - 2 * tau + bb);
}

// W of the odd continuation on the nodes of a shell
__global__ void rhs6_wband_kernel(const Grid3 gg, const Shell sh, const StencilCoef c,
                                  const double *__restrict__ U, double *__restrict__ W)
{
    const Geo g = make_geo(gg);
    const int cnt = (int)sh.count;
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < cnt; t += gridDim.x * blockDim.x) {
        int j[3];
        shell_node(sh, t, j);
        w_node(g, c, U, W, j, true);
    }
}

// R on the core nodes (all active indices in 2..M-2) into the dense interior array.
__global__ void rhs6_core_kernel(const Grid3 gg, const double *__restrict__ W, double *__restrict__ R)
{
    const Geo g = make_geo(gg);
    const int k2 = blockIdx.x * blockDim.x + threadIdx.x;
    const int k1 = blockIdx.y * blockDim.y + threadIdx.y;
    const int k0 = blockIdx.z;
    if (k2 >= g.ni[2] || k1 >= g.ni[1]) return;
    const int i[3] = {g.act[0] ? k0 + 1 : 0, k1 + 1, k2 + 1};
    for (int s = 0; s < 3; ++s)
        if (g.act[s] && (i[s] < 2 || i[s] > g.M[s] - 2)) return;
    const int64_t nodes = (int64_t)g.n[0] * g.n[1] * g.n[2];
    const int64_t node = i[0] * g.ns[0] + (int64_t)i[1] * g.ns[1] + i[2];
    double acc = 0.0;
    for (int s = 0; s < 3; ++s) {
        if (!g.act[s]) continue;
        const double *w = W + (int64_t)s * nodes + node;
        const int64_t st = g.ns[s];
        const double outer = w[-2 * st] + w[2 * st];
        const double inner = w[-st] + w[st];
        acc += fma(6.0, w[0], fma(-4.0, inner, outer));
    }
    R[k0 * g.is[0] + (int64_t)k1 * g.is[1] + k2] = acc;
}

// Cubic extrapolation to the layers next to the boundary (section 5): along
// each axis the value at layer 1 is 4R_2 - 6R_3 + 4R_4 - R_5 (mirrored at
// layer M-1); applied as the tensor product over the axes.
__global__ void rhs6_extrap_kernel(const Grid3 gg, double *R)
{
    // one thread per node of the layers next to the boundary (the shell of the
    // interior box), enumerated like the gtilde parts: the slabs of axis 0, then
    // those of axis 1 inside them, then those of axis 2
    const Geo g = make_geo(gg);
    const int n0 = g.ni[0], n1 = g.ni[1], n2 = g.ni[2];
    const int s0 = g.act[0] ? 2 * n1 * n2 : 0;
    const int s1 = 2 * (g.act[0] ? n0 - 2 : 1) * n2;
    const int s2 = 2 * (g.act[0] ? n0 - 2 : 1) * (n1 - 2);
    const double wts[4] = {4.0, -6.0, 4.0, -1.0};
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < s0 + s1 + s2; t += gridDim.x * blockDim.x) {
        int k[3];   // interior indices
        if (t < s0) {
            const int side = t / (n1 * n2), r = t - side * n1 * n2;
            k[0] = side ? n0 - 1 : 0; k[1] = r / n2; k[2] = r - k[1] * n2;
        } else if (t < s0 + s1) {
            const int q = t - s0, m0 = g.act[0] ? n0 - 2 : 1;
            const int side = q / (m0 * n2), r = q - side * m0 * n2;
            k[0] = g.act[0] ? r / n2 + 1 : 0; k[1] = side ? n1 - 1 : 0; k[2] = r % n2;
        } else {
            const int q = t - s0 - s1, m0 = g.act[0] ? n0 - 2 : 1;
            const int side = q / (m0 * (n1 - 2)), r = q - side * m0 * (n1 - 2);
            k[0] = g.act[0] ? r / (n1 - 2) + 1 : 0; k[1] = r % (n1 - 2) + 1; k[2] = side ? n2 - 1 : 0;
        }
        const int i[3] = {g.act[0] ? k[0] + 1 : 0, k[1] + 1, k[2] + 1};
        // per axis: first tap index (interior coordinate), step and count
        int first[3], step[3], ntap[3];
        for (int s = 0; s < 3; ++s) {
            if (g.act[s] && i[s] == 1) { first[s] = 1; step[s] = 1; ntap[s] = 4; }
            else if (g.act[s] && i[s] == g.M[s] - 1) { first[s] = g.M[s] - 3; step[s] = -1; ntap[s] = 4; }
            else { first[s] = k[s]; step[s] = 0; ntap[s] = 1; }
        }
        double acc = 0.0;
        for (int q0 = 0; q0 < ntap[0]; ++q0) {
            const double w0 = ntap[0] == 4 ? wts[q0] : 1.0;
            const int64_t c0 = (first[0] + q0 * step[0]) * g.is[0];
            for (int q1 = 0; q1 < ntap[1]; ++q1) {
                const double w1 = ntap[1] == 4 ? wts[q1] : 1.0;
                const int64_t c1 = c0 + (int64_t)(first[1] + q1 * step[1]) * g.is[1];
                for (int q2 = 0; q2 < ntap[2]; ++q2) {
                    const double w2 = ntap[2] == 4 ? wts[q2] : 1.0;
                    acc = fma(w0 * w1 * w2, R[c1 + first[2] + q2 * step[2]], acc);
                }
            }
        }
        R[k[0] * g.is[0] + (int64_t)k[1] * g.is[1] + k[2]] = acc;
    }
}

// ---------------------------------------------------------------------------
// The 6th-order right-hand side in spectral form (section 5).
//
// Inside the grid u1 equals its sine series, so on the nodes whose stencil stays
// off the faces R is R_spec = S(Lambda_R b) with b the sine coefficients of u1
// and Lambda_R(k) = sum_{s != r} c_sr lam_s(k)^2 lam_r(k) the symbol of the
// stencil (lam_s the eigenvalues of D2_s).  R_spec is the same stencil applied
// to the odd continuation of the interior values of u1 (zero on the faces).
// The difference E = R - R_spec lives on the nodes within 2 of a face:
//   * distance 2 (and no axis at distance 1): the stencil's only tap on a face
//     is [1 -4 6 -4 1]_s at offset -+2, so E = sum over those s of W_s at the
//     face node, W_s from the boundary values g (the second differences of g
//     along the face);
//   * distance 1: R is the cubic extrapolation of the core values, so
//     E = R_extrap - R_spec there.
// So S R = Lambda_R (S S b) + S E, and the sine transform of E is assembled
// from the (d-1)-dimensional transforms of its layers.

// x with its sign flipped when neg (an integer operation: FP64 issue is scarce)
__device__ __forceinline__ double flip_if(double x, bool neg)
{
    return __longlong_as_double(__double_as_longlong(x) ^ ((long long)neg << 63));
}

// W of the odd continuation (band array `W`, odd = 1) at node j shifted by o
// along s: reflected (with a sign change) through the faces of axis s.
__device__ __forceinline__ double w_odd_at(const Geo &g, const double *__restrict__ W, int64_t nodes, int s,
                                           const int j[3], int o)
{
    int q = j[s] + o;
    bool neg = false;
    if (q < 0) { q = -q; neg = true; }
    else if (q > g.M[s]) { q = 2 * g.M[s] - q; neg = true; }
    int jj[3] = {j[0], j[1], j[2]};
    jj[s] = q;
    return flip_if(W[(int64_t)s * nodes + jj[0] * g.ns[0] + (int64_t)jj[1] * g.ns[1] + jj[2]], neg);
}

// W_s at the face node of axis s nearest to j (j at distance 2 from it), from
// the boundary values in U
__device__ __forceinline__ double w_face(const Geo &g, const StencilCoef &c, const double *__restrict__ U, int s,
                                         const int j[3])
{
    int f[3] = {j[0], j[1], j[2]};
    f[s] = j[s] <= g.M[s] / 2 ? 0 : g.M[s];
    const int64_t t = f[0] * g.ns[0] + (int64_t)f[1] * g.ns[1] + f[2];
    const double u0 = U[t];
    double w = 0.0;
    for (int r = 0; r < 3; ++r)
        if (r != s && g.act[r]) w = fma(c.a[s][r], fma(-2.0, u0, U[t + g.ns[r]] + U[t - g.ns[r]]), w);
    return w;
}

// [1 -4 6 -4 1] applied to (w(-2), w(-1), w(0), w(1), w(2)): 2 additions, 2 FMAs
__device__ __forceinline__ double d4(double wm2, double wm1, double w0, double wp1, double wp2)
{
    return fma(6.0, w0, fma(-4.0, wm1 + wp1, wm2 + wp2));
}

// R_spec at node j (any interior node) from the band array of W of the odd continuation
__device__ __forceinline__ double r_spec_at(const Geo &g, const double *__restrict__ W, int64_t nodes,
                                            const int j[3])
{
    double acc = 0.0;
#pragma unroll
    for (int s = 0; s < 3; ++s) {
        if (!g.act[s]) continue;
        acc += d4(w_odd_at(g, W, nodes, s, j, -2), w_odd_at(g, W, nodes, s, j, -1), w_odd_at(g, W, nodes, s, j, 0),
                  w_odd_at(g, W, nodes, s, j, 1), w_odd_at(g, W, nodes, s, j, 2));
    }
    return acc;
}

// The same at a node whose stencil stays inside the grid along every axis
// (all active distances >= 2): no reflections
__device__ __forceinline__ double r_spec_inside(const Geo &g, const double *__restrict__ W, int64_t nodes,
                                                const int j[3])
{
    const int64_t t = j[0] * g.ns[0] + (int64_t)j[1] * g.ns[1] + j[2];
    double acc = 0.0;
#pragma unroll
    for (int s = 0; s < 3; ++s) {
        if (!g.act[s]) continue;
        const double *w = W + (int64_t)s * nodes + t;
        const int64_t st = g.ns[s];
        acc += d4(w[-2 * st], w[-st], w[0], w[st], w[2 * st]);
    }
    return acc;
}

// R (with the boundary values) at core node j (all active distances >= 2)
__device__ __forceinline__ double r_core_at(const Geo &g, const StencilCoef &c, const double *__restrict__ U,
                                            const double *__restrict__ W, int64_t nodes, const int j[3])
{
    double acc = r_spec_inside(g, W, nodes, j);
#pragma unroll
    for (int s = 0; s < 3; ++s)
        if (face_dist(g, s, j[s]) == 2) acc += w_face(g, c, U, s, j);
    return acc;
}

// R on the core nodes within 5 of a face (the taps of the cubic extrapolation),
// enumerated as a shell; written to the dense interior array Rt.
__global__ void rhs6_taps_kernel(const Grid3 gg, const Shell sh, const StencilCoef c,
                                 const double *__restrict__ U, const double *__restrict__ W, double *__restrict__ Rt)
{
    const Geo g = make_geo(gg);
    const int64_t nodes = (int64_t)g.n[0] * g.n[1] * g.n[2];
    const int cnt = (int)sh.count;
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < cnt; t += gridDim.x * blockDim.x) {
        int j[3];
        shell_node(sh, t, j);
        const int64_t k0 = g.act[0] ? j[0] - 1 : 0;
        Rt[k0 * g.is[0] + (int64_t)(j[1] - 1) * g.is[1] + (j[2] - 1)] = r_core_at(g, c, U, W, nodes, j);
    }
}

// weight q (0..3) of the cubic extrapolation from the taps at distance 2..5
__device__ __forceinline__ double extrap_w(int q) { return q == 0 ? 4.0 : q == 1 ? -6.0 : q == 2 ? 4.0 : -1.0; }

// E on the layers at distance 1 and 2 from the faces, split like the gtilde parts
// by the first axis s at distance <= 2:
//   Es[side][l][a][b], l = distance - 1, (a, b) the interior indices of the other
//   two axes in increasing order; entries that belong to a lower part are zero.
// E0 (3-D only) is followed by E1 and E2 in memory.
__global__ void rhs6_e_kernel(const Grid3 gg, const StencilCoef c, const double *__restrict__ U,
                              const double *__restrict__ W, const double *__restrict__ Rt, double *__restrict__ E0,
                              double *__restrict__ E1, double *__restrict__ E2)
{
    const Geo g = make_geo(gg);
    const int n0 = g.ni[0], n1 = g.ni[1], n2 = g.ni[2];
    // 32-bit index arithmetic: 4 (n1 n2 + n0 n2 + n0 n1) < 2^31 for n <= 511
    const int s0 = g.act[0] ? 4 * n1 * n2 : 0, s1 = 4 * n0 * n2, s2 = 4 * n0 * n1;
    const int64_t nodes = (int64_t)g.n[0] * g.n[1] * g.n[2];
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < s0 + s1 + s2; t += gridDim.x * blockDim.x) {
        int sl, a, b, j0, j1, j2;
        bool lower;
        double *dst;
        if (t < s0) {
            const int pl = n1 * n2;
            sl = t / pl; const int r = t - sl * pl;
            a = r / n2; b = r - a * n2; dst = E0 + t;
            const int l = sl & 1;
            j0 = (sl >> 1) ? g.M[0] - 1 - l : 1 + l; j1 = a + 1; j2 = b + 1;
            lower = false;
        } else if (t < s0 + s1) {
            const int q = t - s0, pl = n0 * n2;
            sl = q / pl; const int r = q - sl * pl;
            a = r / n2; b = r - a * n2; dst = E1 + q;
            const int l = sl & 1;
            j0 = g.act[0] ? a + 1 : 0; j1 = (sl >> 1) ? g.M[1] - 1 - l : 1 + l; j2 = b + 1;
            lower = face_dist(g, 0, j0) <= 2;
        } else {
            const int q = t - s0 - s1, pl = n0 * n1;
            sl = q / pl; const int r = q - sl * pl;
            a = r / n1; b = r - a * n1; dst = E2 + q;
            const int l = sl & 1;
            j0 = g.act[0] ? a + 1 : 0; j1 = b + 1; j2 = (sl >> 1) ? g.M[2] - 1 - l : 1 + l;
            lower = face_dist(g, 0, j0) <= 2 || face_dist(g, 1, j1) <= 2;
        }
        double v = 0.0;
        if (!lower) {
            const int j[3] = {j0, j1, j2};
            const int d0 = face_dist(g, 0, j0), d1 = face_dist(g, 1, j1), d2 = face_dist(g, 2, j2);
            if (d0 == 1 || d1 == 1 || d2 == 1) {
                // cubic extrapolation, the tensor product over the axes at distance 1
                // (taps at interior index 1..4 from the low face, M-3..M-6 from the high one)
                const int nt0 = d0 == 1 ? 4 : 1, nt1 = d1 == 1 ? 4 : 1, nt2 = d2 == 1 ? 4 : 1;
                const int f0 = d0 == 1 ? (j0 == 1 ? 1 : g.M[0] - 3) : j0 - (g.act[0] ? 1 : 0);
                const int f1 = d1 == 1 ? (j1 == 1 ? 1 : g.M[1] - 3) : j1 - 1;
                const int f2 = d2 == 1 ? (j2 == 1 ? 1 : g.M[2] - 3) : j2 - 1;
                const int st0 = j0 == 1 ? 1 : -1, st1 = j1 == 1 ? 1 : -1, st2 = j2 == 1 ? 1 : -1;
                double acc;
                if (nt0 + nt1 + nt2 == 6) {
                    // one axis: 4 (R_2 + R_4) - 6 R_3 - R_5 (2 FMAs, 1 addition)
                    const int64_t base = (int64_t)f0 * g.is[0] + (int64_t)f1 * g.is[1] + f2;
                    const int64_t step = nt0 == 4 ? st0 * g.is[0] : nt1 == 4 ? st1 * g.is[1] : st2;
                    acc = fma(4.0, Rt[base] + Rt[base + 2 * step], fma(-6.0, Rt[base + step], -Rt[base + 3 * step]));
                } else {
                    acc = 0.0;
                    for (int q0 = 0; q0 < nt0; ++q0) {
                        const double w0 = nt0 == 4 ? extrap_w(q0) : 1.0;
                        const int64_t c0 = (int64_t)(f0 + q0 * st0) * g.is[0];
                        for (int q1 = 0; q1 < nt1; ++q1) {
                            const double w1 = nt1 == 4 ? w0 * extrap_w(q1) : w0;
                            const int64_t c1 = c0 + (int64_t)(f1 + q1 * st1) * g.is[1];
                            for (int q2 = 0; q2 < nt2; ++q2) {
                                const double w2 = nt2 == 4 ? w1 * extrap_w(q2) : w1;
                                acc = fma(w2, Rt[c1 + f2 + q2 * st2], acc);
                            }
                        }
                    }
                }
                v = acc - r_spec_at(g, W, nodes, j);
            } else {
                if (d0 == 2) v += w_face(g, c, U, 0, j);
                if (d1 == 2) v += w_face(g, c, U, 1, j);
                if (d2 == 2) v += w_face(g, c, U, 2, j);
            }
        }
        *dst = v;
    }
}

// In place, per pair of layers at the two faces of an axis (layers a at offset l*pl,
// b at (nl + l)*pl of each part): (a, b) -> (a + b, a - b), the two sign patterns
// of sin(pi m j / M) and sin(pi m (M - j) / M) = (-1)^(m+1) sin(pi m j / M).
__global__ void layers_combine_kernel(double *__restrict__ P0, int pl0, double *__restrict__ P1, int pl1,
                                      double *__restrict__ P2, int pl2, int nl)
{
    // 32-bit index arithmetic: at most 2 * 3 * 511^2 entries
    const int tot = nl * (pl0 + pl1 + pl2);
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < tot; t += gridDim.x * blockDim.x) {
        double *P;
        int pl, q = t;
        if (q < nl * pl0) { P = P0; pl = pl0; }
        else if ((q -= nl * pl0) < nl * pl1) { P = P1; pl = pl1; }
        else { q -= nl * pl1; P = P2; pl = pl2; }
        const int l = q / pl;
        const int x = q - l * pl;
        const double av = P[l * pl + x], bv = P[(nl + l) * pl + x];
        P[l * pl + x] = av + bv;
        P[(nl + l) * pl + x] = av - bv;
    }
}

// out(k) += tab(k) * (4^d S E)(k) from the transformed, combined layers
// (4^{d-1} S of each, then (a + b, a - b) per pair):
//   sum_s sum_l 4 sin(pi (k_s+1)(l+1)/M_s) Es[k_s odd][l](k_other).
// sin4 / sin4b hold 4 sin(pi (k+1)/M_s) / 4 sin(2 pi (k+1)/M_s) per active axis.
__global__ void rhs6_e_expand_kernel(const Grid3 gg, const double *__restrict__ E0, const double *__restrict__ E1,
                                     const double *__restrict__ E2, const double *__restrict__ sin4,
                                     const double *__restrict__ sin4b, const double *__restrict__ tab,
                                     double *__restrict__ out)
{
    const Geo g = make_geo(gg);
    const int k2 = blockIdx.x * blockDim.x + threadIdx.x;
    const int k1 = blockIdx.y * blockDim.y + threadIdx.y;
    const int k0 = blockIdx.z;
    if (k2 >= g.ni[2] || k1 >= g.ni[1]) return;
    const int n0 = g.ni[0], n1 = g.ni[1], n2 = g.ni[2];
    const int o1 = g.act[0] ? n0 : 0, o2 = o1 + n1;
    double v;
    {
        const int64_t pl = (int64_t)n0 * n2, o = (int64_t)k0 * n2 + k2 + ((k1 & 1) ? 2 * pl : 0);
        v = sin4[o1 + k1] * E1[o];
        v = fma(sin4b[o1 + k1], E1[pl + o], v);
    }
    {
        const int64_t pl = (int64_t)n0 * n1, o = (int64_t)k0 * n1 + k1 + ((k2 & 1) ? 2 * pl : 0);
        v = fma(sin4[o2 + k2], E2[o], v);
        v = fma(sin4b[o2 + k2], E2[pl + o], v);
    }
    if (g.act[0]) {
        const int64_t pl = (int64_t)n1 * n2, o = (int64_t)k1 * n2 + k2 + ((k0 & 1) ? 2 * pl : 0);
        v = fma(sin4[k0], E0[o], v);
        v = fma(sin4b[k0], E0[pl + o], v);
    }
    const int64_t t = k0 * g.is[0] + (int64_t)k1 * g.is[1] + k2;
    out[t] = fma(tab[t], v, out[t]);
}

// x(k) *= Lambda_R(k) (stage output only); ld: per-axis eigenvalues of D2_s,
// axis s at offset off_s
__global__ void rhs6_symbol_kernel(const Grid3 gg, const double *__restrict__ ld, int64_t off1, int64_t off2,
                                   double *__restrict__ x)
{
    const Geo g = make_geo(gg);
    const int k2 = blockIdx.x * blockDim.x + threadIdx.x;
    const int k1 = blockIdx.y * blockDim.y + threadIdx.y;
    const int k0 = blockIdx.z;
    if (k2 >= g.ni[2] || k1 >= g.ni[1]) return;
    const int k[3] = {k0, k1, k2};
    const int64_t off[3] = {0, off1, off2};
    double lam[3];
    for (int s = 0; s < 3; ++s) lam[s] = g.act[s] ? ld[off[s] + k[s]] : 0.0;
    double sym = 0.0;
    for (int s = 0; s < 3; ++s)
        for (int r = 0; r < 3; ++r)
            if (r != s && g.act[s] && g.act[r]) {
                const double hs2 = g.h[s] * g.h[s], hr2 = g.h[r] * g.h[r];
                sym += (hs2 * hs2 / 240.0 + hs2 * hr2 / 144.0) * lam[s] * lam[s] * lam[r];
            }
    x[k0 * g.is[0] + (int64_t)k1 * g.is[1] + k2] *= sym;
}

// out += E on the layers (stage output only)
__global__ void rhs6_e_scatter_kernel(const Grid3 gg, const double *__restrict__ E0, const double *__restrict__ E1,
                                      const double *__restrict__ E2, double *__restrict__ out)
{
    const Geo g = make_geo(gg);
    const int k2 = blockIdx.x * blockDim.x + threadIdx.x;
    const int k1 = blockIdx.y * blockDim.y + threadIdx.y;
    const int k0 = blockIdx.z;
    if (k2 >= g.ni[2] || k1 >= g.ni[1]) return;
    const int n0 = g.ni[0], n1 = g.ni[1], n2 = g.ni[2];
    const int j[3] = {g.act[0] ? k0 + 1 : 0, k1 + 1, k2 + 1};
    double v = 0.0;
    for (int s = 0; s < 3; ++s) {
        const int dd = face_dist(g, s, j[s]);
        if (dd > 2) continue;
        const int sl = (j[s] <= g.M[s] / 2 ? 0 : 2) + (dd - 1);
        if (s == 0) v = E0[((int64_t)sl * n1 + k1) * n2 + k2];
        else if (s == 1) v = E1[((int64_t)sl * n0 + k0) * n2 + k2];
        else v = E2[((int64_t)sl * n0 + k0) * n1 + k1];
        break;
    }
    out[k0 * g.is[0] + (int64_t)k1 * g.is[1] + k2] += v;
}

// tabc = sc / lambda_c, tab4 = sc / Lambda4 on the mode grid (dense interior).
__global__ void eigen_tables_kernel(const Grid3 gg, const double *lc, const double *ld, int64_t off1,
                                    int64_t off2, double sc, double *tabc, double *tab4, double *tabR)
{
    const Geo g = make_geo(gg);
    const int64_t total = (int64_t)g.ni[0] * g.ni[1] * g.ni[2];
    const int64_t off[3] = {0, off1, off2};
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total;
         t += (int64_t)gridDim.x * blockDim.x) {
        int k[3];
        int64_t rem = t;
        for (int s = 0; s < 3; ++s) {
            const int64_t q = rem / g.is[s];
            rem -= q * g.is[s];
            k[s] = (int)q;
        }
        double c = 0.0, d = 0.0, lam[3];
        for (int s = 0; s < 3; ++s) {
            lam[s] = 0.0;
            if (!g.act[s]) continue;
            c += lc[off[s] + k[s]];
            lam[s] = ld[off[s] + k[s]];
            d += lam[s];
        }
        for (int s = 0; s < 3; ++s)
            for (int r = s + 1; r < 3; ++r)
                if (g.act[s] && g.act[r])
                    d += (g.h[s] * g.h[s] + g.h[r] * g.h[r]) / 12.0 * lam[s] * lam[r];
        tabc[t] = sc / c;
        tab4[t] = sc / d;
        if (tabR) {
            // tab4 * Lambda_R / Lambda4 maps u1's coefficients (tab4 * 4^d S gtilde)
            // to those of the smoothing solve of R_spec; tab4 is added so that one
            // table also carries u1 itself into the final transform
            double sym = 0.0;
            for (int s = 0; s < 3; ++s)
                for (int r = 0; r < 3; ++r)
                    if (r != s && g.act[s] && g.act[r]) {
                        const double hs2 = g.h[s] * g.h[s], hr2 = g.h[r] * g.h[r];
                        sym += (hs2 * hs2 / 240.0 + hs2 * hr2 / 144.0) * lam[s] * lam[s] * lam[r];
                    }
            tabR[t] = sc * sym / (d * d) + sc / d;
        }
    }
}

inline int grid_for(int64_t work) { int64_t b = (work + 255) / 256; return (int)(b < 4096 ? (b > 0 ? b : 1) : 4096); }

}  // namespace

StencilCoef make_stencil_coef(const Grid3 &g)
{
    StencilCoef c{};
    const double h[3] = {g.h0, g.h1, g.h2};
    int act[3];
    for (int s = 0; s < 3; ++s) act[s] = (g.d == 3) || (s > 0);
    for (int s = 0; s < 3; ++s) {
        if (!act[s]) continue;
        const double hs2 = h[s] * h[s];
        c.wf[s] = 1.0 / hs2;
        for (int r = 0; r < 3; ++r) {
            if (r == s || !act[r]) continue;
            const double hr2 = h[r] * h[r];
            const double q = (hs2 + hr2) / 12.0 / (hs2 * hr2);
            c.wf[s] -= 2.0 * q;
            c.we[s][r] = q;
            c.a[s][r] = (hs2 * hs2 / 240.0 + hs2 * hr2 / 144.0) / (hs2 * hs2 * hr2);
        }
    }
    return c;
}

dim3 grid3(int x, int y, int z) { return dim3((x + 31) / 32, (y + 7) / 8, z); }

cudaError_t launch_gtilde_planes(const Grid3 &g, const StencilCoef &c, const double *U, double *Q0, double *Q1,
                                 double *Q2, cudaStream_t st)
{
    const int64_t n0 = g.d == 3 ? g.n0 - 2 : 1, n1 = g.n1 - 2, n2 = g.n2 - 2;
    const int64_t total = (g.d == 3 ? 2 * n1 * n2 : 0) + 2 * n0 * n2 + 2 * n0 * n1;
    gtilde_planes_kernel<<<grid_for(total), 256, 0, st>>>(g, c, U, Q0, Q1, Q2);
    return cudaGetLastError();
}

cudaError_t launch_gtilde_expand(const Grid3 &g, const double *Q0, const double *Q1, const double *Q2,
                                 const double *sin4, const double *tab, const double *add, double *out,
                                 cudaStream_t st, const double *tab2, const double *add2, double *out2, int fold,
                                 const double *ascale)
{
    gtilde_expand_kernel<<<grid3(g.n2 - 2, g.n1 - 2, g.d == 3 ? g.n0 - 2 : 1), dim3(32, 8), 0, st>>>(
        g, Q0, Q1, Q2, sin4, tab, add, out, tab2, add2, out2, fold, ascale);
    return cudaGetLastError();
}

cudaError_t launch_gtilde_scatter(const Grid3 &g, const double *Q0, const double *Q1, const double *Q2,
                                  double *out, cudaStream_t st)
{
    gtilde_scatter_kernel<<<grid3(g.n2 - 2, g.n1 - 2, g.d == 3 ? g.n0 - 2 : 1), dim3(32, 8), 0, st>>>(
        g, Q0, Q1, Q2, out);
    return cudaGetLastError();
}

cudaError_t launch_rhs6_w(const Grid3 &g, const StencilCoef &c, const double *U, double *W, cudaStream_t st)
{
    rhs6_w_kernel<<<grid3(g.n2, g.n1, g.n0), dim3(32, 8), 0, st>>>(g, c, U, W);
    return cudaGetLastError();
}

cudaError_t launch_rhs6_core(const Grid3 &g, const double *W, double *R, cudaStream_t st)
{
    rhs6_core_kernel<<<grid3(g.n2 - 2, g.n1 - 2, g.d == 3 ? g.n0 - 2 : 1), dim3(32, 8), 0, st>>>(g, W, R);
    return cudaGetLastError();
}

cudaError_t launch_rhs6_extrap(const Grid3 &g, double *R, cudaStream_t st)
{
    const int64_t n0 = g.d == 3 ? g.n0 - 2 : 1, n1 = g.n1 - 2, n2 = g.n2 - 2;
    const int64_t total = (g.d == 3 ? 2 * n1 * n2 : 0) + 2 * (g.d == 3 ? n0 - 2 : 1) * n2 +
                          2 * (g.d == 3 ? n0 - 2 : 1) * (n1 - 2);
    rhs6_extrap_kernel<<<grid_for(total), 256, 0, st>>>(g, R);
    return cudaGetLastError();
}

cudaError_t launch_rhs6_spectral(const Grid3 &g, const StencilCoef &c, const double *U, double *W, double *Rt,
                                 double *E0, double *E1, double *E2, int kind, cudaStream_t st)
{
    if (kind == 0) {
        // W of the odd continuation on the nodes within 7 of a face
        const Shell sh = make_shell(g, 0, 0, 8);
        rhs6_wband_kernel<<<grid_for(sh.count), 256, 0, st>>>(g, sh, c, U, W);
    } else if (kind == 1) {
        // the core nodes (indices 2..M-2) within 3 of the core's faces
        const Shell sh = make_shell(g, 2, 4, 4);
        rhs6_taps_kernel<<<grid_for(sh.count), 256, 0, st>>>(g, sh, c, U, W, Rt);
    } else {
        const int64_t n0 = g.d == 3 ? g.n0 - 2 : 1, n1 = g.n1 - 2, n2 = g.n2 - 2;
        const int64_t total = 4 * ((g.d == 3 ? n1 * n2 : 0) + n0 * n2 + n0 * n1);
        rhs6_e_kernel<<<grid_for(total), 256, 0, st>>>(g, c, U, W, Rt, E0, E1, E2);
    }
    return cudaGetLastError();
}

cudaError_t launch_layers_combine(double *P0, int64_t pl0, double *P1, int64_t pl1, double *P2, int64_t pl2,
                                  int nl, cudaStream_t st)
{
    layers_combine_kernel<<<grid_for((int64_t)nl * (pl0 + pl1 + pl2)), 256, 0, st>>>(P0, (int)pl0, P1, (int)pl1, P2,
                                                                                   (int)pl2, nl);
    return cudaGetLastError();
}

cudaError_t launch_rhs6_e_expand(const Grid3 &g, const double *E0, const double *E1, const double *E2,
                                 const double *sin4, const double *sin4b, const double *tab, double *out,
                                 cudaStream_t st)
{
    rhs6_e_expand_kernel<<<grid3(g.n2 - 2, g.n1 - 2, g.d == 3 ? g.n0 - 2 : 1), dim3(32, 8), 0, st>>>(
        g, E0, E1, E2, sin4, sin4b, tab, out);
    return cudaGetLastError();
}

cudaError_t launch_rhs6_symbol(const Grid3 &g, const double *ld, int64_t off1, int64_t off2, double *x,
                               cudaStream_t st)
{
    rhs6_symbol_kernel<<<grid3(g.n2 - 2, g.n1 - 2, g.d == 3 ? g.n0 - 2 : 1), dim3(32, 8), 0, st>>>(
        g, ld, off1, off2, x);
    return cudaGetLastError();
}

cudaError_t launch_rhs6_e_scatter(const Grid3 &g, const double *E0, const double *E1, const double *E2,
                                  double *out, cudaStream_t st)
{
    rhs6_e_scatter_kernel<<<grid3(g.n2 - 2, g.n1 - 2, g.d == 3 ? g.n0 - 2 : 1), dim3(32, 8), 0, st>>>(
        g, E0, E1, E2, out);
    return cudaGetLastError();
}

namespace {
__global__ void box_copy_kernel(const double *__restrict__ src, int64_t s0, int64_t s1, double *__restrict__ dst,
                                int64_t d0, int64_t d1, int e0, int e1, int e2)
{
    const int64_t total = (int64_t)e0 * e1 * e2;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t row = i / e2;
        const int i2 = (int)(i - row * e2);
        const int i0 = (int)(row / e1), i1 = (int)(row - (int64_t)i0 * e1);
        dst[i0 * d0 + i1 * d1 + i2] = src[i0 * s0 + i1 * s1 + i2];
    }
}

__global__ void validate_rho_kernel(const double *__restrict__ rho, int n0, int n1, int n2, int act0, int act1,
                                    int act2, int k, int *word)
{
    const int64_t total = (int64_t)n0 * n1 * n2;
    int bits = 0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t row = i / n2;
        const int i2 = (int)(i - row * n2);
        const int i0 = (int)(row / n1), i1 = (int)(row - (int64_t)i0 * n1);
        // interior nodes only (the boundary entries of rho are not used)
        const bool b0 = act0 && (i0 == 0 || i0 == n0 - 1), b1 = act1 && (i1 == 0 || i1 == n1 - 1),
                   b2 = act2 && (i2 == 0 || i2 == n2 - 1);
        if (b0 || b1 || b2) continue;
        // integer tests on the bits: exponent all ones = NaN or infinity; zero = +-0
        const long long u = __double_as_longlong(rho[i]);
        if (((u >> 52) & 0x7ff) == 0x7ff) {
            bits |= 1;
        } else if ((u << 1) != 0) {
            const bool near0 = act0 && (i0 < k || i0 > n0 - 1 - k), near1 = act1 && (i1 < k || i1 > n1 - 1 - k),
                       near2 = act2 && (i2 < k || i2 > n2 - 1 - k);
            if (near0 || near1 || near2) bits |= 2;
        }
    }
    if (bits) atomicOr(word, bits);
}

__global__ void to_dd_kernel(const double *x, ddr *y, int64_t n)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        y[i] = dd_from(x[i]);
}
}  // namespace

cudaError_t launch_box_copy(const double *src, int64_t s0, int64_t s1, double *dst, int64_t d0, int64_t d1,
                            int e0, int e1, int e2, cudaStream_t st)
{
    const int64_t total = (int64_t)e0 * e1 * e2;
    if (total <= 0) return cudaSuccess;
    box_copy_kernel<<<grid_for(total), 256, 0, st>>>(src, s0, s1, dst, d0, d1, e0, e1, e2);
    return cudaGetLastError();
}

cudaError_t launch_validate_rho(const double *rho, int n0, int n1, int n2, int act0, int act1, int act2, int k,
                                int *word, cudaStream_t st)
{
    validate_rho_kernel<<<grid_for((int64_t)n0 * n1 * n2), 256, 0, st>>>(rho, n0, n1, n2, act0, act1, act2, k,
                                                                          word);
    return cudaGetLastError();
}

cudaError_t launch_to_dd(const double *x, ddr *y, int64_t n, cudaStream_t st)
{
    to_dd_kernel<<<grid_for(n), 256, 0, st>>>(x, y, n);
    return cudaGetLastError();
}

cudaError_t launch_eigen_tables(const Grid3 &g, const double *lc, const double *ld, int64_t off1,
                                int64_t off2, double sc, double *tabc, double *tab4, double *tabR, cudaStream_t st)
{
    const int64_t total = (int64_t)(g.d == 3 ? g.n0 - 2 : 1) * (g.n1 - 2) * (g.n2 - 2);
    eigen_tables_kernel<<<grid_for(total), 256, 0, st>>>(g, lc, ld, off1, off2, sc, tabc, tab4, tabR);
    return cudaGetLastError();
}

}  // namespace idp
