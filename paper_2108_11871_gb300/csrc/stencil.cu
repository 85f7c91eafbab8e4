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

// Forward sine transform of gtilde from the transformed parts (U = 4^d S gtilde):
//   val(k) = sum_s sin4_s(k_s) (Qs[0](k_other) + (-1)^{k_s} Qs[1](k_other)),
// sin4_s(k) = 4 sin(pi (k+1)/M_s); Qs holds the (d-1)-dimensional transforms of
// the parts (4^{d-1} S).  out = tab * val (+ add).
__global__ void gtilde_expand_kernel(const Grid3 gg, const double *__restrict__ Q0, const double *__restrict__ Q1,
                                     const double *__restrict__ Q2, const double *__restrict__ sin4,
                                     const double *__restrict__ tab, const double *add, double *out)
{
    const Geo g = make_geo(gg);
    const int k2 = blockIdx.x * blockDim.x + threadIdx.x;
    const int k1 = blockIdx.y * blockDim.y + threadIdx.y;
    const int k0 = blockIdx.z;
    if (k2 >= g.ni[2] || k1 >= g.ni[1]) return;
    const int n0 = g.ni[0], n1 = g.ni[1], n2 = g.ni[2];
    const double *sn0 = sin4, *sn1 = sin4 + (g.act[0] ? n0 : 0), *sn2 = sn1 + n1;
    double v;
    {
        const double a = Q1[(int64_t)k0 * n2 + k2], b = Q1[(int64_t)(n0 + k0) * n2 + k2];
        v = sn1[k1] * ((k1 & 1) ? a - b : a + b);
    }
    {
        const double a = Q2[(int64_t)k0 * n1 + k1], b = Q2[(int64_t)(n0 + k0) * n1 + k1];
        v = fma(sn2[k2], (k2 & 1) ? a - b : a + b, v);
    }
    if (g.act[0]) {
        const int64_t o = (int64_t)k1 * n2 + k2;
        const double a = Q0[o], b = Q0[(int64_t)n1 * n2 + o];
        v = fma(sn0[k0], (k0 & 1) ? a - b : a + b, v);
    }
    const int64_t t = k0 * g.is[0] + (int64_t)k1 * g.is[1] + k2;
    out[t] = add ? fma(tab[t], v, add[t]) : tab[t] * v;
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
// of c_sr D2_s D2_s D2_r u.  Grid: x = node index 2, y = index 1, z = index 0.
__global__ void rhs6_w_kernel(const Grid3 gg, const StencilCoef c, const double *__restrict__ U,
                              double *__restrict__ W)
{
    const Geo g = make_geo(gg);
    const int j2 = blockIdx.x * blockDim.x + threadIdx.x;
    const int j1 = blockIdx.y * blockDim.y + threadIdx.y;
    const int j0 = blockIdx.z;
    if (j2 >= g.n[2] || j1 >= g.n[1]) return;
    const int j[3] = {j0, j1, j2};
    const int64_t nodes = (int64_t)g.n[0] * g.n[1] * g.n[2];
    const int64_t t = j0 * g.ns[0] + (int64_t)j1 * g.ns[1] + j2;
    const double u0 = U[t];
    double e[3];
    bool inner[3];
    for (int r = 0; r < 3; ++r) {
        inner[r] = !g.act[r] || (j[r] >= 1 && j[r] <= g.M[r] - 1);
        e[r] = 0.0;
        if (g.act[r] && inner[r]) e[r] = fma(-2.0, u0, U[t + g.ns[r]] + U[t - g.ns[r]]);
    }
    for (int s = 0; s < 3; ++s) {
        if (!g.act[s]) continue;
        bool ok = true;
        for (int r = 0; r < 3; ++r)
            if (r != s && !inner[r]) ok = false;
        if (!ok) continue;
        double w = 0.0;
        for (int r = 0; r < 3; ++r)
            if (r != s && g.act[r]) w = fma(c.a[s][r], e[r], w);
        W[(int64_t)s * nodes + t] = w;
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

// tabc = sc / lambda_c, tab4 = sc / Lambda4 on the mode grid (dense interior).
__global__ void eigen_tables_kernel(const Grid3 gg, const double *lc, const double *ld, int64_t off1,
                                    int64_t off2, double sc, double *tabc, double *tab4)
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
                                 cudaStream_t st)
{
    gtilde_expand_kernel<<<grid3(g.n2 - 2, g.n1 - 2, g.d == 3 ? g.n0 - 2 : 1), dim3(32, 8), 0, st>>>(
        g, Q0, Q1, Q2, sin4, tab, add, out);
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

namespace {
__global__ void to_dd_kernel(const double *x, ddr *y, int64_t n)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        y[i] = dd_from(x[i]);
}
}  // namespace

cudaError_t launch_to_dd(const double *x, ddr *y, int64_t n, cudaStream_t st)
{
    to_dd_kernel<<<grid_for(n), 256, 0, st>>>(x, y, n);
    return cudaGetLastError();
}

cudaError_t launch_eigen_tables(const Grid3 &g, const double *lc, const double *ld, int64_t off1,
                                int64_t off2, double sc, double *tabc, double *tab4, cudaStream_t st)
{
    const int64_t total = (int64_t)(g.d == 3 ? g.n0 - 2 : 1) * (g.n1 - 2) * (g.n2 - 2);
    eigen_tables_kernel<<<grid_for(total), 256, 0, st>>>(g, lc, ld, off1, off2, sc, tabc, tab4);
    return cudaGetLastError();
}

}  // namespace idp
