// Allocation-free variant of the 6th-order right-hand-side step.
//
// Some callers cannot let a library call cudaMalloc: applications whose own
// pool allocator has reserved nearly all of the GPU's memory up front (a
// library allocation would then fail or fragment the pool), and time-critical
// loops in which the implicit device synchronisation of cudaMalloc/cudaFree is
// not acceptable.  idp_rhs6_noalloc serves them: it computes the same
// right-hand side R as the plan-based solver, but keeps its scratch (the three
// second-difference arrays W_s) in the fixed device array below instead of
// plan workspace.  The caller passes u1 and R; nothing is allocated.
#include "idp_internal.cuh"
#include "../../include/idp.h"

using namespace idp;

namespace {

// Fixed scratch: 3 node arrays of at most IDP_RHS6_NOALLOC_MAX_NODES doubles
// (12 MiB).  It lives in every GPU that loads the library until the process
// exits, and it is shared by all calls.
static __device__ __align__(256) double g_rhs6_scratch[3 * IDP_RHS6_NOALLOC_MAX_NODES];

// Device address of the scratch array on the current device.  The host-side
// symbol is only a stand-in, not a device address, so the address is looked up
// on every call (cheap once the device code is loaded): a cached address would
// go stale when the caller resets the device and the library's device code is
// loaded again, possibly elsewhere.
int scratch_for_current_device(double **out)
{
    void *p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_rhs6_scratch);
    if (e != cudaSuccess || !p) return IDP_ECUDA;
    *out = static_cast<double *>(p);
    return IDP_OK;
}

}  // namespace

extern "C" int idp_rhs6_noalloc(int d, const int64_t n[], const double h[], const double *u1, double *R,
                                void *stream)
{
    if (!n || !h || !u1 || !R) return IDP_EINVAL;
    if (d != 2 && d != 3) return IDP_EINVAL;
    int64_t nodes = 1, interior = 1;
    for (int s = 0; s < d; ++s) {
        if (!(h[s] > 0.0)) return IDP_EINVAL;
        if (n[s] < 8) return IDP_EINVAL;   // the extrapolation reads layers 2..5
        // checked before each product, so that no product can overflow
        if (n[s] > IDP_RHS6_NOALLOC_MAX_NODES / nodes) return IDP_ESCRATCH;
        nodes *= n[s];
        interior *= n[s] - 2;
    }
    const char *a = (const char *)u1, *b = (const char *)R;
    if (a < b + interior * 8 && b < a + nodes * 8) return IDP_EALIAS;
    double *W = nullptr;
    int rc = scratch_for_current_device(&W);
    if (rc) return rc;
    const int o = 3 - d;
    int nn[3] = {1, 1, 1};
    double hh[3] = {1.0, 1.0, 1.0};
    for (int s = 0; s < d; ++s) {
        nn[s + o] = (int)n[s];
        hh[s + o] = h[s];
    }
    const Grid3 g{d, nn[0], nn[1], nn[2], hh[0], hh[1], hh[2]};
    const StencilCoef c = make_stencil_coef(g);
    cudaStream_t st = (cudaStream_t)stream;
    // Every W entry that the core kernel reads is written by the first kernel of
    // this call, so nothing in the scratch has to start at zero.
    if (launch_rhs6_w(g, c, u1, W, st) != cudaSuccess) return IDP_ECUDA;
    if (launch_rhs6_core(g, W, R, st) != cudaSuccess) return IDP_ECUDA;
    if (launch_rhs6_extrap(g, R, st) != cudaSuccess) return IDP_ECUDA;
    return IDP_OK;
}
