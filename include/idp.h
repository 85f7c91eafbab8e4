/*
 * idp.h -- C ABI of the GB300 infinite-domain Poisson solver.
 *
 * The library evaluates, at every node of a uniform 1-D, 2-D or 3-D grid, the
 * convolution of the free-space Green's function of the Laplacian with a
 * density rho whose support lies inside the grid (arXiv 2108.11871, section 1,
 * eqs. GreensFcnIntegral / InfDomainPoisson):
 *
 *     phi = phi* + phi_H                       (section 2, eqs. PhiStarEqn, PhiHeqn)
 *
 *   phi*  : Dirichlet-0 Poisson solve by discrete sine transforms (section 3);
 *   g     : phi_H on the boundary, the trapezoid sum of G * rho evaluated as
 *           per-slice FFT convolutions (section 4, eqs. TrapOrig2D, Trap2D,
 *           convolution);
 *   gtilde: the boundary data moved to the right-hand side of the compact
 *           4th-order operator (section 5, eq. harmonic4thOrderNH2D);
 *   u1    : the 4th-order harmonic solve (section 5, eigenvectors = sines);
 *   R, u2 : the 6th-order deferred correction with cubic extrapolation next
 *           to the boundary (section 5, eqs. 6thOrderRelation2D/3D).
 *
 * Conventions shared by every entry point
 *   - Grids: d in {1, 2, 3}; n[s] = node count along array axis s INCLUDING
 *     the two boundary nodes (n[s] = M_s + 1, M_s panels, n[s] >= 3); h[s] > 0
 *     is the mesh width.  Arrays are FP64, C order, last axis contiguous,
 *     prod(n) entries.
 *   - Sizes: the FFT-based transforms take M_s = 2^a with 16 <= M_s <= 512 or
 *     M_s = 3 * 2^a with 48 <= M_s <= 384; idp_create_plan pads any other
 *     M_s <= 512 to the next of these (section 2), idp_create_plan_exact solves
 *     any 7 <= M_s <= 512 on the grid as given; M_s > 512 gives IDP_ESUPPORT.
 *   - rho is read on interior nodes only; its boundary entries are ignored.
 *     The method assumes rho vanishes near the boundary (section 2); the
 *     library checks it only in validation mode (IDP_KEY_VALIDATE).
 *   - Device pointers are CUDA device memory owned by the caller and must
 *     stay valid until the work queued on `stream` has finished.
 *   - `stream` is a cudaStream_t passed as void* (NULL = legacy default stream).
 *     All device work is queued on it; calls return before it completes.
 *   - Return value: IDP_OK (0) or a negative IDP_E* code.  Errors in the
 *     arguments are reported synchronously and nothing is queued.  Errors
 *     raised later by queued work are reported by idp_plan_status().
 *   - A plan may be used by one stream at a time; calls on one plan must not
 *     overlap on the device.
 */
#ifndef IDP_H
#define IDP_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum {
    IDP_OK = 0,
    IDP_EINVAL = -1,     /* bad argument (dimension, size, order, null pointer) */
    IDP_ENOMEM = -2,     /* device or host allocation failed */
    IDP_ECUDA = -3,      /* a CUDA call failed; see idp_last_cuda_error() */
    IDP_EALIAS = -4,     /* rho and phi overlap */
    IDP_ESUPPORT = -5,   /* size or option outside the supported set */
    IDP_ESCRATCH = -6,   /* problem larger than the fixed scratch of idp_rhs6_noalloc */
    IDP_ETIMEOUT = -7,   /* a device-side wait exceeded its iteration limit */
    IDP_EGUARD = -8      /* a guard region around a workspace buffer was overwritten (idp_plan_check_guards) */
};

/* keys for idp_plan_set */
enum {
    IDP_KEY_USE_GRAPH = 1,  /* 1 (default): replay solves from a CUDA graph; 0: plain launches */
    IDP_KEY_PRECISION = 2,  /* IDP_PRECISION_*: arithmetic of the full-volume sine transforms */
    IDP_KEY_AUTOTUNE = 4,   /* value 1: time candidate settings now on the plan's buffers and keep
                               the fastest -- slice chunking of the 3-D face convolutions, block
                               shape of the full-volume sine passes and, in precision MIXED,
                               tensor-core matrix pass vs double-float FFT pass (both within the
                               mixed accuracy); synchronises the device */
    IDP_KEY_DST_SHAPE = 5,  /* block shape of the full-volume sine passes (results are the same
                               bits for every shape): 0 by size (default), 8 = 8 lines per block,
                               -8 = 8 lines on 128 threads (M = 128 only), 32 = 32 lines (M = 128
                               only), 16 = 16 lines (M = 256 only), 4 = 4 lines on 128 threads
                               (M = 256 and 512 only); a shape that does not apply to a length
                               falls back to 0 */
    IDP_KEY_STALL_TEST = 3, /* test hook for failure handling (mixed precision only): the next
                               tensor-core pass issues no products, so its bounded wait expires
                               (after ~5 ms); the kernel records the failure, frees its tensor
                               memory and returns, and idp_plan_status reports IDP_ETIMEOUT */
    IDP_KEY_MIXED_BOUNDARY_DF32 = 8, /* value 1: in the tensor-core modes (IDP_PRECISION_MIXED_*) the 3-D
                               boundary convolutions run in double-float arithmetic (48 significant
                               bits, as in IDP_PRECISION_DF32) instead of FP64; value 0 (default):
                               FP64.  No effect in the other modes.  Setting 1 allocates the
                               double-float copies of the kernel spectra. */
    IDP_KEY_NVTX = 9,       /* value 1: NVTX ranges (NVTX v3, host side, at enqueue time) around every
                               kernel launch of a solve or stage, named after its IDP_KERNEL_* family
                               ("idp:dst", "idp:face", ...), and around the solve and its stages
                               ("idp:solve", "idp:boundary values g", "idp:sine transform ..."), so
                               that a profiler attributes the kernels to the steps of the method;
                               solves then use plain launches (ranges recorded while a graph is
                               captured would not recur on its replays).  0 (default): none.
                               Results are the same bits either way. */
    IDP_KEY_GUARD_TEST = 7, /* test hook for idp_plan_check_guards: value 1 overwrites the first
                               byte of the guard region in front of the plan's first buffer (a
                               write inside that allocation, from the host), value 0 restores it;
                               synchronises the device */
    IDP_KEY_VALIDATE = 6    /* validation mode, value k >= 0 (0, the default: off).  Every solve
                               or stage first checks the caller's rho on the device: a NaN or
                               infinite value anywhere makes the next idp_plan_status return
                               IDP_EINVAL; a non-zero value on a node within k layers of the
                               boundary (some index i_s with 0 < i_s < k or M_s - k < i_s < M_s;
                               section 2 assumes rho vanishes near the boundary) makes it return
                               IDP_ESUPPORT (checked first: IDP_EINVAL).  The solve itself still
                               runs; its output is then not to be used.  Costs one read of rho. */
};

/* values of IDP_KEY_PRECISION */
enum {
    IDP_PRECISION_FP64 = 0,        /* FP64 FFT-based sine transforms (default) */
    IDP_PRECISION_MIXED_BF16X3 = 1, /* the sine transforms of rho, of R and the final inverse become
                                      dense sine-matrix products on the tensor cores: operands split
                                      into three BF16 pieces, six products, FP32 accumulation
                                      (relative error of phi ~1e-5 or better); the eigenvalue division,
                                      the boundary values (see IDP_KEY_MIXED_BOUNDARY_DF32) and the
                                      stencils stay FP64; the transform that produces u1 (whose sixth
                                      differences form R) and the transforms of the boundary layers run
                                      in double-float arithmetic (48 significant bits).  Setting it
                                      allocates the pieces of the sine matrices and FP32 temporaries. */
    IDP_PRECISION_DF32 = 2,        /* the FFT-based transforms (sine transforms of rho, R and the final
                                      inverse, and the 3-D boundary convolutions) in double-float
                                      arithmetic (a value is a pair of FP32 numbers, ~48 significant
                                      bits) on the FP32 pipe, FP64 arrays in and out; the transform
                                      producing u1 and all stencils stay FP64.  Results agree with
                                      FP64 to a few 1e-13 relative. */
    IDP_PRECISION_MIXED_TF32X3 = 3 /* as MIXED_BF16X3, with the operands split into two TF32 pieces
                                      (hi + lo, ~22 significant bits) and three products (hi*hi,
                                      hi*lo, lo*hi; tcgen05 kind::tf32), FP32 accumulation */
};

/* stages for idp_solve_stage */
enum {
    IDP_STAGE_BOUNDARY = 1, /* out: node array, g on the boundary, 0 inside (section 4) */
    IDP_STAGE_GTILDE = 2,   /* out: interior array prod(n[s]-2), gtilde (eq. harmonic4thOrderNH2D) */
    IDP_STAGE_PHISTAR = 3,  /* out: node array, phi* (section 3), 0 on the boundary */
    IDP_STAGE_U1 = 4,       /* out: node array, u1 inside, g on the boundary (section 5) */
    IDP_STAGE_R = 5,        /* out: interior array, 6th-order right-hand side R incl. extrapolation */
    IDP_STAGE_PHI = 6       /* out: node array, phi (same as idp_solve) */
};

typedef struct idp_plan_s *idp_plan;

/* Create a plan for one grid (section 3 grid, section 5 order).
 *   out   : receives the plan handle (owned by the caller; free with idp_destroy_plan)
 *   d     : 1, 2 or 3
 *   n[d]  : node counts including boundary nodes, n[s] >= 3.  Panel counts
 *           n[s] - 1 of 16, 32, 48, 64, 96, 128, 192, 256, 384 or 512 are solved
 *           as given; any other count up to 512 is padded (section 2: the domain
 *           is extended by a few panels, h unchanged, the extra panels split
 *           between the two ends) to the next of these, the solve runs on the
 *           larger grid and phi is returned at the caller's nodes (the
 *           free-space potential there, to the method's accuracy); larger counts
 *           give IDP_ESUPPORT.  A padded plan offers full solves only
 *           (idp_solve, _host, _batched, _profile_solve, stage PHI; other stages:
 *           IDP_ESUPPORT).  idp_plan_grid reports the grid solved on.
 *   h[d]  : mesh widths
 *   order : 4 or 6 (accuracy order of the harmonic correction, section 5; for
 *           d = 1 the correction is exact, the straight line through the two
 *           end values of g (section 5), and order has no effect)
 * d = 1 plans run FP64 only (IDP_KEY_PRECISION other than FP64: IDP_ESUPPORT);
 * their stages are BOUNDARY, PHISTAR, U1 (the straight line, g at the ends)
 * and PHI (GTILDE and R: IDP_ESUPPORT).
 * Allocates all device workspace and precomputes the sine/twiddle tables,
 * the eigenvalue tables and the spectra of the boundary convolution kernels
 * on the current CUDA device; synchronises that device before returning. */
int idp_create_plan(idp_plan *out, int d, const int64_t n[], const double h[], int order);

/* Create a plan that solves on the grid as given, for any panel count
 * 7 <= n[s] - 1 <= 512 (no padding; section 2's remedy of extending the domain
 * is what idp_create_plan does).  Arguments as idp_create_plan; n[s] >= 8.
 * Sine transforms whose length has no FFT here run as direct sums
 * (O(n) work per point and axis: FP64 in precision FP64, double-float in the
 * other modes) -- except in the tensor-core modes, whose sine-matrix products
 * take any length, so that there only the transform producing u1 and the
 * transforms of the boundary layers are direct sums.  The boundary
 * convolutions use the smallest FFT length 2P >= 2M (P = M where M has one).
 * Meant for the tensor-core modes (the precision sweep of 256^3 and
 * 384 x 256 x 256 interior points); in FP64 a padded plan is faster. */
int idp_create_plan_exact(idp_plan *out, int d, const int64_t n[], const double h[], int order);

/* Set a plan option (IDP_KEY_*). */
int idp_plan_set(idp_plan plan, int key, int64_t value);

/* phi = G * rho on every node (section 2).  rho, phi: device arrays of prod(n)
 * doubles; they must not overlap (IDP_EALIAS). */
int idp_solve(idp_plan plan, const double *rho, double *phi, void *stream);

/* Same as idp_solve with HOST arrays of prod(n) doubles; waits for the stream
 * before returning.  Page-locked buffers (cudaHostAlloc / cudaHostRegister)
 * are read and written by the kernels themselves through their device views
 * (the first real-FFT pass reads rho and leaves a device copy; the kernels that
 * produce phi write it), from a CUDA graph of their own keyed by the two
 * pointers; pageable buffers are copied up and back around the solve.  The plan
 * allocates its device staging buffers on the first call. */
int idp_solve_host(idp_plan plan, const double *rho_host, double *phi_host, void *stream);

/* Solve `count` independent problems, plans[i] with rho[i] -> phi[i]
 * (device arrays), all queued on `stream`.  The plans must be distinct.  The
 * problems run concurrently, so no phi[i] may overlap any rho[j] or any other
 * phi[j] (IDP_EALIAS). */
int idp_solve_batched(int count, const idp_plan plans[], const double *const rho[],
                      double *const phi[], void *stream);

/* Run the method up to one intermediate stage and write it to `out`
 * (device array; layout given by the IDP_STAGE_* comment).  For checking
 * the components against a reference. */
int idp_solve_stage(idp_plan plan, int stage, const double *rho, double *out, void *stream);

/* Device-side status of the plan's last queued work: IDP_OK, IDP_ECUDA if a
 * launch or asynchronous error was recorded, IDP_ETIMEOUT if a bounded
 * device-side wait gave up, or (validation mode, IDP_KEY_VALIDATE) IDP_EINVAL /
 * IDP_ESUPPORT if a rho checked since the last call failed the check (each
 * reported once; the outputs of that solve are invalid, the plan stays usable).
 * Synchronises the plan's last stream. */
int idp_plan_status(idp_plan plan);

/* kernel families reported by idp_profile_solve */
enum {
    IDP_KERNEL_DST = 1,          /* sine-transform pass along one axis (sections 3, 5) */
    IDP_KERNEL_RFFT = 2,         /* boundary stage 1: real FFT of zero-padded lines (section 4) */
    IDP_KERNEL_FACE = 3,         /* boundary stage 2: per-slice FFT x kernel spectrum, summed over slices */
    IDP_KERNEL_FACE_INVB = 4,    /* boundary stage 3a: inverse FFT across the face */
    IDP_KERNEL_FACE_C2R = 5,     /* boundary stage 3b: inverse real FFT and scatter to the face nodes */
    IDP_KERNEL_GTILDE = 6,       /* gtilde stencil on the boundary-adjacent layers (eq. harmonic4thOrderNH2D) */
    IDP_KERNEL_RHS6_W = 7,       /* 6th-order RHS: second differences of the odd continuation of u1 near the faces */
    IDP_KERNEL_RHS6_CORE = 8,    /* 6th-order RHS at the taps of the cubic extrapolation */
    IDP_KERNEL_RHS6_EXTRAP = 9,  /* layers of E = R - R_spec: cubic extrapolation and boundary terms */
    IDP_KERNEL_GTILDE_EXPAND = 10, /* sine transform of gtilde assembled from its transformed layers */
    IDP_KERNEL_DST_PARTS = 11,   /* sine passes over the boundary-adjacent layers of gtilde */
    IDP_KERNEL_MIXED = 12,       /* tensor-core sine-matrix pass (IDP_PRECISION_MIXED_BF16X3 / _TF32X3) */
    IDP_KERNEL_SUPPORT = 13,     /* reserved: no longer launched (the support flags of rho are made by the
                                    stage-1 pass along axis 2, timed under IDP_KERNEL_RFFT) */
    IDP_KERNEL_RHS6_EXPAND = 14, /* sine transform of the 6th-order layer correction from its layer transforms */
    IDP_KERNEL_LINE1D = 15,      /* d = 1: g at the two ends and the straight-line correction (section 5) */
    IDP_KERNEL_PAD = 16,         /* padded plans: rho into the padded grid, phi back to the caller's nodes */
    IDP_KERNEL_VALIDATE = 17     /* validation mode (IDP_KEY_VALIDATE): the check of rho */
};

/* Run one solve (as idp_solve, but with plain launches, all on `stream`, none
 * overlapped) and time every kernel launch with CUDA events recorded on `stream`.  kinds[i] receives the
 * IDP_KERNEL_* family and ms[i] the duration of launch i, for at most
 * `capacity` launches.  Synchronises the stream.  Returns the number of
 * launches timed (>= 0) or a negative IDP_E* code. */
int idp_profile_solve(idp_plan plan, const double *rho, double *phi, void *stream, int capacity,
                      int *kinds, float *ms);

/* Settings chosen by IDP_KEY_AUTOTUNE (or the defaults): out[0] = 1 if tuned,
 * out[1] = mixed path (0 tensor-core matrix, 1 double-float FFT), out[2..4] =
 * slice chunks of the face passes of axes 0..2, out[5..7] = slices per chunk,
 * out[8] = block shape of the full-volume sine passes (IDP_KEY_DST_SHAPE values). */
int idp_plan_tuning(idp_plan plan, int64_t out[9]);

/* Number of kernel launches one solve of this plan queues (valid after the
 * first solve). */
int idp_plan_launches(idp_plan plan, int64_t *launches);

/* Query the plan: node count of the caller's arrays, interior count of the grid
 * solved on, and device workspace bytes. */
int idp_plan_info(idp_plan plan, int64_t *nodes, int64_t *interior, int64_t *workspace_bytes);

/* Check the guard regions around every device buffer the plan allocated (256
 * bytes on each side, filled with a fixed byte at allocation): IDP_OK if all are
 * intact, IDP_EGUARD if a kernel wrote past the start or end of a buffer.  A
 * check for tests in place of a memory checker; synchronises the device and reads
 * back 512 bytes per buffer.  The paper has no counterpart. */
int idp_plan_check_guards(idp_plan plan);

/* The grid a plan solves on (section 2: a panel count the transforms do not
 * take is met by extending the domain by a few panels): n_solved[d] node counts
 * per axis, offset[d] the index of the caller's node 0 in it.  Equal to n[] and
 * 0 when no axis needed padding. */
int idp_plan_grid(idp_plan plan, int64_t n_solved[], int64_t offset[]);

/* Release the plan and all its device memory (synchronises the device). */
int idp_destroy_plan(idp_plan plan);

/* Allocation-free 6th-order right-hand side (no counterpart in the paper:
 * it exists for callers that cannot let a library allocate device memory --
 * applications whose own pool allocator holds nearly all GPU memory, and
 * time-critical loops that cannot afford cudaMalloc's implicit
 * synchronisation).
 *
 * Computes the R of the 6th-order step of idp_solve (IDP_STAGE_R) up to
 * rounding -- here by the direct stencil, where the plan-based solver forms R
 * in spectral form plus a correction next to the boundary:
 * R = sum over ordered axis pairs s != r of (h_s^4/240 + h_s^2 h_r^2/144)
 * D2_s D2_s D2_r u1 on the nodes whose indices all lie in 2..M-2, extended
 * to the layers next to the boundary by cubic extrapolation.
 *   d, n[d], h[d] : grid as in idp_create_plan (any n[s] >= 8, not only powers of two)
 *   u1            : device node array, prod(n) doubles (boundary values included)
 *   R             : device interior array, prod(n[s]-2) doubles; must not overlap u1
 * Scratch: a fixed device array of 3 * IDP_RHS6_NOALLOC_MAX_NODES doubles
 * (12 MiB), held by every GPU that loads the library until the process exits.
 * Problems with more than IDP_RHS6_NOALLOC_MAX_NODES nodes return IDP_ESCRATCH.
 * The call allocates nothing.  Every call looks up the scratch's device
 * address on the current device (cudaGetSymbolAddress; the host-side symbol is
 * not a device address); the first call on a device also loads the library's
 * device code there, so make that first call before any stream capture.
 * All calls share the one scratch array, which
 * keeps the last call's contents: calls whose work overlaps on the GPU (other
 * streams, other host threads) race and must be serialised by the caller. */
#define IDP_RHS6_NOALLOC_MAX_NODES 524288
int idp_rhs6_noalloc(int d, const int64_t n[], const double h[], const double *u1, double *R,
                     void *stream);

/* Static description of an IDP_* code. */
const char *idp_strerror(int code);

/* Name of the last CUDA error seen by the library in this thread ("" if none). */
const char *idp_last_cuda_error(void);

#ifdef __cplusplus
}
#endif
#endif /* IDP_H */
