"""GB300-native infinite-domain Poisson solver (arXiv 2108.11871).

phi = G * rho at every node of a uniform 2-D/3-D grid, computed as the
Dirichlet sine-transform solve phi* plus a 4th/6th-order harmonic correction
whose boundary values come from FFT convolutions (sections 2-5).  All work
runs in the CUDA library ``libidp.so`` (C ABI in ``include/idp.h``); this
package only marshals arguments to it.
"""
from .binding import (  # noqa: F401
    IDP_OK, IDP_EINVAL, IDP_ENOMEM, IDP_ECUDA, IDP_EALIAS, IDP_ESUPPORT, IDP_ESCRATCH, IDP_EGUARD,
    IDP_RHS6_NOALLOC_MAX_NODES, rhs6_noalloc,
    IDP_STAGE_BOUNDARY, IDP_STAGE_GTILDE, IDP_STAGE_PHISTAR, IDP_STAGE_U1,
    IDP_STAGE_R, IDP_STAGE_PHI, IDP_KEY_USE_GRAPH, IDP_KEY_PRECISION, IDP_KEY_STALL_TEST, IDP_KEY_AUTOTUNE, IDP_KEY_DST_SHAPE, IDP_KEY_VALIDATE,
    IDP_KEY_GUARD_TEST, IDP_KEY_MIXED_BOUNDARY_DF32, IDP_KEY_NVTX,
    IDP_PRECISION_FP64,
    IDP_PRECISION_MIXED_BF16X3, IDP_PRECISION_DF32, IDP_PRECISION_MIXED_TF32X3, IDP_ETIMEOUT, IdpError, Plan, create_plan,
    destroy_plan, library, plan_check_guards, plan_grid, plan_info, plan_set, plan_tuning, plan_status, solve, solve_batched,
    solve_host, solve_stage, strerror,
)
