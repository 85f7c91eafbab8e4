"""Plain FP64 CPU oracle for the infinite-domain Poisson method (arXiv 2108.11871).

TEST INFRASTRUCTURE ONLY.  Only the test suite, ``__graft_entry__.smoke()`` and
the CPU-baseline leg of ``bench.py`` may import or run anything in this
package.  The CUDA library never calls it, and it shares no code with the
CUDA path.

Each function follows one passage of the paper and is written for checking by
eye, not for speed: sine transforms are direct O(n^2) sums (a matrix product
with the sine matrix along each axis), stencils are written out with array
slices, and the boundary potential is either the direct trapezoid sum
(eq. TrapOrig2D, in C with compensated summation) or its convolution
rearrangement (eqs. Trap2D and convolution) with numpy's FFT as the
convolution primitive.

Modules
  dst          -- sine matrices, eigenvalues, the spectral Dirichlet solve (section 3)
  greens       -- Green's function and boundary values g (section 4)
  harmonic     -- 4th/6th-order harmonic correction (section 5)
  solve        -- phi = phi* + phi_H (section 2)
  closed_form  -- exact radial potentials of the bump densities (section 6)

Parity pins: every function is pinned by tests in ``tests/test_oracle_*.py``
against closed forms, identities or brute force; none is "parity unpinned".
"""
from . import dst, greens, harmonic, solve, closed_form  # noqa: F401
