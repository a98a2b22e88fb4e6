"""CPU oracle for the Zernike basis / series path.

TEST INFRASTRUCTURE ONLY.  Nothing in the product path may import, call or execute this
package: only the tests, the smoke check and the benchmark's CPU-baseline leg (and its
`--impl reference` arm) use it.  It shares no code, table or constant with the CUDA
library: the oracle evaluates the explicit factorial sum of the radial polynomial in exact
rational arithmetic (paper Sec. 2, the radial-part sum and its binomial form), while the
library walks the Jacobi three-term recursion on the GPU.

Modules:
  radial  -- exact integer coefficients and exact-rational R_n^m(rho) and d^k/drho^k R
  trig    -- cos/sin(m*theta) in big-integer fixed point (no mpmath dependency)
  basis   -- Z_n^m and its rho / theta derivatives, rounded once to float64
  series  -- series F = Z C and its adjoint, exact sums over the rounded basis
  fit     -- weighted least-squares coefficients (normal equations)
"""
from . import radial, trig, basis, series, fit  # noqa: F401
