"""CPU FP64 oracle for the doubly-periodic FCM mobility product M·[F;T] -> [U;Ω].

TEST INFRASTRUCTURE ONLY.  This package is a plain, slow, step-by-step restatement of the
method of Hashemi et al., "Computing hydrodynamic interactions in confined doubly-periodic
geometries in linear time" (Secs. II-III and Appendix A).  Only the test-suite, the smoke
check and the CPU-baseline leg of the benchmark may import it.  The product (the CUDA library
and its Python binding) never imports, calls or links anything here, and nothing here imports
the product: the two share no code.

Modules
-------
params   : problem description, Tables I/II kernel constants.
cheb     : Chebyshev grid, Clenshaw-Curtis weights, DCT-I, derivative/antiderivative.
kernel   : ES kernel (Eq. 54) with its normalisation, wall images (Eq. 9).
transfer : spreading (Eq. 7, step 1 of Sec. III.D) and interpolation (Eqs. 10-11, step 8).
bvp      : the per-wavenumber Chebyshev boundary-value problems (Eqs. 15-24) in the
           spectral-integration form, assembled densely and solved by LU.
stokes   : DP solve, wall corrections (Eqs. 41-44; Eqs. A4-A10), zero mode (Sec. III.C, App. A.2),
           curl, and the full mobility product.

Parity status of each function is stated in its docstring; every function is pinned by the
``-m "not gpu"`` tests in ``tests/test_oracle_*.py`` except where a docstring says
"parity unpinned".
"""

from .params import Params, table1, table2  # noqa: F401
from .stokes import mobility  # noqa: F401
