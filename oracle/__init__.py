"""CPU oracle for generalized approximate deconvolution (San & Vedula,
"Generalized deconvolution procedure for structural modeling of turbulence").

TEST INFRASTRUCTURE ONLY. This package is a plain, slow, float64 NumPy
restatement of the paper's operator and algorithms. It exists to check the
CUDA library; only the tests, the smoke check and the benchmark's CPU
baseline may import it. The library never calls it and it never calls the
library.

Contents
  spectral.py  -- the Germano elliptic differential filter G (Eq. df, Eq. df2)
                  and its exact Fourier inverse.
  solvers.py   -- Van Cittert (Algorithm 1), steepest descent (Algorithm 2),
                  conjugate gradient (Algorithm 3) and BiCGSTAB (Algorithm 4)
                  for G u = u_bar (Eq. tau3), with the stopping and
                  breakdown rules stated in solvers.py.
  precond.py   -- preconditioned CG with a periodic finite-difference
                  approximation of G^{-1} (no counterpart in the paper).

Parity status: every function here is pinned by the tests under
tests/test_oracle_*.py (closed forms, hand-computed transfer values,
finite-difference residuals, exact rational first iterates, Krylov
invariants); none is "parity unpinned".
"""

from .spectral import (  # noqa: F401
    wavenumber_grid,
    cutoff_wavenumber,
    transfer_function,
    filter_field,
    exact_inverse,
)
from .solvers import (  # noqa: F401
    SolveResult,
    van_cittert,
    steepest_descent,
    conjugate_gradient,
    bicgstab,
    solve,
    inner,
    STATUS_OK,
    STATUS_MAXIT,
    STATUS_BREAKDOWN,
    STATUS_NONFINITE,
)
from .precond import (  # noqa: F401
    stencil_coefficients,
    apply_preconditioner,
    apply_preconditioner_f32,
    preconditioner_symbol,
    preconditioned_cg,
)
