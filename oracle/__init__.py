"""CPU oracle for the flexible shifted-Krylov solver (test infrastructure).

This package is a plain, slow, complex128 NumPy/SciPy statement of what the
GPU path computes. It exists only to check the GPU path: it may be imported by
the tests, by the smoke check and by the benchmark's CPU-baseline leg, and by
nothing else. The product path never calls it and shares no code with it.

Modules:
  operator   cell-centred finite-volume K and M (Section 5.1, Eq. phasor1)
  gmg        geometric-multigrid V-cycle inner solve (Section 4, Eq. zmmoditer)
  fgmres     flexible Arnoldi (Algorithm 3) + per-shift FGMRES/FFOM (Algorithm 4)
             with the inexact-preconditioning stopping bound (Eq. trueresidual)
  direct     exact inner solves (sparse LU, the paper's "Flexible" variant) and the
             per-shift direct comparator ("Direct", Section 6.1)
  csr        general sparse K, M and the BiCGSTAB-cycle inner solve (Section 6)
  amg        smoothed-aggregation AMG hierarchy and V-cycle, the preconditioner of
             the BiCGSTAB cycles in the paper's inner solver (Section 6)
  sensitivity  adjoint-state sensitivities of the phasor measurements (Section 5,
             Eq. sensitivity, Eq. adjoint, Algorithm 6)
"""
from .operator import assemble, GridOperator  # noqa: F401
from .gmg import Hierarchy  # noqa: F401
from .fgmres import shifted_solve, true_residuals, SolveResult  # noqa: F401
from .direct import ExactInner, direct_solve  # noqa: F401
from .csr import CSROperator, BiCGStabInner, csr_operator  # noqa: F401
