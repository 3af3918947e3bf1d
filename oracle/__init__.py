"""Plain FP64 CPU oracle for multigrid-preconditioned regularized least squares.

TEST INFRASTRUCTURE ONLY.  Nothing in the product path may import, call or
execute this package: only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` use it.  It shares no code with the CUDA
library (``paper_2306_11067_gb300``); both read the same seeded inputs from
``problemgen``.

What it computes (paper sections in brackets):
  * ``operators``   -- the discrete gradient L [Sec. 2, eq. (gradient)], the
                       normal-equations operator A^T A + lam^2 L^T D^2 L applied
                       in two stages [Sec. 3.2, eq. (normal)], diag(A^T A) as
                       column sums of squares [Sec. 3.2].
  * ``multigrid``   -- the V-cycle of Algorithm 1 on lam^2 L^T D^2 L + diag(A^T A)
                       with Galerkin coarse operators P^T K P and R = P^T
                       [Sec. 3.1], cell-centred bilinear P, l1-Jacobi smoothing,
                       a dense Cholesky solve on the coarsest level.
  * ``krylov``      -- preconditioned CG on the normal equations.
  * ``lcurve``      -- L-curve values, the corner, the weight update of eq. (g),
                       the lambda window and the outer stopping rule [Sec. 3.3,
                       3.4, 3.5, Algorithm 2].
  * ``outer``       -- Algorithm 2 end to end (sequential warm-start chain).
  * ``closed_forms``-- independent closed forms used to pin the above.

Every function is written for clarity, not speed: assembled scipy CSR
matrices, numpy vectors, FP64 throughout.

Parity pins: every function here is pinned by ``tests/test_oracle_*.py``
against closed forms, brute force or the paper's definitions; none is
"parity unpinned".
"""
from . import operators, multigrid, krylov, lcurve, outer, closed_forms  # noqa: F401
