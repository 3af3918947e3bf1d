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
  * ``paper_mg``    -- the paper's own cycle: one-sided hierarchies
                       A_{k+1} = A_k P_k, M_{k+1} = M_k P_k, diagonally
                       preconditioned CG relaxation, V(2,1), flexible GMRES
                       [Sec. 3.2, 3.3].
  * ``amg``         -- classical AMG coarsening of L^T D^2 L: strength,
                       two-pass C/F split, interpolation [Sec. 3.1].
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
from . import operators, multigrid, krylov, lcurve, outer, closed_forms, paper_mg, amg  # noqa: F401
