"""The two-kernels-per-level V-cycle (params.vfuse = 2: always) against the oracle.

Each level runs as a down kernel (pre-smoothing from zero, residual,
restriction) and an up kernel (prolongation, post-smoothing) over 8 x 8
coarse-point tiles with their stencil halos in shared memory.  The grids
below span several tiles with ragged last tiles (coarse sides 20, 12, 36,
28, 5) and both stencils (the 5-point finest level, the 25-point Galerkin
levels); nu = 1 and 2, both smoothers.
"""
import numpy as np
import pytest
import scipy.sparse as sp
import torch

import problemgen as pg
from oracle import operators as ops
from oracle import multigrid as mg
from oracle import krylov
from paper_2306_11067_gb300 import Solver, lcmg as L

pytestmark = pytest.mark.gpu


def _rel(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


@pytest.mark.parametrize("smoother", [L.SMOOTH_L1_JACOBI, L.SMOOTH_JACOBI])
@pytest.mark.parametrize("n_v,n_h,levels", [(32, 32, 3), (40, 24, 3), (72, 56, 4), (10, 10, 2), (16, 64, 4)])
@pytest.mark.parametrize("nu", [1, 2])
@pytest.mark.parametrize("precision", [L.PREC_FP64, L.PREC_MIXED])
def test_vfused_vcycle_matches_oracle(smoother, n_v, n_h, levels, nu, precision):
    A = pg.blur_csr(n_v, n_h, pg.gaussian_psf(2, 1.0))
    s = Solver(n_v, n_h, levels=levels, smoother=smoother, nu=nu, vfuse=2, precision=precision)
    s.set_forward_csr(A)
    d = pg.random_weights(ops.n_edges(n_v, n_h), 9)
    s.set_weights(d)
    lams = np.array([1e-3, 0.1, 10.0])
    R = pg.rng(4).standard_normal((3, n_v * n_h))
    rd = torch.tensor(R, device="cuda", dtype=torch.float64)
    zd = torch.empty_like(rd)
    L.lcmg_apply_vcycle_dev(s.ctx, lams, rd, zd)
    s.close()
    F = ops.ForwardCSR(A.to_scipy())
    Lg = ops.gradient(n_v, n_h)
    H = mg.build_hierarchy(mg.weighted_laplacian(Lg, d), sp.diags(F.diag_AtA()), n_v, n_h, levels)
    sm = "l1" if smoother == L.SMOOTH_L1_JACOBI else "jacobi"
    # FP32 V-cycle: a few hundred roundings of unit size per level
    bound = 1e-12 if precision == L.PREC_FP64 else 1e-5
    for j, lam in enumerate(lams):
        ref = mg.VCycle(H, lam, nu=nu, smoother=sm)(R[j])
        assert _rel(zd[j].cpu().numpy(), ref) <= bound, (lam, _rel(zd[j].cpu().numpy(), ref))


def test_vfused_matches_per_step_kernels():
    """Same V-cycle through both paths on a 256 x 256 grid (5 levels, the
    benchmark hierarchy): FP64 results agree to rounding."""
    n = 256
    A = sp.identity(n * n, format="csr") * 0.5
    Acsr = pg.CSR(n * n, n * n, A.indptr.astype(np.int64), A.indices.astype(np.int32), A.data.astype(np.float64))
    d = pg.random_weights(ops.n_edges(n, n), 12, d_min=0.05)
    lams = np.array([0.01, 1.0])
    R = pg.rng(8).standard_normal((2, n * n))
    out = []
    for vf in (0, 2):
        s = Solver(n, n, vfuse=vf)
        s.set_forward_csr(Acsr)
        s.set_weights(d)
        assert L.lcmg_num_levels(s.ctx) == 5
        rd = torch.tensor(R, device="cuda", dtype=torch.float64)
        zd = torch.empty_like(rd)
        L.lcmg_apply_vcycle_dev(s.ctx, lams, rd, zd)
        out.append(zd.cpu().numpy())
        s.close()
    for j in range(2):
        assert _rel(out[1][j], out[0][j]) <= 1e-13


@pytest.mark.parametrize("precision,bound", [(L.PREC_FP64, 1e-8), (L.PREC_MIXED, 1e-6)])
@pytest.mark.parametrize("nlam", [1, 3, 20])
def test_vfused_ct_solve_matches_oracle(precision, bound, nlam):
    """PCG with the fused V-cycle on the CT matrix reaches the oracle's
    solution; the level-0 up kernel supplies the r.z partials."""
    N = 48
    P = pg.make_problem("ct256", size=N)
    d = pg.random_weights(ops.n_edges(N, N), 5, d_min=0.05)
    lams = np.geomspace(0.02, 5.0, nlam) if nlam > 1 else np.array([0.2])
    # every lambda from zero, as the oracle solves it (the chain's warm starts
    # would add a forward error of up to cond(K) x 1e-12 between the two)
    # FP64: both sides to 1e-13, so that their forward errors (up to
    # cond(K) x tol each, cond ~ 1e5 at lambda = 0.02) stay well inside 1e-8
    tol = 1e-13 if precision == L.PREC_FP64 else 1e-12
    s = Solver(N, N, levels=4, vfuse=2, precision=precision, tol=tol, maxit=20000, mode=L.MODE_BATCHED)
    s.set_forward_csr(P.A)
    s.set_weights(d)
    out = s.solve(lams, P.b[:, 0])
    s.close()
    F = ops.ForwardCSR(P.A.to_scipy())
    Lg = ops.gradient(N, N)
    H = mg.build_hierarchy(mg.weighted_laplacian(Lg, d), sp.diags(F.diag_AtA()), N, N, 4)
    c = ops.rhs(F, P.b[:, 0])
    for j in range(0, nlam, max(1, nlam // 4)):
        lam = lams[j]
        x, *_ = krylov.pcg(lambda v: ops.normal_apply(F, Lg, d, lam, v), c, None, mg.VCycle(H, lam),
                           tol=tol, maxit=20000)
        assert out["status"][0, j] == 0
        assert _rel(out["x"][0, j], x) <= bound
