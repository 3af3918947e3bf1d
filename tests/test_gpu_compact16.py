"""FP16 smoother data (params.smoother_fp16, the default for mixed-precision
batches whose columns share one lambda) against the oracle's model of the
same storage (oracle.multigrid, storage="fp16"), and the FP32 form of the
same batches against the exact cycle.

A cycle agrees with its model to FP32 rounding (1e-5, as the FP32 cycle
with the exact one); PCG with the rounded cycle reaches the oracle's exact
solution (1e-6), since the preconditioner does not change the system.
"""
import functools

import numpy as np
import pytest
import scipy.sparse as sp

import problemgen as pg
from oracle import operators as ops
from oracle import multigrid as mg
from oracle import krylov

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2306_11067_gb300 import lcmg as L  # noqa: E402
from paper_2306_11067_gb300 import Solver  # noqa: E402


def _rel(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


@pytest.mark.parametrize("n_v,n_h,levels", [(32, 32, 3), (40, 24, 3), (72, 56, 4), (16, 64, 4), (96, 96, 5)])
@pytest.mark.parametrize("nu", [1, 2])
@pytest.mark.parametrize("smoother", [L.SMOOTH_L1_JACOBI, L.SMOOTH_JACOBI])
@pytest.mark.parametrize("fp16", [1, 0])
def test_one_lambda_cycle_matches_its_model(n_v, n_h, levels, nu, smoother, fp16):
    A = pg.blur_csr(n_v, n_h, pg.gaussian_psf(2, 1.0))
    s = Solver(n_v, n_h, levels=levels, smoother=smoother, nu=nu, precision=L.PREC_MIXED, smoother_fp16=fp16)
    s.set_forward_csr(A)
    d = pg.random_weights(ops.n_edges(n_v, n_h), 9, d_min=0.02)
    s.set_weights(d)
    R = pg.rng(4).standard_normal((1, n_v * n_h))
    rd = torch.tensor(R, device="cuda", dtype=torch.float64)
    F = ops.ForwardCSR(A.to_scipy())
    Lg = ops.gradient(n_v, n_h)
    H = mg.build_hierarchy(mg.weighted_laplacian(Lg, d), sp.diags(F.diag_AtA()), n_v, n_h, levels)
    sm = "l1" if smoother == L.SMOOTH_L1_JACOBI else "jacobi"
    for lam in (1e-3, 0.1, 10.0):
        zd = torch.empty_like(rd)
        L.lcmg_apply_vcycle_dev(s.ctx, np.array([lam]), rd, zd)
        ref = mg.VCycle(H, lam, nu=nu, smoother=sm, storage="fp16" if fp16 else "fp64")(R[0])
        assert _rel(zd[0].cpu().numpy(), ref) <= 1e-5, (lam, _rel(zd[0].cpu().numpy(), ref))
    s.close()


def test_fp16_cycle_differs_from_the_exact_one():
    """The model is not the exact cycle: the FP16 rounding is visible (so
    the test above would fail against the exact cycle), and small."""
    n = 64
    A = pg.blur_csr(n, n, pg.gaussian_psf(2, 1.0))
    s = Solver(n, n, levels=4, precision=L.PREC_MIXED)
    s.set_forward_csr(A)
    d = pg.random_weights(ops.n_edges(n, n), 9, d_min=0.02)
    s.set_weights(d)
    r = pg.rng(4).standard_normal(n * n)
    rd = torch.tensor(r, device="cuda", dtype=torch.float64).reshape(1, -1)
    zd = torch.empty_like(rd)
    L.lcmg_apply_vcycle_dev(s.ctx, np.array([1e-3]), rd, zd)
    s.close()
    F = ops.ForwardCSR(A.to_scipy())
    H = mg.build_hierarchy(mg.weighted_laplacian(ops.gradient(n, n), d), sp.diags(F.diag_AtA()), n, n, 4)
    exact = mg.VCycle(H, 1e-3, nu=1)(r)
    e = _rel(zd[0].cpu().numpy(), exact)
    assert 1e-5 < e < 1e-2, e


@functools.lru_cache(maxsize=None)
def _chain_case(kind, nrhs):
    if kind == "ct":
        N = 48
        P = pg.make_problem("ct256", size=N)
        imgs = [pg.phantom_ellipses(N, N, 6, 40 + r) for r in range(nrhs)]
        B = np.stack([P.A.to_scipy() @ pg.vec(im) for im in imgs], 1)
        F = ops.ForwardCSR(P.A.to_scipy())
        fwd = P.A
    else:
        N = 64
        fwd = pg.gaussian_psf(6, 2.0)
        imgs = [pg.phantom_mixed(N, N, 6, 40 + r) for r in range(nrhs)]
        B = np.stack([pg.vec(pg.blur_apply(im, fwd)) for im in imgs], 1)
        F = ops.ForwardPSF(fwd, N, N)
    B = B + 0.01 * pg.rng(3).standard_normal(B.shape) * np.abs(B).max()
    d = pg.random_weights(ops.n_edges(N, N), 5, d_min=0.05)
    lams = (0.05, 0.3)
    Lg = ops.gradient(N, N)
    H = mg.build_hierarchy(mg.weighted_laplacian(Lg, d), sp.diags(F.diag_AtA()), N, N, mg.default_levels(N, N))
    ref = np.zeros((nrhs, len(lams), N * N))
    for r in range(nrhs):
        c = ops.rhs(F, B[:, r])
        for j, lam in enumerate(lams):
            ref[r, j], *_ = krylov.pcg(lambda v: ops.normal_apply(F, Lg, d, lam, v), c, None,
                                       mg.VCycle(H, lam, nu=1), tol=1e-12, maxit=20000)
    return N, fwd, B, d, np.array(lams), ref


@pytest.mark.parametrize("kind", ["ct", "separable"])
@pytest.mark.parametrize("nrhs", [1, 3])
def test_solves_with_fp16_smoother_reach_oracle(kind, nrhs):
    """The chain (one column per lambda) and its right-hand-side batches
    (columns sharing lambda) both use the FP16 smoother data."""
    N, fwd, B, d, lams, ref = _chain_case(kind, nrhs)
    s = Solver(N, N, precision=L.PREC_MIXED, mode=L.MODE_SEQUENTIAL, tol=1e-12, maxit=20000)
    if kind == "ct":
        s.set_forward_csr(fwd)
    else:
        s.set_forward_stencil(fwd)
    s.set_weights(d)
    out = s.solve(lams, B.T)
    s.close()
    for r in range(nrhs):
        for j, lam in enumerate(lams):
            assert out["status"][r, j] == 0
            assert _rel(out["x"][r, j], ref[r, j]) <= 1e-6, (r, lam, _rel(out["x"][r, j], ref[r, j]))
