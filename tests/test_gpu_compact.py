"""16-bit column offsets of the one-column transposed SpMV pass
(params.compact_cols = 1, the default): the same arithmetic in the same order as the int32 indices,
so results are bitwise identical; a matrix with a row spanning more than
65,535 columns falls back to int32 indices.  The int32 path itself is
checked against the oracle by the parity tests, which run through the
compact path too (the default)."""
import numpy as np
import pytest
import scipy.sparse as sp

import problemgen as pg
from oracle import operators as ops
from oracle import krylov
from oracle import multigrid as mg
from paper_2306_11067_gb300 import Solver, lcmg as L

pytestmark = pytest.mark.gpu


def _solve(n_v, n_h, A, b, lams, **kw):
    s = Solver(n_v, n_h, mode=L.MODE_SEQUENTIAL, tol=1e-10, maxit=20000, **kw)
    s.set_forward_csr(A)
    out = s.solve(lams, b)
    s.close()
    return out


@pytest.mark.parametrize("precision", [L.PREC_MIXED, L.PREC_FP64])
def test_compact_columns_are_bitwise_identical(precision):
    P = pg.make_problem("ct256", size=48)
    lams = np.array([0.03, 0.3, 3.0])
    outs = [_solve(48, 48, P.A, P.b[:, 0], lams, precision=precision, compact_cols=cc) for cc in (1, 0)]
    for key in ("x", "rho", "eta", "iters", "status"):
        assert np.array_equal(outs[0][key], outs[1][key]), key


def test_wide_rows_fall_back_to_int32_columns():
    """A 256 x 264 image (67,584 pixels) with one row hitting the first and
    the last pixel: that row spans 67,583 columns, so the int32 indices are
    read; the solve agrees with the oracle."""
    n_v, n_h = 256, 264
    n = n_v * n_h
    rows = [sp.identity(n, format="csr") * 0.7]
    wide = sp.csr_matrix((np.array([1.0, 1.0]), (np.array([0, 0]), np.array([0, n - 1]))), shape=(1, n))
    M = sp.vstack(rows + [wide]).tocsr()
    M.sort_indices()
    A = pg.CSR(M.shape[0], n, M.indptr.astype(np.int64), M.indices.astype(np.int32), M.data.astype(np.float32))
    b = pg.rng(3).standard_normal(M.shape[0])
    lams = np.array([0.5])
    outs = [_solve(n_v, n_h, A, b, lams, precision=L.PREC_FP64, levels=4, compact_cols=cc) for cc in (1, 0)]
    assert np.array_equal(outs[0]["x"], outs[1]["x"])
    F = ops.ForwardCSR(M)
    Lg = ops.gradient(n_v, n_h)
    d = np.ones(ops.n_edges(n_v, n_h))
    H = mg.build_hierarchy(mg.weighted_laplacian(Lg, d), sp.diags(F.diag_AtA()), n_v, n_h, 4)
    c = ops.rhs(F, b)
    x, *_ = krylov.pcg(lambda v: ops.normal_apply(F, Lg, d, 0.5, v), c, None, mg.VCycle(H, 0.5), tol=1e-12,
                       maxit=5000)
    assert np.linalg.norm(outs[0]["x"][0, 0] - x) <= 1e-7 * np.linalg.norm(x)


@pytest.mark.parametrize("precision,bound", [(L.PREC_FP64, 1e-8), (L.PREC_MIXED, 1e-6)])
def test_scalars_inside_the_updates_match_the_scalar_kernels(precision, bound):
    """One column: alpha and beta taken by every block of the x/r and p
    updates (alpha_fuse = beta_fuse = 1, the default), alpha only, or both
    by the scalar kernels, sum in different orders; every form solves to
    the oracle's solution (reliable updates and restarts included at
    tol 1e-12) in about the same number of iterations."""
    P = pg.make_problem("ct256", size=48)
    lams = np.array([0.05, 0.5])
    outs = []
    for af, bf in ((1, 1), (1, 0), (0, 0)):
        s = Solver(48, 48, mode=L.MODE_SEQUENTIAL, tol=1e-12, maxit=20000, precision=precision, alpha_fuse=af,
                   beta_fuse=bf)
        s.set_forward_csr(P.A)
        outs.append(s.solve(lams, P.b[:, 0]))
        s.close()
    F = ops.ForwardCSR(P.A.to_scipy())
    Lg = ops.gradient(48, 48)
    d = np.ones(ops.n_edges(48, 48))
    H = mg.build_hierarchy(mg.weighted_laplacian(Lg, d), sp.diags(F.diag_AtA()), 48, 48, 3)
    c = ops.rhs(F, P.b[:, 0])
    for j, lam in enumerate(lams):
        x, *_ = krylov.pcg(lambda v: ops.normal_apply(F, Lg, d, lam, v), c, None, mg.VCycle(H, lam), tol=1e-12,
                           maxit=20000)
        ref_its = int(outs[-1]["iters"][0, j])
        for out in outs:
            assert out["status"][0, j] == 0
            assert np.linalg.norm(out["x"][0, j] - x) <= bound * np.linalg.norm(x)
            assert abs(int(out["iters"][0, j]) - ref_its) <= max(3, 0.05 * ref_its)


@pytest.mark.parametrize("fuse", [0, 1])
def test_iteration_limit_with_scalars_inside_the_updates(fuse):
    """The fused beta step takes the iteration-limit decision as the scalar
    kernel does: status MAXIT after exactly maxit iterations."""
    P = pg.make_problem("ct256", size=48)
    s = Solver(48, 48, mode=L.MODE_SEQUENTIAL, tol=1e-14, maxit=7, precision=L.PREC_MIXED, alpha_fuse=fuse,
               beta_fuse=fuse)
    s.set_forward_csr(P.A)
    out = s.solve([1e-3], P.b[:, 0])
    s.close()
    assert out["status"][0, 0] == L.MAXIT
    assert int(out["iters"][0, 0]) == 7
