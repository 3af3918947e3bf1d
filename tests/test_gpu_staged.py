"""The shared-memory-staged CSR SpMM (params.staged = 1) against the oracle.

The staged kernel cuts the rows of A and A^T into chunks of at most 2048
nonzeros and 32 rows, copies each chunk into shared memory with bulk
asynchronous copies and computes from there; a row longer than 2048
nonzeros is read from global memory directly.  These tests drive every
mode of the operator passes (A p; A^T y + lam2 L^T W L p with its dot
product; the true residual; ||A x - b||) through it, on the CT matrix and on
a ragged matrix that has empty rows, a 2304-nonzero row of A, a 2100-nonzero
row of A^T and runs of one-nonzero rows longer than a chunk's row limit.
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


def _ragged(N, dtype):
    """CT rows of an N x N image, interleaved with empty rows, one dense row
    (N^2 > 2048 nonzeros) and 2100 rows hitting pixel 0 only."""
    P = pg.make_problem("ct256", size=N)
    A = P.A.to_scipy()
    n = P.n
    r = pg.rng(11)
    dense = sp.csr_matrix(r.uniform(0.1, 1.0, (1, n)))
    k = 2100
    single = sp.csr_matrix((r.uniform(0.5, 1.5, k), (np.arange(k), np.zeros(k, dtype=np.int64))), shape=(k, n))
    empty = sp.csr_matrix((7, n))
    M = sp.vstack([A[:100], empty, dense, A[100:], single, empty]).tocsr()
    M.sort_indices()
    return P, pg.CSR(M.shape[0], n, M.indptr.astype(np.int64), M.indices.astype(np.int32), M.data.astype(dtype))


def _matrix(kind):
    if kind == "ct":
        P = pg.make_problem("ct256", size=48)
        return P, P.A
    return _ragged(48, np.float32 if kind == "ragged32" else np.float64)


@pytest.mark.parametrize("kind", ["ct", "ragged32", "ragged64"])
@pytest.mark.parametrize("ncols", [1, 2, 3, 8, 13, 20, 33, 70])
def test_staged_normal_apply_matches_oracle(kind, ncols):
    """K x through both operator passes (FP64 vectors), every lane split of
    the batch width, including widths above one launch's 64 columns."""
    P, A = _matrix(kind)
    d = pg.random_weights(ops.n_edges(P.n_v, P.n_h), 2)
    lams = np.geomspace(1e-3, 5.0, ncols)
    X = pg.rng(3).standard_normal((ncols, P.n))
    F = ops.ForwardCSR(A.to_scipy())
    Lg = ops.gradient(P.n_v, P.n_h)
    outs = []
    for staged in (1, 0):
        s = Solver(P.n_v, P.n_h, staged=staged)
        s.set_forward_csr(A)
        s.set_weights(d)
        xd = torch.tensor(X, device="cuda", dtype=torch.float64)
        yd = torch.empty_like(xd)
        L.lcmg_apply_normal_dev(s.ctx, lams, xd, yd)
        outs.append(yd.cpu().numpy())
        s.close()
    for j, lam in enumerate(lams):
        ref = ops.normal_apply(F, Lg, d, lam, X[j])
        assert _rel(outs[0][j], ref) <= 1e-13
        # the two kernels differ only in summation order
        assert _rel(outs[0][j], outs[1][j]) <= 1e-13


@pytest.mark.parametrize("kind", ["ct", "ragged32"])
@pytest.mark.parametrize("precision", [L.PREC_FP64, L.PREC_MIXED])
@pytest.mark.parametrize("nlam", [1, 3])
def test_staged_solve_matches_oracle(kind, precision, nlam):
    """PCG through the staged passes reaches the oracle's solution, and the
    reported ||A x - b|| (the rho pass) is the oracle's for that x."""
    P, A = _matrix(kind)
    if kind != "ct":
        xt = pg.phantom_ellipses(P.n_v, P.n_h, 10, 5).ravel(order="F")
        b = A.to_scipy() @ xt
        b = pg.add_noise(b, 0.01, 6)
    else:
        b = P.b[:, 0]
    lams = np.array([0.05, 0.4, 2.0])[:nlam]
    d = pg.random_weights(ops.n_edges(P.n_v, P.n_h), 4, d_min=0.05)
    s = Solver(P.n_v, P.n_h, levels=3, staged=1, precision=precision, tol=1e-12, maxit=20000)
    s.set_forward_csr(A)
    s.set_weights(d)
    out = s.solve(lams, b)
    s.close()
    F = ops.ForwardCSR(A.to_scipy())
    Lg = ops.gradient(P.n_v, P.n_h)
    H = mg.build_hierarchy(mg.weighted_laplacian(Lg, d), sp.diags(F.diag_AtA()), P.n_v, P.n_h, 3)
    c = ops.rhs(F, b)
    bound = 1e-8 if precision == L.PREC_FP64 else 1e-6
    for j, lam in enumerate(lams):
        x, *_ = krylov.pcg(lambda v: ops.normal_apply(F, Lg, d, lam, v), c, None, mg.VCycle(H, lam),
                           tol=1e-12, maxit=20000)
        assert out["status"][0, j] == 0
        xg = out["x"][0, j]
        assert _rel(xg, x) <= bound
        rho_ref = np.linalg.norm(F.matvec(xg) - b)
        assert abs(out["rho"][0, j] - rho_ref) <= 1e-12 * rho_ref


def test_staged_lcurve_run_matches_direct():
    """A short Algorithm 2 run (the warm-start chain) picks the same corners
    with the staged and the direct passes."""
    P = pg.make_problem("ct256", size=48)
    lams = np.logspace(-3, 0, 8)
    hist = []
    for staged in (1, 0):
        s = Solver(P.n_v, P.n_h, levels=3, staged=staged, precision=L.PREC_MIXED, mode=L.MODE_SEQUENTIAL,
                   tol=1e-6)
        s.set_forward_csr(P.A)
        r = s.lcurve_run(lams, P.b[:, 0], max_outer=3)
        hist.append(list(r["history"]))
        s.close()
    assert hist[0] == hist[1]
