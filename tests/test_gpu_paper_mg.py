"""The paper's own method on the GPU (params.precond = 1): the V(2,1) cycle on
the whole normal operator with one-sided coarse operators and CG
relaxation, and FGMRES, against the oracle's version (oracle.paper_mg)."""
import numpy as np
import pytest
import torch

import problemgen as pg
from oracle import operators as ops
from oracle import paper_mg as pm
from oracle import krylov
from paper_2306_11067_gb300 import Solver, LcmgError, lcmg as L

pytestmark = pytest.mark.gpu


def _rel(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


class _Grid:
    def __init__(self, n_v, n_h, b=None):
        self.n_v, self.n_h, self.b = n_v, n_h, b


def _problem(kind):
    if kind == "blur":
        P = pg.make_problem("deblur32_csr")
        return P, P.A
    if kind == "blur40x24":
        return _Grid(40, 24), pg.blur_csr(40, 24, pg.gaussian_psf(2, 1.0))
    P = pg.make_problem("ct256", size=32)
    return P, P.A


@pytest.mark.parametrize("kind,levels", [("blur", 3), ("blur40x24", 3), ("ct", 2), ("ct", 3)])
def test_paper_cycle_matches_oracle(kind, levels):
    P, A = _problem(kind)
    n_v, n_h = P.n_v, P.n_h
    d = pg.random_weights(ops.n_edges(n_v, n_h), 6, d_min=0.05)
    s = Solver(n_v, n_h, levels=levels, precond=1)
    s.set_forward_csr(A)
    s.set_weights(d)
    lams = np.array([1e-2, 0.3, 3.0])
    R = pg.rng(5).standard_normal((3, n_v * n_h))
    rd = torch.tensor(R, device="cuda", dtype=torch.float64)
    zd = torch.empty_like(rd)
    L.lcmg_apply_vcycle_dev(s.ctx, lams, rd, zd)
    s.close()
    h = pm.build_one_sided(A.to_scipy(), ops.gradient(n_v, n_h), d, n_v, n_h, levels)
    for j, lam in enumerate(lams):
        ref = pm.PaperVCycle(h, lam)(R[j])
        assert _rel(zd[j].cpu().numpy(), ref) <= 1e-10, (lam, _rel(zd[j].cpu().numpy(), ref))


@pytest.mark.parametrize("kind,levels", [("blur", 3), ("ct", 3)])
@pytest.mark.parametrize("restart", [200, 7])
def test_paper_fgmres_solve_matches_oracle(kind, levels, restart):
    """To 1e-12 where FP64 FGMRES reaches it (at small lambda its residual
    stalls near 1e-9: the update x0 + Z y carries the rounding of the
    strongly amplifying preconditioner).  Iteration counts are compared at
    1e-8 (next test): this close to the floor they depend on when the true
    residual check restarts the iteration."""
    P, A = _problem(kind)
    n_v, n_h = P.n_v, P.n_h
    d = pg.random_weights(ops.n_edges(n_v, n_h), 7, d_min=0.05)
    lams = np.array([0.2, 0.5, 2.0])
    # every lambda from zero, as the oracle solves it
    s = Solver(n_v, n_h, levels=levels, precond=1, tol=1e-12, maxit=2000, gmres_restart=restart,
               mode=L.MODE_BATCHED)
    s.set_forward_csr(A)
    s.set_weights(d)
    out = s.solve(lams, P.b[:, 0])
    s.close()
    F = ops.ForwardCSR(A.to_scipy())
    Lg = ops.gradient(n_v, n_h)
    c = ops.rhs(F, P.b[:, 0])
    for j, lam in enumerate(lams):
        x, it, st, _ = pm.solve(F, Lg, d, n_v, n_h, levels, c, lam, tol=1e-12, maxit=2000, restart=restart)
        assert st == krylov.CONVERGED and out["status"][0, j] == 0
        assert _rel(out["x"][0, j], x) <= 1e-8
        rho = np.linalg.norm(F.matvec(out["x"][0, j]) - P.b[:, 0])
        assert abs(out["rho"][0, j] - rho) <= 1e-10 * rho


@pytest.mark.parametrize("lam", [1e-2, 0.05, 0.2, 2.0])
def test_paper_fgmres_iterations_and_lcurve_values(lam):
    """Without restarts (the paper's setting), at the paper's tolerance 1e-6
    both sides take the same number of FGMRES steps within 10%; the oracle
    orthogonalises as the GPU does (classical Gram-Schmidt twice): at
    lambda = 0.01 the count moves by ~10% with the Gram-Schmidt variant and
    even with the summation order of the dot products.  At 1e-8 the
    GPU solution meets the tolerance on the oracle's own normal-equation
    residual, and for lambda >= 0.2 its L-curve values are the oracle's
    within 1e-6.  Below, 1e-8 is within a few times of the FP64 residual
    floor and two solutions that both meet it differ in the seminorm by
    4e-6 (lambda = 0.05) to 4e-5 (0.01) relative, so only the residual is
    compared there."""
    P, A = _problem("ct")
    d = np.ones(ops.n_edges(32, 32))
    F = ops.ForwardCSR(A.to_scipy())
    Lg = ops.gradient(32, 32)
    c = ops.rhs(F, P.b[:, 0])
    out = {}
    for tol in (1e-6, 1e-8):
        s = Solver(32, 32, levels=3, precond=1, tol=tol, maxit=2000, gmres_restart=2000)
        s.set_forward_csr(A)
        out[tol] = s.solve([lam], P.b[:, 0])
        s.close()
        assert out[tol]["status"][0, 0] == 0
    _, it, st, _ = pm.solve(F, Lg, d, 32, 32, 3, c, lam, tol=1e-6, maxit=2000, restart=2000, orth="cgs2")
    assert st == krylov.CONVERGED
    gi = int(out[1e-6]["iters"][0, 0])
    assert abs(gi - it) <= max(3, 0.1 * it), (gi, it)
    xg = out[1e-8]["x"][0, 0]
    assert np.linalg.norm(c - ops.normal_apply(F, Lg, d, lam, xg)) <= 1.01e-8 * np.linalg.norm(c)
    if lam < 0.2:
        return
    x, _, st, _ = pm.solve(F, Lg, d, 32, 32, 3, c, lam, tol=1e-8, maxit=2000, restart=2000)
    assert st == krylov.CONVERGED
    rho_ref = np.linalg.norm(F.matvec(x) - P.b[:, 0])
    eta_ref = np.linalg.norm(Lg @ x)
    assert abs(out[1e-8]["rho"][0, 0] - rho_ref) <= 1e-6 * rho_ref
    assert abs(out[1e-8]["eta"][0, 0] - eta_ref) <= 1e-6 * eta_ref


def test_paper_method_selects_the_same_corners():
    """Algorithm 2 with the paper's solver and with the default one, both to
    1e-9 (reachable by FP64 FGMRES for lambda >= 0.03): the same selections."""
    P = pg.make_problem("ct256", size=32)
    lams = np.logspace(-1.5, 0.5, 10)
    hist = []
    for precond in (0, 1):
        s = Solver(32, 32, levels=2, precond=precond, tol=1e-9, maxit=20000, mode=L.MODE_SEQUENTIAL)
        s.set_forward_csr(P.A)
        r = s.lcurve_run(lams, P.b[:, 0], max_outer=3)
        hist.append([int(h) for h in r["history"]])
        s.close()
    assert hist[0] == hist[1]


def test_paper_method_argument_errors():
    P = pg.make_problem("ct256", size=32)
    s = Solver(32, 32, levels=2, precond=1, precision=L.PREC_MIXED)
    s.set_forward_csr(P.A)
    with pytest.raises(LcmgError):
        s.solve([0.1], P.b[:, 0])
    s.close()
    Q = pg.make_problem("deblur512", size=32, n_rhs=1)
    s = Solver(32, 32, levels=2, precond=1)
    s.set_forward_stencil(Q.psf)
    with pytest.raises(LcmgError):
        s.solve([0.1], Q.b[:, 0])
    s.close()


@pytest.mark.parametrize("coarsening", [0, 1])
def test_paper_cycle_graph_is_bitwise_the_launched_cycle(coarsening):
    """With params.graphs the FGMRES loop replays the cycle as one captured
    CUDA graph: the same kernels in the same order, so the same bits."""
    P, A = _problem("ct")
    d = pg.random_weights(ops.n_edges(32, 32), 3, d_min=0.05)
    outs = []
    for graphs in (1, 0):
        s = Solver(32, 32, levels=3, precond=1, coarsening=coarsening, graphs=graphs, tol=1e-10, maxit=500)
        s.set_forward_csr(A)
        s.set_weights(d)
        outs.append(s.solve([0.05, 0.5], P.b[:, 0]))
        s.close()
    for key in ("x", "rho", "eta", "iters", "status"):
        assert np.array_equal(outs[0][key], outs[1][key]), key
