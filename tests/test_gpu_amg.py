"""The paper's method with classical AMG coarsening (params.precond = 1,
coarsening = 1) on the GPU against the oracle (oracle.paper_mg with
oracle.amg): level sizes, one V(2,1) cycle, FGMRES solutions and step
counts, the rebuild when D changes, and Algorithm 2's selections."""
import numpy as np
import pytest
import torch

import problemgen as pg
from oracle import amg
from oracle import operators as ops
from oracle import multigrid as mg
from oracle import paper_mg as pm
from oracle import krylov
from paper_2306_11067_gb300 import Solver, lcmg as L

pytestmark = pytest.mark.gpu


def _rel(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def _problem(kind):
    if kind == "blur":
        P = pg.make_problem("deblur32_csr")
        return 32, 32, P.A, P.b[:, 0]
    if kind == "blur40x24":
        A = pg.blur_csr(40, 24, pg.gaussian_psf(2, 1.0))
        b = pg.rng(3).standard_normal(A.m)
        return 40, 24, A, b
    N = 128 if kind == "ct128" else 32
    P = pg.make_problem("ct256", size=N)
    return N, N, P.A, P.b[:, 0]


def _oracle_sizes(n_v, n_h, d, max_coarse, max_levels=64):
    Ks, _, _ = amg.hierarchy(mg.weighted_laplacian(ops.gradient(n_v, n_h), d), max_levels, max_coarse)
    return [K.shape[0] for K in Ks]


@pytest.mark.parametrize("kind,coarse_max", [("blur", 256), ("blur", 24), ("blur40x24", 256), ("blur40x24", 24),
                                             ("ct", 256), ("ct", 24), ("ct128", 256)])
def test_amg_cycle_matches_oracle(kind, coarse_max):
    """ct128 (1.9M nonzeros) builds A_1 = A P_0 with the threaded host
    product."""
    n_v, n_h, A, _ = _problem(kind)
    d = pg.random_weights(ops.n_edges(n_v, n_h), 6, d_min=0.05)
    s = Solver(n_v, n_h, precond=1, coarsening=1, amg_coarse_max=coarse_max)
    s.set_forward_csr(A)
    s.set_weights(d)
    lams = np.array([1e-2, 0.3, 3.0])
    R = pg.rng(5).standard_normal((3, n_v * n_h))
    rd = torch.tensor(R, device="cuda", dtype=torch.float64)
    zd = torch.empty_like(rd)
    L.lcmg_apply_vcycle_dev(s.ctx, lams, rd, zd)
    sizes = L.lcmg_amg_levels(s.ctx)
    s.close()
    h = pm.build_one_sided_amg(A.to_scipy(), ops.gradient(n_v, n_h), d, 64, coarse_max)
    assert sizes.tolist() == [a.shape[1] for a in h.A]
    assert len(sizes) >= 3
    for j, lam in enumerate(lams):
        ref = pm.PaperVCycle(h, lam)(R[j])
        assert _rel(zd[j].cpu().numpy(), ref) <= 1e-10, (lam, _rel(zd[j].cpu().numpy(), ref))


def test_amg_levels_bound_and_rebuild_on_new_weights():
    """`levels` bounds the AMG depth; new weights rebuild the hierarchy (the
    sizes follow the oracle's for each D)."""
    n_v, n_h, A, b = _problem("ct")
    s = Solver(n_v, n_h, precond=1, coarsening=1, amg_coarse_max=32, tol=1e-6, maxit=500)
    s.set_forward_csr(A)
    for seed in (1, 2):
        d = pg.random_weights(ops.n_edges(n_v, n_h), seed, d_min=0.02)
        s.set_weights(d)
        out = s.solve([0.5], b)
        assert out["status"][0, 0] == 0
        assert L.lcmg_amg_levels(s.ctx).tolist() == _oracle_sizes(n_v, n_h, d, 32)
    s.set_params(levels=2)
    s.solve([0.5], b)
    assert L.lcmg_amg_levels(s.ctx).tolist() == _oracle_sizes(n_v, n_h, d, 32, 2)
    s.close()


@pytest.mark.parametrize("kind", ["blur", "ct"])
def test_amg_fgmres_solve_matches_oracle(kind):
    n_v, n_h, A, b = _problem(kind)
    d = pg.random_weights(ops.n_edges(n_v, n_h), 7, d_min=0.05)
    lams = np.array([0.2, 0.5, 2.0])
    s = Solver(n_v, n_h, precond=1, coarsening=1, tol=1e-12, maxit=2000)
    s.set_forward_csr(A)
    s.set_weights(d)
    out = s.solve(lams, b)
    s.close()
    F = ops.ForwardCSR(A.to_scipy())
    Lg = ops.gradient(n_v, n_h)
    c = ops.rhs(F, b)
    for j, lam in enumerate(lams):
        x, it, st, _ = pm.solve(F, Lg, d, n_v, n_h, 64, c, lam, tol=1e-12, maxit=2000, coarsening="amg")
        assert st == krylov.CONVERGED and out["status"][0, j] == 0
        assert _rel(out["x"][0, j], x) <= 1e-8
        rho = np.linalg.norm(F.matvec(out["x"][0, j]) - b)
        assert abs(out["rho"][0, j] - rho) <= 1e-10 * rho


@pytest.mark.parametrize("lam", [0.05, 0.5])
def test_amg_fgmres_iterations_match_oracle(lam):
    """At the paper's tolerance 1e-6 without restarts, both sides (classical
    Gram-Schmidt twice) take the same number of steps within 10%, and fewer
    than with the geometric interpolation."""
    n_v, n_h, A, b = _problem("ct")
    d = np.ones(ops.n_edges(n_v, n_h))
    its = {}
    for co in (1, 0):
        s = Solver(n_v, n_h, precond=1, coarsening=co, levels=0 if co else 3, tol=1e-6, maxit=2000,
                   gmres_restart=2000)
        s.set_forward_csr(A)
        out = s.solve([lam], b)
        s.close()
        assert out["status"][0, 0] == 0
        its[co] = int(out["iters"][0, 0])
    F = ops.ForwardCSR(A.to_scipy())
    c = ops.rhs(F, b)
    _, it, st, _ = pm.solve(F, ops.gradient(n_v, n_h), d, n_v, n_h, 64, c, lam, tol=1e-6, maxit=2000,
                            restart=2000, coarsening="amg", orth="cgs2")
    assert st == krylov.CONVERGED
    assert abs(its[1] - it) <= max(3, 0.1 * it), (its[1], it)
    assert its[1] < its[0]


def test_amg_method_selects_the_same_corners():
    """Algorithm 2 (weights, and so the AMG hierarchy, change every outer
    iteration) with the paper's solver and AMG, and with the default one:
    the same selections."""
    P = pg.make_problem("ct256", size=32)
    lams = np.logspace(-1.5, 0.5, 10)
    hist = []
    for kw in (dict(precond=0, levels=2), dict(precond=1, coarsening=1)):
        s = Solver(32, 32, tol=1e-9, maxit=20000, mode=L.MODE_SEQUENTIAL, **kw)
        s.set_forward_csr(P.A)
        r = s.lcurve_run(lams, P.b[:, 0], max_outer=3)
        hist.append([int(h) for h in r["history"]])
        s.close()
    assert hist[0] == hist[1]


def test_amg_argument_errors():
    with pytest.raises(L.LcmgError):
        Solver(32, 32, precond=1, coarsening=3)
    with pytest.raises(L.LcmgError):
        Solver(32, 32, precond=1, coarsening=1, amg_coarse_max=1)
    P = pg.make_problem("ct256", size=32)
    s = Solver(32, 32, precond=1, coarsening=1)
    s.set_forward_csr(P.A)
    with pytest.raises(L.LcmgError) as e:
        L.lcmg_amg_levels(s.ctx)                 # nothing built yet
    assert e.value.status == L.LCMG_ERR_STATE
    s.set_params(amg_coarse_max=2048)            # 1024 points: no coarse level
    with pytest.raises(L.LcmgError):
        s.solve([0.1], P.b[:, 0])
    s.close()


@pytest.mark.parametrize("n_v,n_h,seed", [(32, 32, 1), (40, 24, 2), (64, 64, 3)])
def test_pmis_split_on_the_device_matches_oracle(n_v, n_h, seed):
    """lcmg_pmis_split (device rounds) on every level of the oracle's PMIS
    hierarchy: the same split, bit for bit, with the level's seed."""
    d = pg.random_weights(ops.n_edges(n_v, n_h), seed, d_min=0.02)
    Ks, _, cfs = amg.hierarchy(mg.weighted_laplacian(ops.gradient(n_v, n_h), d), max_coarse=16, method="pmis")
    assert len(cfs) >= 2
    for k, cf in enumerate(cfs):
        got = L.lcmg_pmis_split(Ks[k], amg.PMIS_SEED + k)
        assert np.array_equal(got, cf), (k, int((got != cf).sum()))


@pytest.mark.parametrize("kind", ["blur", "ct"])
def test_pmis_cycle_and_solve_match_oracle(kind):
    """coarsening = 2: the hierarchy split by PMIS on the device; the cycle
    to 1e-10 and FGMRES solutions to 1e-8 against the oracle's."""
    n_v, n_h, A, b = _problem(kind)
    d = pg.random_weights(ops.n_edges(n_v, n_h), 6, d_min=0.05)
    s = Solver(n_v, n_h, precond=1, coarsening=2, amg_coarse_max=24, tol=1e-12, maxit=2000)
    s.set_forward_csr(A)
    s.set_weights(d)
    lams = np.array([1e-2, 0.3, 3.0])
    R = pg.rng(5).standard_normal((3, n_v * n_h))
    rd = torch.tensor(R, device="cuda", dtype=torch.float64)
    zd = torch.empty_like(rd)
    L.lcmg_apply_vcycle_dev(s.ctx, lams, rd, zd)
    sizes = L.lcmg_amg_levels(s.ctx)
    out = s.solve(lams[1:], b)
    s.close()
    h = pm.build_one_sided_amg(A.to_scipy(), ops.gradient(n_v, n_h), d, 64, 24, method="pmis")
    assert sizes.tolist() == [a.shape[1] for a in h.A]
    for j, lam in enumerate(lams):
        ref = pm.PaperVCycle(h, lam)(R[j])
        assert _rel(zd[j].cpu().numpy(), ref) <= 1e-10, (lam, _rel(zd[j].cpu().numpy(), ref))
    F = ops.ForwardCSR(A.to_scipy())
    c = ops.rhs(F, b)
    for j, lam in enumerate(lams[1:]):
        x, _, st, _ = pm.solve(F, ops.gradient(n_v, n_h), d, n_v, n_h, 64, c, lam, tol=1e-12, maxit=2000,
                               coarsening="pmis", max_coarse=24)
        assert st == krylov.CONVERGED and out["status"][0, j] == 0
        assert _rel(out["x"][0, j], x) <= 1e-8
