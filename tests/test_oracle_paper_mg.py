"""Pins of the oracle's version of the paper's own preconditioner
(one-sided hierarchy, CG relaxation, V(2,1)) and of flexible GMRES, each
against something other than the module itself: the explicit Galerkin
products of A^T A, the stencil hierarchy of oracle.multigrid, CG's finite
termination, GMRES's minimal-residual property by brute force over the
Krylov space, and dense solves."""
import numpy as np
import pytest
import scipy.sparse as sp

import problemgen as pg
from oracle import operators as ops
from oracle import multigrid as mg
from oracle import paper_mg as pm
from oracle import krylov


def _blur(n_v, n_h):
    A = pg.blur_csr(n_v, n_h, pg.gaussian_psf(2, 1.0)).to_scipy()
    return A, ops.gradient(n_v, n_h)


def test_one_sided_hierarchy_is_the_galerkin_hierarchy_of_the_normal_operator():
    n_v, n_h = 16, 12
    A, Lg = _blur(n_v, n_h)
    d = pg.random_weights(ops.n_edges(n_v, n_h), 4, d_min=0.05)
    h = pm.build_one_sided(A, Lg, d, n_v, n_h, 3)
    ref = mg.build_hierarchy(mg.weighted_laplacian(Lg, d), (A.T @ A).tocsr(), n_v, n_h, 3)
    for k in range(3):
        AtA = (h.A[k].T @ h.A[k]).toarray()
        MtM = (h.M[k].T @ h.M[k]).toarray()
        # A_k^T A_k = P^T ... P^T A^T A P ... P  and  M_k^T M_k = G_L^k
        assert np.abs(AtA - ref.G_A[k].toarray()).max() <= 1e-13 * np.abs(AtA).max()
        assert np.abs(MtM - ref.G_L[k].toarray()).max() <= 1e-13 * np.abs(MtM).max()
        assert np.allclose(h.dA[k], np.diag(AtA), rtol=1e-13, atol=0)
        assert np.allclose(h.dM[k], np.diag(MtM), rtol=1e-13, atol=0)
        assert h.A[k].shape == (A.shape[0], h.shapes[k][0] * h.shapes[k][1])


def test_pcg_steps_terminate_and_decrease_the_energy_error():
    g = pg.rng(3)
    n = 12
    Q = g.standard_normal((n, n))
    K = Q @ Q.T + n * np.eye(n)
    b = g.standard_normal(n)
    x_star = np.linalg.solve(K, b)
    dinv = 1.0 / np.diag(K)
    Kf = lambda v: K @ v
    x = pm.pcg_steps(Kf, dinv, np.zeros(n), b, n)          # CG ends in n steps
    assert np.linalg.norm(x - x_star) <= 1e-9 * np.linalg.norm(x_star)
    errs = []
    for s in range(6):
        e = pm.pcg_steps(Kf, dinv, np.zeros(n), b, s) - x_star
        errs.append(e @ K @ e)
    assert all(e1 <= e0 * (1 + 1e-12) for e0, e1 in zip(errs, errs[1:]))


@pytest.mark.parametrize("orth", ["mgs", "cgs2"])
@pytest.mark.parametrize("k", [1, 3, 7])
def test_fgmres_residual_is_the_krylov_minimum(k, orth):
    """Unpreconditioned, no restart: after k steps the residual is the
    least-squares minimum over x0 + span{r0, K r0, ..., K^(k-1) r0}."""
    g = pg.rng(9)
    n = 20
    K = g.standard_normal((n, n)) + 6 * np.eye(n)             # nonsymmetric
    c = g.standard_normal(n)
    x0 = g.standard_normal(n)
    x, it, st, rel = pm.fgmres(lambda v: K @ v, c, x0, None, tol=0.0, maxit=k, restart=50, orth=orth)
    assert it == k
    r0 = c - K @ x0
    basis = np.column_stack([np.linalg.matrix_power(K, i) @ r0 for i in range(k)])
    y, *_ = np.linalg.lstsq(K @ basis, r0, rcond=None)
    best = np.linalg.norm(r0 - K @ basis @ y)
    assert abs(np.linalg.norm(c - K @ x) - best) <= 1e-9 * np.linalg.norm(r0)


@pytest.mark.parametrize("orth", ["mgs", "cgs2"])
def test_fgmres_with_the_exact_inverse_takes_one_step(orth):
    g = pg.rng(2)
    n = 15
    Q = g.standard_normal((n, n))
    K = Q @ Q.T + np.eye(n)
    c = g.standard_normal(n)
    Kinv = np.linalg.inv(K)
    x, it, st, rel = pm.fgmres(lambda v: K @ v, c, None, lambda v: Kinv @ v, tol=1e-12, maxit=10, orth=orth)
    assert st == krylov.CONVERGED and it == 1


def test_one_level_cycle_is_the_exact_solve():
    n_v, n_h = 8, 8
    A, Lg = _blur(n_v, n_h)
    d = np.ones(ops.n_edges(n_v, n_h))
    F = ops.ForwardCSR(A)
    c = ops.rhs(F, pg.rng(1).standard_normal(A.shape[0]))
    x, it, st, rel = pm.solve(F, Lg, d, n_v, n_h, 1, c, 0.3, tol=1e-12, maxit=10)
    assert st == krylov.CONVERGED and it == 1


@pytest.mark.parametrize("n", [8, 12, 16])
@pytest.mark.parametrize("lam", [1e-2, 0.3, 3.0])
def test_paper_solver_reaches_the_dense_solution(n, lam):
    A, Lg = _blur(n, n)
    d = pg.random_weights(ops.n_edges(n, n), 5, d_min=0.05)
    F = ops.ForwardCSR(A)
    b = pg.rng(4).standard_normal(A.shape[0])
    c = ops.rhs(F, b)
    Kd = (A.T @ A + lam * lam * (Lg.T @ sp.diags(d * d) @ Lg)).toarray()
    x_ref = np.linalg.solve(Kd, c)
    tol = 1e-12
    x, it, st, rel = pm.solve(F, Lg, d, n, n, 2, c, lam, tol=tol, maxit=500)
    assert st == krylov.CONVERGED
    assert np.linalg.norm(x - x_ref) <= 10 * np.linalg.cond(Kd) * tol * np.linalg.norm(x_ref)


def test_paper_cycle_beats_the_jacobi_preconditioner():
    """The cycle is a useful preconditioner: on a 32^2 CT problem at a small
    lambda FGMRES with it takes fewer steps than with the Jacobi
    preconditioner diag(A^T A) + lam^2 diag(M^T M) alone (loose check)."""
    P = pg.make_problem("ct256", size=32)
    F = ops.ForwardCSR(P.A.to_scipy())
    Lg = ops.gradient(32, 32)
    d = np.ones(ops.n_edges(32, 32))
    c = ops.rhs(F, P.b[:, 0])
    lam = 0.01
    h = pm.build_one_sided(F.A, Lg, d, 32, 32, 3)
    V = pm.PaperVCycle(h, lam)
    K = lambda v: V.K(0, v)
    _, it_mg, st_mg, _ = pm.fgmres(K, c, None, V, 1e-6, 2000)
    _, it_j, st_j, _ = pm.fgmres(K, c, None, lambda v: V.dinv[0] * v, 1e-6, 2000)
    assert st_mg == krylov.CONVERGED and it_mg < it_j


@pytest.mark.parametrize("orth", ["mgs", "cgs2"])
def test_fgmres_restart_one_is_the_minimal_residual_iteration(orth):
    """Restarted after every step, unpreconditioned GMRES is the minimal
    residual iteration x <- x + a r, a = (r.Kr) / (Kr.Kr): the restart
    logic (true residual, new basis) against that closed form."""
    g = pg.rng(11)
    n = 16
    K = g.standard_normal((n, n)) + 8 * np.eye(n)
    c = g.standard_normal(n)
    x_ref = np.zeros(n)
    for _ in range(5):
        r = c - K @ x_ref
        Kr = K @ r
        x_ref = x_ref + (r @ Kr) / (Kr @ Kr) * r
    x, it, st, _ = pm.fgmres(lambda v: K @ v, c, None, None, tol=0.0, maxit=5, restart=1, orth=orth)
    assert it == 5
    assert np.linalg.norm(x - x_ref) <= 1e-12 * np.linalg.norm(x_ref)


@pytest.mark.parametrize("lam", [0.05, 0.7])
def test_two_level_cycle_by_krylov_optimality(lam):
    """A two-level cycle with a 2-column coarse space P, built from
    characterisations independent of the module: k steps of
    Jacobi-preconditioned CG from 0 minimise the K-norm error over
    span{D^-1 b, (D^-1 K) D^-1 b, ...}; the coarse correction is the exact
    Galerkin correction along P; one CG step from x minimises the K-norm
    error over x + span{D^-1 r}.  D = diag(A^T A) + lam^2 diag(M^T M)."""
    g = pg.rng(21)
    n_v, n_h = 4, 3
    n = n_v * n_h
    A = sp.csr_matrix(g.standard_normal((15, n)))
    Lg = ops.gradient(n_v, n_h)
    d = g.uniform(0.3, 1.0, ops.n_edges(n_v, n_h))
    M = (sp.diags(d) @ Lg).tocsr()
    P = sp.csr_matrix(g.standard_normal((n, 2)))
    As = [A, (A @ P).tocsr()]
    Ms = [M, (M @ P).tocsr()]
    dA = [np.asarray(X.multiply(X).sum(axis=0)).ravel() for X in As]
    dM = [np.asarray(X.multiply(X).sum(axis=0)).ravel() for X in Ms]
    h = pm.OneSided([(n, 1), (2, 1)], As, Ms, [P], dA, dM)
    b = g.standard_normal(n)
    z = pm.PaperVCycle(h, lam, nu1=2, nu2=1)(b)

    K = (A.T @ A + lam * lam * (M.T @ M)).toarray()
    Dinv = 1.0 / np.diag(K)
    xs = np.linalg.solve(K, b)
    # pre-relaxation: K-norm minimiser over the 2-dimensional Krylov space
    v1 = Dinv * b
    V = np.column_stack([v1, Dinv * (K @ v1)])
    x = V @ np.linalg.solve(V.T @ K @ V, V.T @ K @ xs)
    # exact coarse correction along P
    Pd = P.toarray()
    x = x + Pd @ np.linalg.solve(Pd.T @ K @ Pd, Pd.T @ (b - K @ x))
    # one post-relaxation step: K-norm minimiser over x + span{D^-1 r}
    w = Dinv * (b - K @ x)
    x = x + (w @ (b - K @ x)) / (w @ K @ w) * w
    assert np.linalg.norm(z - x) <= 1e-10 * np.linalg.norm(x)
