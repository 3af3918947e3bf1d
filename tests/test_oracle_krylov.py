"""Pins of the oracle's PCG solve of eq. (normal) (Sec. 3.2).

* Dense Cholesky solves of the assembled normal equations on 8x8 to 16x16
  deblurring grids with random weights and several lambda.
* The closed form for A = I, D = I: (I + lam^2 L^T L) x = b is diagonalised
  by the 2-D DCT-II (L^T L is the Neumann Laplacian).
* CG invariants: monotone decrease of the K-norm error, r^T z > 0, and the
  status codes for the iteration limit and a zero right-hand side.
"""
import numpy as np
import pytest
import scipy.sparse as sp

import problemgen as pg
from oracle import operators as ops
from oracle import multigrid as mg
from oracle import krylov
from oracle import outer
from oracle import closed_forms as cf


def _blur_problem(N, seed, radius=2, sigma=1.0):
    psf = pg.gaussian_psf(radius, sigma)
    A = pg.blur_csr(N, N, psf).to_scipy()
    img = pg.phantom_rectangles(N, N, 3, seed)
    b = pg.add_noise(A @ pg.vec(img), 0.01, seed + 100)
    return A, b


@pytest.mark.parametrize("N,levels", [(8, 2), (12, 2), (16, 3)])
@pytest.mark.parametrize("lam", [1e-3, 0.05, 2.0])
def test_pcg_matches_dense_cholesky(N, levels, lam):
    A, b = _blur_problem(N, N)
    F = ops.ForwardCSR(A)
    L = ops.gradient(N, N)
    d = pg.random_weights(ops.n_edges(N, N), N + 1)
    K = (A.T @ A + lam ** 2 * L.T @ sp.diags(d * d) @ L).toarray()
    c = A.T @ b
    x_ref = cf.dense_cholesky_solve(K, c)
    H = mg.build_hierarchy(mg.weighted_laplacian(L, d), sp.diags(F.diag_AtA()), N, N, levels)
    V = mg.VCycle(H, lam)
    x, it, st, rel = krylov.pcg(lambda v: ops.normal_apply(F, L, d, lam, v), c, None, V,
                                tol=1e-13, maxit=5000)
    assert st == krylov.CONVERGED
    # forward error <= cond(K) * relative residual (plus rounding of both solves)
    bound = 10.0 * np.linalg.cond(K) * (1e-13 + 1e-15)
    assert np.linalg.norm(x - x_ref) / np.linalg.norm(x_ref) <= max(bound, 1e-12)


@pytest.mark.parametrize("n_v,n_h,lam,levels", [(64, 64, 3.0, 4), (40, 24, 0.5, 3), (32, 32, 20.0, 2)])
def test_pcg_identity_forward_matches_dct_closed_form(n_v, n_h, lam, levels):
    n = n_v * n_h
    F = ops.ForwardCSR(sp.identity(n, format="csr"))
    L = ops.gradient(n_v, n_h)
    d = np.ones(ops.n_edges(n_v, n_h))
    b = pg.vec(pg.phantom_ellipses(n_v, n_h, 4, 5)) + 0.05 * pg.rng(6).standard_normal(n)
    H = mg.build_hierarchy(mg.weighted_laplacian(L, d), sp.identity(n), n_v, n_h, levels)
    x, it, st, rel = krylov.pcg(lambda v: ops.normal_apply(F, L, d, lam, v), b, None,
                                mg.VCycle(H, lam), tol=1e-13, maxit=2000)
    xr = cf.identity_tikhonov_solve(b, n_v, n_h, lam)
    assert st == krylov.CONVERGED
    assert np.linalg.norm(x - xr) / np.linalg.norm(xr) <= 1e-10


def test_pcg_K_norm_error_decreases_monotonically():
    N, lam = 16, 0.05
    A, b = _blur_problem(N, 3)
    F = ops.ForwardCSR(A)
    L = ops.gradient(N, N)
    d = pg.random_weights(ops.n_edges(N, N), 8)
    K = (A.T @ A + lam ** 2 * L.T @ sp.diags(d * d) @ L).toarray()
    c = A.T @ b
    xs = cf.dense_cholesky_solve(K, c)
    H = mg.build_hierarchy(mg.weighted_laplacian(L, d), sp.diags(F.diag_AtA()), N, N, 3)
    V = mg.VCycle(H, lam)
    errs, rzs = [], []

    def cb(x, r):
        e = x - xs
        errs.append(e @ K @ e)
        rzs.append(r @ V(r))

    krylov.pcg(lambda v: K @ v, c, None, V, tol=1e-12, maxit=500, callback=cb)
    assert len(errs) > 5
    assert all(e2 <= e1 * (1 + 1e-9) for e1, e2 in zip(errs, errs[1:]))
    assert all(v > 0 for v in rzs[:-1])


def test_pcg_status_codes():
    K = np.diag(np.arange(1.0, 101.0))
    c = np.ones(100)
    x, it, st, rel = krylov.pcg(lambda v: K @ v, c, tol=1e-14, maxit=3)
    assert st == krylov.MAXIT and it == 3
    x, it, st, rel = krylov.pcg(lambda v: K @ v, np.zeros(100), tol=1e-6)
    assert st == krylov.CONVERGED and it == 0 and np.all(x == 0)
    x, it, st, rel = krylov.pcg(lambda v: -K @ v, c, tol=1e-6)
    assert st == krylov.BREAKDOWN


def test_warm_start_chain_equals_cold_solves():
    P = pg.make_problem("deblur32_csr")
    S = outer.setup(P)
    prm = outer.Params(levels=3, tol=1e-11)
    d = pg.random_weights(ops.n_edges(32, 32), 4)
    H = outer.hierarchy(S, d, prm)
    c = ops.rhs(S.F, P.b[:, 0])
    A, L = S.F.A, S.L
    x_prev = None
    for lam in (1.0, 0.1, 0.01):
        K = (A.T @ A + lam ** 2 * L.T @ sp.diags(d * d) @ L).toarray()
        xw, itw, _, _ = outer.solve(S, H, d, c, lam, x_prev, prm)
        xc, itc, _, _ = outer.solve(S, H, d, c, lam, None, prm)
        # both satisfy ||c - K x|| <= tol ||c||, so they differ by at most
        # 2 cond(K) tol relative to the exact solution
        bound = 2.0 * np.linalg.cond(K) * prm.tol
        assert np.linalg.norm(xw - xc) / np.linalg.norm(xc) <= bound
        x_prev = xw


def test_pcg_confirms_convergence_on_the_true_residual():
    """A perturbation of x injected after an early step makes the recursive
    residual drift from c - K x; convergence must still hold on the true
    residual (the check at exit restarts from it)."""
    import numpy as np
    g = np.random.default_rng(3)
    n = 30
    Q = g.standard_normal((n, n))
    K = Q @ Q.T + n * np.eye(n)
    c = g.standard_normal(n)
    hit = {"done": False}

    def cb(x, r):
        if not hit["done"]:
            x += 1e-3 * g.standard_normal(n)     # x moves, the recursive r does not
            hit["done"] = True

    tol = 1e-10
    x, it, st, rel = krylov.pcg(lambda v: K @ v, c, None, None, tol=tol, maxit=500, callback=cb)
    assert hit["done"] and st == krylov.CONVERGED
    assert np.linalg.norm(c - K @ x) <= tol * np.linalg.norm(c) * (1 + 1e-9)
