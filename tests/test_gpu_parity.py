"""GPU parity of the CUDA path (through the C ABI) against the FP64 oracle.

Tolerances (FP64 path): operator applications and V-cycles agree to
rounding (1e-12 relative or better; an integer case bitwise); solutions of
eq. (normal) agree to ||x - x_ref|| / ||x_ref|| <= 1e-8 when both sides are
solved to a relative residual of 1e-12 (the forward error of each side is
at most cond(K) * 1e-12); L-curve values rho and eta to 1e-6 relative; the
mixed-precision path to 1e-6.
"""
import numpy as np
import pytest
import scipy.sparse as sp

import problemgen as pg
from oracle import operators as ops
from oracle import multigrid as mg
from oracle import krylov
from oracle import lcurve
from oracle import outer

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2306_11067_gb300 import lcmg as L  # noqa: E402
from paper_2306_11067_gb300 import Solver  # noqa: E402


def _rel(a, b):
    return np.linalg.norm(np.asarray(a) - np.asarray(b)) / max(np.linalg.norm(b), 1e-300)


def _oracle(P, d, levels, lam, tol=1e-12, nu=2, smoother="l1", x0=None):
    F = ops.make_forward(P)
    Lg = ops.gradient(P.n_v, P.n_h)
    H = mg.build_hierarchy(mg.weighted_laplacian(Lg, d), sp.diags(F.diag_AtA()), P.n_v, P.n_h, levels)
    c = ops.rhs(F, P.b[:, 0])
    x, it, st, rel = krylov.pcg(lambda v: ops.normal_apply(F, Lg, d, lam, v), c, x0,
                                mg.VCycle(H, lam, nu=nu, smoother=smoother), tol=tol, maxit=20000)
    rho, eta = lcurve.lcurve_values(F, Lg, d, P.b[:, 0], x)
    return x, it, st, rho, eta


def _solver(P, **kw):
    s = Solver(P.n_v, P.n_h, **kw)
    if P.A is not None:
        s.set_forward_csr(P.A)
    else:
        s.set_forward_stencil(P.psf)
    return s


def _ct(N, seed_shift=0):
    return pg.make_problem("ct256", size=N)


# --------------------------------------------------------------------------
# operators
# --------------------------------------------------------------------------
@pytest.mark.parametrize("kind", ["blur_csr", "ct", "psf"])
def test_diag_AtA(kind):
    if kind == "blur_csr":
        P = pg.make_problem("deblur32_csr")
    elif kind == "ct":
        P = _ct(48)
    else:
        P = pg.make_problem("deblur512", size=40, n_rhs=1)
    s = _solver(P)
    g = L.lcmg_get_diag(s.ctx, P.n)
    ref = ops.make_forward(P).diag_AtA()
    assert _rel(g, ref) <= 1e-13
    s.close()


@pytest.mark.parametrize("kind", ["blur_csr", "ct", "psf"])
def test_normal_apply_parity(kind):
    P = {"blur_csr": lambda: pg.make_problem("deblur32_csr"),
         "ct": lambda: _ct(40),
         "psf": lambda: pg.make_problem("deblur512", size=24, n_rhs=1)}[kind]()
    s = _solver(P)
    d = pg.random_weights(ops.n_edges(P.n_v, P.n_h), 2)
    s.set_weights(d)
    lams = np.array([1e-3, 0.3, 7.0])
    X = pg.rng(3).standard_normal((3, P.n))
    xd = torch.tensor(X, device="cuda", dtype=torch.float64)
    yd = torch.empty_like(xd)
    L.lcmg_apply_normal_dev(s.ctx, lams, xd, yd)
    Y = yd.cpu().numpy()
    F = ops.make_forward(P)
    Lg = ops.gradient(P.n_v, P.n_h)
    for j, lam in enumerate(lams):
        assert _rel(Y[j], ops.normal_apply(F, Lg, d, lam, X[j])) <= 1e-13
    s.close()


def test_normal_apply_integer_exact():
    """A = I, integer weights, integer x and lambda: every product and sum is
    an exactly representable integer, so the GPU must match bitwise."""
    n_v, n_h = 9, 7
    n = n_v * n_h
    A = pg.CSR(n, n, np.arange(n + 1, dtype=np.int64), np.arange(n, dtype=np.int32), np.ones(n))
    s = Solver(n_v, n_h)
    s.set_forward_csr(A)
    d = pg.rng(1).integers(1, 3, ops.n_edges(n_v, n_h)).astype(float)
    s.set_weights(d)
    X = pg.rng(2).integers(-5, 6, (2, n)).astype(float)
    lams = np.array([1.0, 2.0])
    xd = torch.tensor(X, device="cuda", dtype=torch.float64)
    yd = torch.empty_like(xd)
    L.lcmg_apply_normal_dev(s.ctx, lams, xd, yd)
    F = ops.ForwardCSR(sp.identity(n, format="csr"))
    Lg = ops.gradient(n_v, n_h)
    for j, lam in enumerate(lams):
        assert np.array_equal(yd[j].cpu().numpy(), ops.normal_apply(F, Lg, d, lam, X[j]))
    s.close()


@pytest.mark.parametrize("n_v,n_h,levels", [(32, 32, 3), (40, 24, 3), (16, 64, 4)])
def test_galerkin_levels_parity(n_v, n_h, levels):
    psf = pg.gaussian_psf(2, 1.0)
    A = pg.blur_csr(n_v, n_h, psf)
    s = Solver(n_v, n_h, levels=levels)
    s.set_forward_csr(A)
    d = pg.random_weights(ops.n_edges(n_v, n_h), 7)
    s.set_weights(d)
    F = ops.ForwardCSR(A.to_scipy())
    Lg = ops.gradient(n_v, n_h)
    H = mg.build_hierarchy(mg.weighted_laplacian(Lg, d), sp.diags(F.diag_AtA()), n_v, n_h, levels)
    assert L.lcmg_num_levels(s.ctx) == levels
    for k in range(1, levels):
        nv, nh, gl, ga = L.lcmg_get_level(s.ctx, k)
        assert (nv, nh) == H.shapes[k]
        for arr, ref in ((gl, H.G_L[k]), (ga, H.G_A[k])):
            nk = nv * nh
            K = np.zeros((nk, nk))
            for o in range(25):
                di, dj = o % 5 - 2, o // 5 - 2
                for p in range(nk):
                    i, j = p % nv, p // nv
                    if 0 <= i + di < nv and 0 <= j + dj < nh:
                        K[p, (i + di) + (j + dj) * nv] = arr[o, p]
                    else:
                        assert arr[o, p] == 0.0
            R = ref.toarray()
            assert np.abs(K - R).max() <= 1e-13 * np.abs(R).max()
    s.close()


@pytest.mark.parametrize("smoother", [L.SMOOTH_L1_JACOBI, L.SMOOTH_JACOBI])
@pytest.mark.parametrize("n_v,n_h,levels", [(32, 32, 3), (40, 24, 3), (8, 8, 1)])
@pytest.mark.parametrize("nu", [1, 2])
def test_vcycle_parity(smoother, n_v, n_h, levels, nu):
    """The one-kernel-per-level-step V-cycle (vfuse = 0)."""
    A = pg.blur_csr(n_v, n_h, pg.gaussian_psf(2, 1.0))
    s = Solver(n_v, n_h, levels=levels, smoother=smoother, vfuse=0, nu=nu)
    s.set_forward_csr(A)
    d = pg.random_weights(ops.n_edges(n_v, n_h), 9)
    s.set_weights(d)
    lams = np.array([1e-3, 0.1, 10.0])
    R = pg.rng(4).standard_normal((3, n_v * n_h))
    rd = torch.tensor(R, device="cuda", dtype=torch.float64)
    zd = torch.empty_like(rd)
    L.lcmg_apply_vcycle_dev(s.ctx, lams, rd, zd)
    F = ops.ForwardCSR(A.to_scipy())
    Lg = ops.gradient(n_v, n_h)
    H = mg.build_hierarchy(mg.weighted_laplacian(Lg, d), sp.diags(F.diag_AtA()), n_v, n_h, levels)
    sm = "l1" if smoother == L.SMOOTH_L1_JACOBI else "jacobi"
    for j, lam in enumerate(lams):
        ref = mg.VCycle(H, lam, nu=nu, smoother=sm)(R[j])
        assert _rel(zd[j].cpu().numpy(), ref) <= 1e-12, (lam, _rel(zd[j].cpu().numpy(), ref))
    s.close()


# --------------------------------------------------------------------------
# solves
# --------------------------------------------------------------------------
def test_solve_deblur32_csr_parity():
    """32x32 deblurring, 9x9 Gaussian (sigma 1.5) as an FP64 CSR matrix,
    D = I, lambda = 0.05, 3-level V-cycle."""
    P = pg.make_problem("deblur32_csr")
    d = np.ones(ops.n_edges(32, 32))
    for tol in (1e-12, 1e-10):
        s = _solver(P, levels=3, tol=tol)
        out = s.solve([0.05], P.b[:, 0])
        x, it, st, rho, eta = _oracle(P, d, 3, 0.05, tol=tol)
        assert out["status"][0, 0] == 0 and st == 0
        if tol == 1e-12:
            assert _rel(out["x"][0, 0], x) <= 1e-8
        assert abs(out["rho"][0, 0] - rho) <= 1e-6 * rho
        assert abs(out["eta"][0, 0] - eta) <= 1e-6 * eta
        assert abs(int(out["iters"][0, 0]) - it) <= max(2, 0.1 * it)
        s.close()


@pytest.mark.parametrize("precision,bound", [(L.PREC_FP64, 1e-8), (L.PREC_MIXED, 1e-6)])
@pytest.mark.parametrize("N", [32, 48])
def test_solve_ct_batched_parity(precision, bound, N):
    P = _ct(N)
    lams = np.array([0.03, 0.3, 3.0, 30.0])
    d = pg.random_weights(ops.n_edges(N, N), 5, d_min=0.05)
    s = _solver(P, tol=1e-13, precision=precision, maxit=20000, mode=L.MODE_BATCHED)
    s.set_weights(d)
    levels = mg.default_levels(N, N)
    out = s.solve(lams, P.b[:, 0])
    for j, lam in enumerate(lams):
        x, it, st, rho, eta = _oracle(P, d, levels, lam, tol=1e-13)
        assert out["status"][0, j] == 0
        assert _rel(out["x"][0, j], x) <= bound, (lam, _rel(out["x"][0, j], x))
        assert abs(out["rho"][0, j] - rho) <= 1e-6 * rho
        assert abs(out["eta"][0, j] - eta) <= 1e-6 * eta
    s.close()


def test_solve_multi_rhs_and_sequential_mode():
    P = pg.make_problem("deblur512", size=32, n_rhs=3)
    lams = np.array([0.01, 0.1, 1.0])
    s = _solver(P, levels=2, tol=1e-12)
    out_b = s.solve(lams, P.b.T)
    s.set_params(mode=L.MODE_SEQUENTIAL)
    out_s = s.solve(lams, P.b.T)
    F = ops.make_forward(P)
    Lg = ops.gradient(32, 32)
    d = np.ones(ops.n_edges(32, 32))
    H = mg.build_hierarchy(mg.weighted_laplacian(Lg, d), sp.diags(F.diag_AtA()), 32, 32, 2)
    for r in range(3):
        c = ops.rhs(F, P.b[:, r])
        for j, lam in enumerate(lams):
            x, *_ = krylov.pcg(lambda v: ops.normal_apply(F, Lg, d, lam, v), c, None,
                               mg.VCycle(H, lam), tol=1e-12, maxit=20000)
            assert _rel(out_b["x"][r, j], x) <= 1e-8
            assert _rel(out_s["x"][r, j], x) <= 1e-8
    s.close()


@pytest.mark.parametrize("precision", [L.PREC_FP64, L.PREC_MIXED])
def test_solve_psf_parity(precision):
    P = pg.make_problem("deblur512", size=32, n_rhs=1)
    d = pg.random_weights(ops.n_edges(32, 32), 8, d_min=0.05)
    lams = np.array([1e-2, 0.2])
    # FP64: both sides to 1e-13 (forward errors up to cond(K) x tol each)
    tol = 1e-13 if precision == L.PREC_FP64 else 1e-12
    s = _solver(P, levels=2, tol=tol, precision=precision)
    s.set_weights(d)
    out = s.solve(lams, P.b[:, 0])
    for j, lam in enumerate(lams):
        x, it, st, rho, eta = _oracle(P, d, 2, lam, tol=tol)
        assert _rel(out["x"][0, j], x) <= (1e-8 if precision == L.PREC_FP64 else 1e-6)
        assert abs(out["rho"][0, j] - rho) <= 1e-6 * rho
    s.close()


def test_update_weights_parity():
    P = pg.make_problem("deblur32_csr")
    s = _solver(P, levels=3)
    d0 = pg.random_weights(ops.n_edges(32, 32), 11)
    s.set_weights(d0)
    x = P.x_true[:, 0] + 0.01 * pg.rng(12).standard_normal(P.n)
    for q in (1.0, 2.0, 0.7):
        s.set_weights(d0)
        dg = s.update_weights(x, q=q, d_min=1e-3)
        ref = lcurve.update_weights(d0, ops.gradient(32, 32), x, q=q, d_min=1e-3)
        assert np.allclose(dg, ref, rtol=1e-14, atol=0)
    s.close()


@pytest.mark.parametrize("mode", [L.MODE_SEQUENTIAL, L.MODE_BATCHED])
def test_lcurve_run_history_matches_oracle(mode):
    P = pg.make_problem("deblur32_csr", size=16)
    lams = np.logspace(-4, 1, 14)
    prm = outer.Params(levels=2, tol=1e-11)
    ref = outer.lcurve_run(P, prm, max_outer=8, lambdas=lams)
    s = _solver(P, levels=2, tol=1e-11, mode=mode)
    out = s.lcurve_run(lams, P.b[:, 0], max_outer=8)
    assert out["history"] == ref.history
    assert _rel(out["x"], ref.x) <= 1e-6
    assert out["n_solves"] == sum(r.window[1] - r.window[0] + 1 for r in ref.records)
    s.close()


# --------------------------------------------------------------------------
# edge cases and errors
# --------------------------------------------------------------------------
def test_zero_rhs_and_iteration_limit():
    P = pg.make_problem("deblur32_csr", size=16)
    s = _solver(P, levels=2, tol=1e-10)
    out = s.solve([0.1, 1.0], np.zeros(P.m))
    assert np.all(out["x"] == 0) and np.all(out["status"] == 0) and np.all(out["iters"] == 0)
    s.set_params(maxit=3)
    out = s.solve([0.001], P.b[:, 0])
    assert out["status"][0, 0] == L.MAXIT and out["iters"][0, 0] == 3
    s.close()


def test_argument_errors():
    P = pg.make_problem("deblur32_csr", size=16)
    s = _solver(P, levels=2)
    with pytest.raises(L.LcmgError) as e:
        s.solve([0.1, 0.05], P.b[:, 0])                 # not increasing
    assert e.value.status == L.LCMG_ERR_INVALID_ARG
    with pytest.raises(L.LcmgError):
        s.set_weights(np.zeros(ops.n_edges(16, 16)))      # non-positive weights
    with pytest.raises(L.LcmgError):
        s.set_weights(np.ones(5))                         # wrong count
    s.set_params(levels=6)                                # 16 -> ... -> 0.5: not divisible
    with pytest.raises(L.LcmgError):
        s.solve([0.1], P.b[:, 0])
    s.close()
    bad = pg.CSR(4, 16 * 16, np.array([0, 2, 1, 3, 3]), np.zeros(3, np.int32), np.ones(3))
    s = Solver(16, 16)
    with pytest.raises(L.LcmgError):
        s.set_forward_csr(bad)                            # row_ptr decreasing
    s.close()


def test_ragged_grid_and_single_level():
    """40 x 24 (not a power of two, three levels) and a one-level dense solve."""
    for n_v, n_h, levels in ((40, 24, 3), (12, 10, 1)):
        A = pg.blur_csr(n_v, n_h, pg.gaussian_psf(2, 1.2))
        img = pg.phantom_rectangles(n_v, n_h, 3, 4)
        b = pg.add_noise(A.to_scipy() @ pg.vec(img), 0.01, 5)
        P = pg.Problem("ragged", n_v, n_h, "csr", A, None, pg.vec(img)[:, None], b[:, None],
                       np.array([0.05]), levels, 1e-12)
        s = _solver(P, levels=levels, tol=1e-12)
        out = s.solve([0.05, 0.5], b)
        for j, lam in enumerate([0.05, 0.5]):
            x, *_ = _oracle(P, np.ones(ops.n_edges(n_v, n_h)), levels, lam)
            assert _rel(out["x"][0, j], x) <= 1e-8
        s.close()


@pytest.mark.parametrize("nu,levels,nrhs", [(2, 3, 1), (1, 3, 1), (3, 2, 2), (2, 1, 1), (2, 4, 3)])
@pytest.mark.parametrize("precision", [L.PREC_FP64, L.PREC_MIXED])
@pytest.mark.parametrize("mode", [L.MODE_SEQUENTIAL, L.MODE_BATCHED])
def test_iteration_reaches_oracle(nu, levels, nrhs, precision, mode):
    """PCG over V(nu, nu) cycles of 1-4 levels, one or several right-hand
    sides, in the chain and in the batched protocol, reaches the oracle's
    solution."""
    n = 32 if levels > 1 else 12
    P = pg.make_problem("deblur512", size=n, n_rhs=nrhs)
    lams = np.array([0.01, 0.2, 3.0])
    d = pg.random_weights(ops.n_edges(n, n), 21, d_min=0.05)
    # FP64: both sides to 1e-13 (forward errors up to cond(K) x tol each; the
    # chain's warm starts and the oracle's zero starts reach different points)
    tol = 1e-13 if precision == L.PREC_FP64 else 1e-12
    s = _solver(P, levels=levels, nu=nu, tol=tol, precision=precision, mode=mode, maxit=20000)
    s.set_weights(d)
    out = s.solve(lams, P.b.T)
    s.close()
    F = ops.make_forward(P)
    Lg = ops.gradient(n, n)
    H = mg.build_hierarchy(mg.weighted_laplacian(Lg, d), sp.diags(F.diag_AtA()), n, n, levels)
    bound = 1e-8 if precision == L.PREC_FP64 else 1e-6
    for r in range(nrhs):
        c = ops.rhs(F, P.b[:, r])
        for j, lam in enumerate(lams):
            x, it, st, _ = krylov.pcg(lambda v: ops.normal_apply(F, Lg, d, lam, v), c, None,
                                      mg.VCycle(H, lam, nu=nu), tol=tol, maxit=20000)
            assert out["status"][r, j] == 0
            assert _rel(out["x"][r, j], x) <= bound


@pytest.mark.parametrize("mode", [L.MODE_SEQUENTIAL, L.MODE_BATCHED])
def test_lcurve_run_lx_stop_rule_matches_oracle(mode):
    """stop_rule 1 (stop once ||L x*|| decreases): the same selections, the
    same stopping iteration and the same final solution as the oracle."""
    P = pg.make_problem("deblur32_csr", size=16)
    lams = np.logspace(-4, 1, 14)
    ref = outer.lcurve_run(P, outer.Params(levels=2, tol=1e-12, stop_rule=1), max_outer=8, lambdas=lams)
    s = _solver(P, levels=2, tol=1e-12, stop_rule=1, mode=mode, maxit=20000)
    r = s.lcurve_run(lams, P.b[:, 0], max_outer=8)
    s.close()
    assert [int(h) for h in r["history"]] == ref.history
    assert _rel(r["x"], ref.x) <= 1e-8


@pytest.mark.parametrize("name,N", [("ct256_limited", 40), ("deblur256_aniso", 32)])
@pytest.mark.parametrize("precision,bound", [(L.PREC_FP64, 1e-8), (L.PREC_MIXED, 1e-6)])
def test_workload_variants_solve_parity(name, N, precision, bound):
    """Limited-angle CT and the anisotropic separable blur (Sec. 4 variants)."""
    P = pg.make_problem(name, size=N)
    d = pg.random_weights(ops.n_edges(N, N), 8, d_min=0.05)
    lams = np.array([0.01, 0.2])
    s = _solver(P, levels=3, tol=1e-12, precision=precision, maxit=20000)
    s.set_weights(d)
    out = s.solve(lams, P.b[:, 0])
    s.close()
    F = ops.make_forward(P)
    Lg = ops.gradient(N, N)
    H = mg.build_hierarchy(mg.weighted_laplacian(Lg, d), sp.diags(F.diag_AtA()), N, N, 3)
    c = ops.rhs(F, P.b[:, 0])
    for j, lam in enumerate(lams):
        x, *_ = krylov.pcg(lambda v: ops.normal_apply(F, Lg, d, lam, v), c, None, mg.VCycle(H, lam),
                           tol=1e-12, maxit=20000)
        assert out["status"][0, j] == 0
        assert _rel(out["x"][0, j], x) <= bound
