"""Pins of Algorithm 2 as a whole (oracle) and of the problem generators.

* For exact (tightly converged) Tikhonov solutions the residual norm
  rho(lambda) is non-decreasing and the seminorm eta(lambda) non-increasing
  in lambda (a textbook property of the regularized least-squares family).
* The outer loop's bookkeeping: windows follow the trimming rule, the
  selection is an interior point of its window, the run stops exactly when
  three consecutive selections agree or at the iteration limit.
* Generators: the deblurring CSR size of a 32x32 image with a 9x9 PSF, the
  PSF normalisation, and Cavalieri's principle for the CT ray lengths (per
  angle the ray sums over unit-spaced parallel rays add up to the area of
  the image square, and an axis-aligned ray has length N).
"""
import numpy as np
import pytest

import problemgen as pg
from oracle import outer
from oracle import lcurve
from oracle import operators as ops


def test_rho_eta_monotone_in_lambda():
    P = pg.make_problem("deblur32_csr", size=16)
    lams = np.logspace(-3, 1, 8)
    r = outer.lcurve_run(P, outer.Params(levels=2, tol=1e-12), max_outer=1, lambdas=lams)
    rec = r.records[0]
    assert np.all(rec.status == 0)
    assert np.all(np.diff(rec.rho) >= -1e-9 * rec.rho[:-1])
    assert np.all(np.diff(rec.eta) <= 1e-9 * rec.eta[:-1])


def test_outer_loop_bookkeeping():
    P = pg.make_problem("deblur32_csr", size=16)
    lams = np.logspace(-4, 1, 14)
    r = outer.lcurve_run(P, outer.Params(levels=2, tol=1e-8), max_outer=8, lambdas=lams)
    m = len(lams)
    prev = 0
    for ell, rec in enumerate(r.records, start=1):
        assert rec.window == lcurve.lambda_window(m, prev)
        lo, hi = rec.window
        assert lo < rec.selected < hi
        assert np.all(rec.status == 0)
        prev = rec.selected
    stopped = lcurve.should_stop(r.history)
    assert stopped or len(r.history) == 8
    for k in range(3, len(r.history)):
        assert not lcurve.should_stop(r.history[:k])
    assert np.all((r.d > 0) & (r.d <= 1))


def test_generator_blur32_csr_size():
    A = pg.blur_csr(32, 32, pg.gaussian_psf(4, 1.5))
    assert A.nnz == 71824
    assert pg.gaussian_psf(9, 3.0).sum() == pytest.approx(1.0, abs=1e-15)


def test_generator_ct_cavalieri():
    N = 48
    A = pg.ct_csr(N, 30, 69)
    S = A.to_scipy()
    r = (S @ np.ones(A.n)).reshape(30, 69)
    assert np.allclose(r.sum(axis=1), N * N, rtol=2e-3)
    # theta = 0: rays are vertical lines x = s; the one at s = 0.5 - N/2 + k is
    # not present (integer offsets), but every ray with |s| < N/2 has length N
    s = np.arange(69) - 34.0
    inside = np.abs(s) < N / 2
    assert np.allclose(r[0, inside], N)
    assert A.col.dtype == np.int32 and A.val.dtype == np.float32


def test_outer_loop_lx_rule():
    """stop_rule 1: the run ends at the first outer iteration whose
    ||L x*||_2 is below the previous one (or at max_outer), and the
    recorded norms are those of the selected solutions."""
    P = pg.make_problem("deblur32_csr", size=16)
    lams = np.logspace(-4, 1, 14)
    r = outer.lcurve_run(P, outer.Params(levels=2, tol=1e-8, stop_rule=1), max_outer=8, lambdas=lams)
    assert len(r.lx) == len(r.history)
    for k in range(1, len(r.lx) - 1):
        assert r.lx[k] >= r.lx[k - 1]
    assert lcurve.should_stop_lx(r.lx) or len(r.lx) == 8
    Lg = ops.gradient(16, 16)
    assert abs(np.linalg.norm(Lg @ r.x) - r.lx[-1]) <= 1e-12 * r.lx[-1]


def test_constant_image_only_the_first_solve_iterates():
    """b = A 1: the constant image solves eq. (normal) exactly for every
    lambda and every D (L 1 = 0, A^T A 1 = A^T b).  Sweeping from the
    largest lambda to the smallest, each solve warm-started from the previous
    one and each outer iteration from x^(*, l-1) (Sec. 3.3), only the very
    first solve of the run starts away from a solution: every later one
    passes the convergence test at iteration 0."""
    P = pg.make_problem("deblur32_csr", size=16)
    F = ops.make_forward(P)
    P.b = F.matvec(np.ones(F.n))[:, None]
    lams = np.logspace(-4, 1, 14)
    r = outer.lcurve_run(P, outer.Params(levels=2, tol=1e-8), max_outer=3, lambdas=lams)
    assert len(r.records) == 3
    first = r.records[0]
    assert first.window == (1, 14)
    assert first.iters[-1] > 0 and np.all(first.iters[:-1] == 0)
    for rec in r.records[1:]:
        assert np.all(rec.iters == 0)
    for rec in r.records:
        assert np.all(rec.status == 0)
    assert np.max(np.abs(r.x - 1.0)) < 1e-7


def test_repeated_lambda_reuses_the_previous_solution():
    """With a lambda listed twice, the copy swept second (the lower index:
    the sweep runs from the largest lambda down) starts from the other
    copy's converged solution and stops at iteration 0 with it unchanged."""
    P = pg.make_problem("deblur32_csr", size=16)
    lams = np.sort(np.concatenate([np.logspace(-4, 1, 11), [0.01]]))
    i = int(np.flatnonzero(lams == 0.01)[0])
    r = outer.lcurve_run(P, outer.Params(levels=2, tol=1e-8), max_outer=1, lambdas=lams)
    rec = r.records[0]
    assert rec.iters[i] == 0 and rec.iters[i + 1] > 0
    assert np.all(rec.iters[:i] > 0) and np.all(rec.iters[i + 2:] > 0)
    assert np.array_equal(rec.x[i], rec.x[i + 1])


@pytest.fixture(scope="module")
def run16():
    P = pg.make_problem("deblur32_csr", size=16)
    prm = outer.Params(levels=2, tol=1e-8)
    r = outer.lcurve_run(P, prm, max_outer=3, lambdas=np.logspace(-4, 1, 14))
    Ad = P.A.to_scipy().toarray().astype(np.float64)
    return P, prm, r, Ad, ops.gradient(16, 16).toarray()


def test_weights_follow_eq_g(run16):
    """D^(1) = I (Sec. 2); each update multiplies D^(l) by factors in
    [d_min, 1], and the edge where |D^(l) L x^(*, l)| is largest gets
    exactly d_min (there g = 1 and 1 - g^q = 0)."""
    P, prm, r, Ad, Ld = run16
    assert np.all(r.records[0].d == 1.0)
    for prev, rec in zip(r.records, r.records[1:]):
        x_star = prev.x[prev.selected - prev.window[0]]
        v = prev.d * (Ld @ x_star)
        ratio = rec.d / prev.d
        assert np.all(ratio >= prm.d_min) and np.all(ratio <= 1.0)
        assert ratio[np.argmax(np.abs(v))] == prm.d_min


def test_lcurve_points_and_solutions_use_the_current_weights(run16):
    """rho = ||A x - b||_2 and eta = ||D^(l) L x||_2 (Sec. 3.3) of each
    solution, and each solution's true relative residual of
    (A^T A + lam^2 L^T (D^(l))^2 L) x = A^T b within the tolerance, with dense
    matrices."""
    P, prm, r, Ad, Ld = run16
    b = P.b[:, 0]
    c = Ad.T @ b
    for rec in r.records:
        K0 = Ld.T @ np.diag(rec.d ** 2) @ Ld
        for j, (lam, x) in enumerate(zip(rec.lambdas, rec.x)):
            assert rec.rho[j] == pytest.approx(np.linalg.norm(Ad @ x - b), rel=1e-12)
            assert rec.eta[j] == pytest.approx(np.linalg.norm(rec.d * (Ld @ x)), rel=1e-12)
            res = c - (Ad.T @ (Ad @ x) + lam ** 2 * (K0 @ x))
            assert np.linalg.norm(res) <= 1.0001 * prm.tol * np.linalg.norm(c)


def test_hierarchy_is_built_on_the_current_weights(run16):
    """The finest level of each outer iteration's hierarchy holds the two
    parts the cycle works on (Sec. 3.2): L^T (D^(l))^2 L and diag(A^T A), the
    latter from the dense A."""
    P, prm, r, Ad, Ld = run16
    dAA = np.diag(Ad.T @ Ad)
    for rec in r.records:
        assert np.allclose(rec.hier.G_L[0].toarray(), Ld.T @ np.diag(rec.d ** 2) @ Ld,
                           rtol=0, atol=1e-14)
        assert np.allclose(rec.hier.G_A[0].toarray(), np.diag(dAA), rtol=1e-13, atol=0)


def test_each_solve_replays_as_the_preconditioned_solve(run16):
    """Data flow of Algorithm 2: replaying each outer iteration's solves from
    its recorded weights and hierarchy, largest lambda first, each from the
    previous solution and the first from x^(*, l-1), reproduces the recorded
    iterations and solutions bit for bit."""
    P, prm, r, Ad, Ld = run16
    S = outer.setup(P)
    c = ops.rhs(S.F, P.b[:, 0])
    x_prev = np.zeros(S.F.n)
    for rec in r.records:
        x_next = rec.x[rec.selected - rec.window[0]]
        for j in range(len(rec.lambdas) - 1, -1, -1):
            x, it, st, _ = outer.solve(S, rec.hier, rec.d, c, rec.lambdas[j], x_prev, prm)
            assert it == rec.iters[j] and st == rec.status[j]
            assert np.array_equal(x, rec.x[j])
            x_prev = x
        x_prev = x_next
