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
