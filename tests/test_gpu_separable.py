"""The separable blur operator (A = A_h (x) A_v, Sec. 4) against the FP64
oracle, whose A is the zero-boundary 2-D correlation with the full PSF.

Sizes span several 128 x 32 tiles with ragged tails in both directions,
and images smaller than the band, where every row is a boundary row of
both ends of A^T A.  Operator applications agree to 1e-13 (FP64 rounding
of different summation orders), solutions to 1e-8 (FP64) and 1e-6 (mixed)
at tol 1e-12, L-curve values to 1e-6.
"""
import functools

import numpy as np
import pytest
import scipy.sparse as sp

import problemgen as pg
from oracle import operators as ops
from oracle import multigrid as mg
from oracle import krylov
from oracle import lcurve

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2306_11067_gb300 import lcmg as L  # noqa: E402
from paper_2306_11067_gb300 import Solver  # noqa: E402


def _rel(a, b):
    return np.linalg.norm(np.asarray(a) - np.asarray(b)) / max(np.linalg.norm(b), 1e-300)


def _asym(r, seed):
    """A 1-D filter of 2r + 1 positive taps that is not symmetric."""
    f = pg.rng(seed).uniform(0.2, 1.0, 2 * r + 1)
    return f / f.sum()


CASES = [  # n_v, n_h, r_v, r_h (even sides: the grid coarsens below the dense limit)
    (200, 136, 15, 15),   # two and five tiles, ragged in both directions
    (132, 260, 9, 4),     # four samples past a tile
    (24, 20, 15, 15),     # smaller than the band: every row is a boundary row
    (300, 34, 2, 12),
]


@pytest.mark.parametrize("n_v,n_h,rv,rh", CASES)
@pytest.mark.parametrize("how", ["gaussian", "factors"])
def test_separable_normal_apply_matches_oracle(n_v, n_h, rv, rh, how):
    s = Solver(n_v, n_h)
    if how == "gaussian":
        fv, fh = pg.gaussian_psf(rv, 2.0)[:, rv] , pg.gaussian_psf(rh, 3.0)[rh, :]
        psf = np.outer(fv, fh)
        psf /= psf.sum()
        s.set_forward_stencil(psf)
    else:
        fv, fh = _asym(rv, 1), _asym(rh, 2)
        psf = np.outer(fv, fh)
        s.set_forward_separable(fv, fh)
    assert s.forward_form() == L.FORM_SEPARABLE
    d = pg.random_weights(ops.n_edges(n_v, n_h), 3)
    s.set_weights(d)
    lams = np.array([1e-4, 0.3, 5.0])
    X = pg.rng(7).standard_normal((3, n_v * n_h))
    xd = torch.tensor(X, device="cuda", dtype=torch.float64)
    yd = torch.empty_like(xd)
    L.lcmg_apply_normal_dev(s.ctx, lams, xd, yd)
    Y = yd.cpu().numpy()
    F = ops.ForwardPSF(psf, n_v, n_h)
    Lg = ops.gradient(n_v, n_h)
    for j, lam in enumerate(lams):
        assert _rel(Y[j], ops.normal_apply(F, Lg, d, lam, X[j])) <= 1e-13
    # the oracle's diag(A^T A) is a 2-D convolution summing up to (2r + 1)^2
    # = 961 products per pixel: against math.fsum its rounding reaches
    # 2.5e-13 relative at r = 15, where the separable product of two 1-D
    # sums is within 1e-15
    assert _rel(L.lcmg_get_diag(s.ctx, n_v * n_h), F.diag_AtA()) <= 1e-12
    s.close()


def test_non_separable_psf_keeps_the_2d_form():
    n_v, n_h = 40, 36
    psf = pg.rng(5).uniform(0.0, 1.0, (7, 5))
    psf /= psf.sum()
    s = Solver(n_v, n_h)
    s.set_forward_stencil(psf)
    assert s.forward_form() == L.FORM_PSF2D
    d = pg.random_weights(ops.n_edges(n_v, n_h), 4)
    s.set_weights(d)
    X = pg.rng(8).standard_normal((1, n_v * n_h))
    xd = torch.tensor(X, device="cuda", dtype=torch.float64)
    yd = torch.empty_like(xd)
    L.lcmg_apply_normal_dev(s.ctx, np.array([0.1]), xd, yd)
    F = ops.ForwardPSF(psf, n_v, n_h)
    assert _rel(yd[0].cpu().numpy(), ops.normal_apply(F, ops.gradient(n_v, n_h), d, 0.1, X[0])) <= 1e-13
    s.close()


SOLVE_CASES = {  # name: n_v, n_h, levels, PSF radius, sigma, lambdas (oracle solves of a few seconds)
    "r6": (96, 80, 3, 6, 2.0, (0.05, 0.5)),
    "r15": (64, 48, 2, 15, 5.0, (0.1, 0.8)),
}


@functools.lru_cache(maxsize=None)
def _solve_case(name):
    n_v, n_h, levels, r, sig, lams = SOLVE_CASES[name]
    psf = pg.gaussian_psf(r, sig)
    img = pg.phantom_mixed(n_v, n_h, 8, 3)
    b = pg.add_noise(pg.vec(pg.blur_apply(img, psf)), 0.02, 4)
    d = pg.random_weights(ops.n_edges(n_v, n_h), 6, d_min=0.05)
    F = ops.ForwardPSF(psf, n_v, n_h)
    Lg = ops.gradient(n_v, n_h)
    H = mg.build_hierarchy(mg.weighted_laplacian(Lg, d), sp.diags(F.diag_AtA()), n_v, n_h, levels)
    c = ops.rhs(F, b)
    ref = []
    for lam in lams:
        x, it, st, _ = krylov.pcg(lambda v: ops.normal_apply(F, Lg, d, lam, v), c, None,
                                  mg.VCycle(H, lam, nu=1), tol=1e-12, maxit=20000)
        assert st == 0
        ref.append((x, *lcurve.lcurve_values(F, Lg, d, b, x)))
    return psf, b, d, ref


@pytest.mark.parametrize("case", list(SOLVE_CASES))
@pytest.mark.parametrize("precision,bound", [(L.PREC_FP64, 1e-8), (L.PREC_MIXED, 1e-6)])
@pytest.mark.parametrize("mode", [L.MODE_SEQUENTIAL, L.MODE_BATCHED])
def test_separable_solve_matches_oracle(case, precision, bound, mode):
    """A^T b, PCG with the separable operator (both precisions, both
    protocols), rho and eta, for a 13 x 13 and a 31 x 31 Gaussian on ragged
    grids."""
    n_v, n_h, levels, _, _, lams = SOLVE_CASES[case]
    psf, b, d, ref = _solve_case(case)
    s = Solver(n_v, n_h, levels=levels, tol=1e-12, maxit=20000, precision=precision, mode=mode)
    s.set_forward_stencil(psf)
    assert s.forward_form() == L.FORM_SEPARABLE
    s.set_weights(d)
    out = s.solve(np.array(lams), b)
    s.close()
    for j, (x, rho, eta) in enumerate(ref):
        assert out["status"][0, j] == 0
        assert _rel(out["x"][0, j], x) <= bound
        assert abs(out["rho"][0, j] - rho) <= 1e-6 * rho
        assert abs(out["eta"][0, j] - eta) <= 1e-6 * eta
