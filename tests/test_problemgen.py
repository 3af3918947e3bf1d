"""Pins of the synthetic input generators (problemgen), from their stated
definitions.  Both the oracle and the CUDA path read these inputs, so a
mistake here would not show in any parity test.

* CT geometry: pixel (i, j) covers x in [-N/2 + j, -N/2 + j + 1] and
  y in [N/2 - i - 1, N/2 - i]; ray (a, b) is the line p . (cos t, sin t) = s_b
  with s_b = b - (n_bins - 1)/2.  With an even bin count the rays fall
  mid-pixel: at t = 0 ray b is the vertical line x = s_b, which crosses
  column b of every row with length 1; at t = 90 degrees it is the
  horizontal line y = s_b, which crosses row N - 1 - b of every column.
* Gaussian PSF: on a window much wider than sigma its second moment along
  either axis is sigma^2 (the discrete sum differs from the integral by
  about exp(-2 pi^2 sigma^2), Poisson summation), and it is symmetric.
* Noise: b = b_true + level ||b_true|| e/||e||, so ||b - b_true|| is exactly
  level ||b_true|| up to rounding.
"""
import numpy as np
import pytest

import problemgen as pg


def _rows(A, r):
    lo, hi = A.row_ptr[r], A.row_ptr[r + 1]
    return A.col[lo:hi].astype(np.int64), A.val[lo:hi].astype(np.float64)


@pytest.mark.parametrize("N", [8, 12])
def test_ct_axis_aligned_rays_hit_the_stated_pixels(N):
    nb = N
    A = pg.ct_csr(N, 2, nb, dtype=np.float64, angles_deg=[0.0, 90.0])
    for b in range(nb):
        cols, vals = _rows(A, b)                        # t = 0: column b
        assert sorted(cols.tolist()) == sorted(i + b * N for i in range(N))
        assert np.allclose(vals, 1.0, rtol=0, atol=1e-12)
        cols, vals = _rows(A, nb + b)                   # t = 90: row N - 1 - b
        assert sorted(cols.tolist()) == sorted((N - 1 - b) + j * N for j in range(N))
        assert np.allclose(vals, 1.0, rtol=0, atol=1e-12)


def test_ct_diagonal_ray_through_the_centre():
    """t = 45 degrees, s = 0 (odd bin count): the line x + y = 0 crosses the
    diagonal pixels (i, i), through their corners, with length sqrt(2) each."""
    N = 8
    A = pg.ct_csr(N, 1, 9, dtype=np.float64, angles_deg=[45.0])
    cols, vals = _rows(A, 4)
    live = vals > 1e-9
    assert sorted(cols[live].tolist()) == sorted(i + i * N for i in range(N))
    assert np.allclose(vals[live], np.sqrt(2.0), rtol=0, atol=1e-9)


@pytest.mark.parametrize("sigma", [1.5, 3.0])
def test_gaussian_psf_second_moment_is_sigma_squared(sigma):
    r = int(np.ceil(12 * sigma))
    psf = pg.gaussian_psf(r, sigma)
    u = np.arange(-r, r + 1, dtype=np.float64)
    assert psf.sum() == pytest.approx(1.0, abs=1e-14)
    assert np.allclose(psf, psf.T, rtol=0, atol=0) and np.allclose(psf, psf[::-1, ::-1], rtol=0, atol=0)
    assert (psf.sum(axis=1) * u * u).sum() == pytest.approx(sigma ** 2, rel=1e-12)
    assert (psf.sum(axis=0) * u * u).sum() == pytest.approx(sigma ** 2, rel=1e-12)


@pytest.mark.parametrize("level", [0.01, 0.05])
def test_noise_has_the_stated_relative_norm(level):
    b_true = pg.rng(3).uniform(0.0, 2.0, 1000)
    b = pg.add_noise(b_true, level, 17)
    assert np.linalg.norm(b - b_true) == pytest.approx(level * np.linalg.norm(b_true), rel=1e-12)
    assert np.array_equal(b, pg.add_noise(b_true, level, 17))
