"""Closed forms used to pin the oracle (test infrastructure).

* L^T L for the gradient of Sec. 2 is the 5-point Laplacian with Neumann
  (reflecting) boundaries.  Its eigenvectors are the 2-D DCT-II basis and
  its eigenvalues are mu_{k,j} = 4 sin^2(pi k / (2 n_v)) + 4 sin^2(pi j / (2 n_h)).
  Hence for A = I and D = I the solution of eq. (normal),
  (I + lam^2 L^T L) x = b, is x = IDCT(DCT(b) / (1 + lam^2 mu)).
* dense_cholesky_solve: the textbook dense solve of K x = c.
"""
from __future__ import annotations

import numpy as np
import scipy.fft as sfft
import scipy.linalg as sla


def neumann_laplacian_eigs(n_v: int, n_h: int) -> np.ndarray:
    k = np.arange(n_v)[:, None]
    j = np.arange(n_h)[None, :]
    return 4 * np.sin(np.pi * k / (2 * n_v)) ** 2 + 4 * np.sin(np.pi * j / (2 * n_h)) ** 2


def identity_tikhonov_solve(b: np.ndarray, n_v: int, n_h: int, lam: float) -> np.ndarray:
    img = np.asarray(b, dtype=np.float64).reshape((n_v, n_h), order="F")
    bh = sfft.dctn(img, type=2, norm="ortho")
    xh = bh / (1.0 + lam * lam * neumann_laplacian_eigs(n_v, n_h))
    return sfft.idctn(xh, type=2, norm="ortho").reshape(-1, order="F")


def dense_cholesky_solve(K: np.ndarray, c: np.ndarray) -> np.ndarray:
    return sla.cho_solve(sla.cho_factor(K, lower=True), c)
