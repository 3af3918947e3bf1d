"""Operators of the regularized normal equations (oracle; test infrastructure).

* gradient(n_v, n_h): L = [I (x) L_v ; L_h (x) I] with L_v, L_h the
  forward-difference matrices with rows (-1, 1)  [Sec. 2, eq. (gradient)].
  Lx has n_h (n_v - 1) vertical differences followed by (n_h - 1) n_v
  horizontal ones.
* ForwardCSR / ForwardPSF: the forward operator A, either an explicit matrix
  or a point-spread function applied as a zero-boundary correlation.
* normal_apply: (A^T A + lam^2 L^T D^2 L) x evaluated in two stages, first
  [A x ; lam D L x], then the transposes  [Sec. 3.2, eq. (normal)].
* diag_AtA: diag(A^T A) as the sum of squares of each column of A  [Sec. 3.2].
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp


def forward_difference(k: int) -> sp.csr_matrix:
    """(k-1) x k matrix with rows (-1, 1): L_v or L_h of Sec. 2."""
    return sp.diags([-np.ones(k - 1), np.ones(k - 1)], [0, 1], shape=(k - 1, k)).tocsr()


def gradient(n_v: int, n_h: int) -> sp.csr_matrix:
    """L = [I_{n_h} (x) L_v ; L_h (x) I_{n_v}]  (Sec. 2, eq. (gradient))."""
    Lv = forward_difference(n_v)
    Lh = forward_difference(n_h)
    top = sp.kron(sp.identity(n_h), Lv)
    bot = sp.kron(Lh, sp.identity(n_v))
    return sp.vstack([top, bot]).tocsr()


def n_edges(n_v: int, n_h: int) -> int:
    return n_h * (n_v - 1) + (n_h - 1) * n_v


class ForwardCSR:
    """A given as an explicit sparse matrix (values promoted to FP64)."""

    def __init__(self, A: sp.spmatrix):
        self.A = sp.csr_matrix(A, dtype=np.float64)
        self.At = self.A.T.tocsr()
        self.m, self.n = self.A.shape

    def matvec(self, x):
        return self.A @ x

    def rmatvec(self, y):
        return self.At @ y

    def diag_AtA(self):
        """Column sums of squares of A (Sec. 3.2)."""
        return np.asarray(self.A.multiply(self.A).sum(axis=0)).ravel()


class ForwardPSF:
    """A x = zero-boundary correlation of the image with ``psf``.

    (A x)(i, j) = sum_{u, v} psf[u + r_v, v + r_h] x(i + u, j + v); its
    transpose is the zero-boundary convolution with the same PSF.
    """

    def __init__(self, psf: np.ndarray, n_v: int, n_h: int):
        self.psf = np.asarray(psf, dtype=np.float64)
        self.n_v, self.n_h = n_v, n_h
        self.m = self.n = n_v * n_h

    def _img(self, x):
        return np.asarray(x, dtype=np.float64).reshape((self.n_v, self.n_h), order="F")

    def matvec(self, x):
        from scipy.ndimage import correlate
        return correlate(self._img(x), self.psf, mode="constant").reshape(-1, order="F")

    def rmatvec(self, y):
        from scipy.ndimage import convolve
        return convolve(self._img(y), self.psf, mode="constant").reshape(-1, order="F")

    def diag_AtA(self):
        """Column sums of squares: column p of A holds psf entries at rows
        r = p - offset that lie inside the image, so the sum is the
        convolution of the all-ones image with psf**2 (zero boundary)."""
        from scipy.ndimage import convolve
        ones = np.ones((self.n_v, self.n_h))
        return convolve(ones, self.psf ** 2, mode="constant").reshape(-1, order="F")


def make_forward(problem) -> ForwardCSR | ForwardPSF:
    if problem.A is not None:
        return ForwardCSR(problem.A.to_scipy())
    return ForwardPSF(problem.psf, problem.n_v, problem.n_h)


def normal_apply(F, L, d, lam, x):
    """(A^T A + lam^2 L^T D^2 L) x in two stages (Sec. 3.2):
    stage 1 forms [A x ; lam D L x], stage 2 applies [A^T, lam L^T D]."""
    top = F.matvec(x)
    bot = lam * (d * (L @ x))
    return F.rmatvec(top) + lam * (L.T @ (d * bot))


def rhs(F, b):
    """A^T b, the right-hand side of eq. (normal)."""
    return F.rmatvec(b)
