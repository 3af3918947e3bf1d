"""Pins of the oracle's operators against definitions and closed forms.

* The gradient of Sec. 2 (eq. (gradient)): shape, kernel, block order and
  the column-major vectorisation, and L^T L's spectrum, which is the closed
  form of the Neumann 5-point Laplacian.
* The normal-equations operator of eq. (normal) against the gradient of the
  functional 1/2||Ax-b||^2 + 1/2 lam^2 ||D L x||^2 evaluated with explicit
  loops over edges (exact integer arithmetic, compared bitwise).
* diag(A^T A) (Sec. 3.2) against brute-force column sums, and the
  zero-boundary PSF operator against its explicit matrix.
"""
import numpy as np
import pytest
import scipy.sparse as sp

import problemgen as pg
from oracle import operators as ops
from oracle import closed_forms as cf


@pytest.mark.parametrize("n_v,n_h", [(5, 4), (8, 8), (3, 7)])
def test_gradient_shape_and_kernel(n_v, n_h):
    L = ops.gradient(n_v, n_h)
    assert L.shape == (n_h * (n_v - 1) + (n_h - 1) * n_v, n_v * n_h)
    assert np.all(L @ np.ones(n_v * n_h) == 0)


def test_gradient_block_order_and_vectorisation():
    n_v, n_h = 6, 4
    L = ops.gradient(n_v, n_h)
    I, J = np.meshgrid(np.arange(n_v), np.arange(n_h), indexing="ij")
    nvert = n_h * (n_v - 1)
    # x(i, j) = i: vertical differences are 1, horizontal ones 0
    gi = L @ pg.vec(I.astype(float))
    assert np.all(gi[:nvert] == 1) and np.all(gi[nvert:] == 0)
    # x(i, j) = 3 j: vertical 0, horizontal 3
    gj = L @ pg.vec(3.0 * J)
    assert np.all(gj[:nvert] == 0) and np.all(gj[nvert:] == 3)
    # first vertical edge is between pixels (0,0) and (1,0): indices 0 and 1
    row0 = L.getrow(0).toarray().ravel()
    assert row0[0] == -1 and row0[1] == 1
    # first horizontal edge is between (0,0) and (0,1): indices 0 and n_v
    rowh = L.getrow(nvert).toarray().ravel()
    assert rowh[0] == -1 and rowh[n_v] == 1


@pytest.mark.parametrize("n_v,n_h", [(6, 5), (7, 7), (4, 9)])
def test_LtL_is_neumann_laplacian(n_v, n_h):
    L = ops.gradient(n_v, n_h).toarray()
    ev = np.sort(np.linalg.eigvalsh(L.T @ L))
    ref = np.sort(cf.neumann_laplacian_eigs(n_v, n_h).ravel())
    assert np.allclose(ev, ref, atol=1e-12)


def _functional_by_loops(A, b, d, lam, x, n_v, n_h):
    """J(x) = 1/2 ||A x - b||^2 + 1/2 lam^2 sum_edges d_e^2 (x_p - x_q)^2,
    with the edges enumerated pixel by pixel (vertical edges first, in
    column-major order, then horizontal edges)."""
    r = A @ x - b
    J = 0.5 * float(r @ r)
    e = 0
    for j in range(n_h):
        for i in range(n_v - 1):
            p, q = i + j * n_v, i + 1 + j * n_v
            J += 0.5 * lam * lam * d[e] ** 2 * (x[q] - x[p]) ** 2
            e += 1
    for j in range(n_h - 1):
        for i in range(n_v):
            p, q = i + j * n_v, i + (j + 1) * n_v
            J += 0.5 * lam * lam * d[e] ** 2 * (x[q] - x[p]) ** 2
            e += 1
    return J


def test_normal_operator_is_gradient_of_functional_exact():
    """For a quadratic J, (J(x + e_k) - J(x - e_k)) / 2 = (K x - A^T b)_k
    exactly; with small integers every quantity is exact in FP64."""
    g = pg.rng(7)
    n_v, n_h = 4, 3
    n = n_v * n_h
    m = 10
    A = g.integers(-2, 3, size=(m, n)).astype(float)
    b = g.integers(-3, 4, size=m).astype(float)
    x = g.integers(-4, 5, size=n).astype(float)
    d = g.integers(1, 3, size=ops.n_edges(n_v, n_h)).astype(float)
    lam = 2.0
    F = ops.ForwardCSR(sp.csr_matrix(A))
    L = ops.gradient(n_v, n_h)
    grad = ops.normal_apply(F, L, d, lam, x) - ops.rhs(F, b)
    for k in range(n):
        ek = np.zeros(n); ek[k] = 1.0
        fd = (_functional_by_loops(A, b, d, lam, x + ek, n_v, n_h)
              - _functional_by_loops(A, b, d, lam, x - ek, n_v, n_h)) / 2.0
        assert fd == grad[k]


def test_diag_AtA_column_sums_bruteforce():
    g = pg.rng(3)
    A = sp.random(30, 20, density=0.3, random_state=4, format="csr")
    F = ops.ForwardCSR(A)
    Ad = A.toarray()
    ref = np.array([sum(Ad[r, p] ** 2 for r in range(30)) for p in range(20)])
    assert np.allclose(F.diag_AtA(), ref, rtol=1e-14, atol=0)
    del g


@pytest.mark.parametrize("n_v,n_h,r,s", [(12, 9, 2, 1.0), (16, 16, 4, 1.5), (7, 10, 3, 0.8)])
def test_psf_operator_matches_explicit_matrix(n_v, n_h, r, s):
    psf = pg.gaussian_psf(r, s)
    # break the symmetry so a transposed PSF would be caught
    psf = psf * (1.0 + 0.3 * np.arange(psf.size).reshape(psf.shape) / psf.size)
    Acsr = pg.blur_csr(n_v, n_h, psf).to_scipy()
    F = ops.ForwardPSF(psf, n_v, n_h)
    x = pg.rng(1).standard_normal(n_v * n_h)
    y = pg.rng(2).standard_normal(n_v * n_h)
    assert np.allclose(F.matvec(x), Acsr @ x, rtol=0, atol=1e-13)
    assert np.allclose(F.rmatvec(y), Acsr.T @ y, rtol=0, atol=1e-13)
    assert np.allclose(F.diag_AtA(), ops.ForwardCSR(Acsr).diag_AtA(), rtol=1e-13)


def test_blur_csr_explicit_entry():
    """(A x)(i, j) = sum psf[u + r, v + r] x(i + u, j + v): check one entry."""
    psf = np.arange(9.0).reshape(3, 3)
    A = pg.blur_csr(5, 4, psf).to_scipy().toarray()
    i, j = 2, 1
    row = i + j * 5
    for u in (-1, 0, 1):
        for v in (-1, 0, 1):
            assert A[row, (i + u) + (j + v) * 5] == psf[u + 1, v + 1]
    # zero boundary: pixel (0, 0) has only the 2 x 2 in-range neighbours
    assert sorted(A[0][A[0] != 0]) == [4.0, 5.0, 7.0, 8.0]


def test_separable_psf_definition():
    """The anisotropic blur of the deblurring experiment: separable (rank 1),
    symmetric, each 1-D factor a truncated Gaussian of width s * side / 64
    whose two-sided sum is 1."""
    n_v, n_h = 64, 128
    psf = pg.separable_psf(n_v, n_h)
    assert psf.shape == (13, 15)
    assert np.allclose(psf, psf[::-1, :]) and np.allclose(psf, psf[:, ::-1])
    sv = np.linalg.svd(psf, compute_uv=False)
    assert sv[1] <= 1e-14 * sv[0]
    kv, kh = psf.sum(axis=1), psf.sum(axis=0)
    assert abs(kv.sum() - 1.0) <= 1e-14 and abs(kh.sum() - 1.0) <= 1e-14
    sig_v, sig_h = 1.25 * n_v / 64, 1.5 * n_h / 64
    for k, sig, c in ((kv, sig_v, 6), (kh, sig_h, 7)):
        for off in range(1, c + 1):
            assert abs(k[c + off] / k[c] - np.exp(-off * off / (2 * sig * sig))) <= 1e-14


def test_limited_angle_ct_workload():
    P = pg.make_problem("ct256_limited", size=32)
    nb = P.A.m // 66
    assert P.A.m == 66 * nb and P.n == 32 * 32
    # angles 0 .. 130 degrees: the 66th angle's rays differ from the 0-degree ones
    A = P.A.to_scipy()
    assert A[:nb].nnz > 0 and A[65 * nb:].nnz > 0
