"""Pins of the oracle's V-cycle (Algorithm 1, Sec. 3.1).

* P: constants preserved, linear functions reproduced at interior fine
  cells (fixes the 3/4-1/4 weights and their orientation), and equality with
  an independently written hat-function interpolation.
* Galerkin coarse operators: symmetric, G_L^k annihilates constants, and
  P^T G P equals the dense product with the hat-function P.
* The V(nu, nu) cycle is symmetric and positive definite, a one-level cycle
  is the exact inverse, and at large lambda with D = I the cycle converges
  fast (spectral radius of I - B K below 0.2).
"""
import numpy as np
import pytest
import scipy.sparse as sp

import problemgen as pg
from oracle import operators as ops
from oracle import multigrid as mg


def hat_interp_1d(n_c):
    """Linear interpolation between coarse cell centres, constant beyond the
    first and last centre.  Fine cell f has its centre at coarse coordinate
    y = (f + 0.5) / 2 - 0.5; the weight of coarse cell I is max(0, 1 - |y - I|)."""
    P = np.zeros((2 * n_c, n_c))
    for f in range(2 * n_c):
        y = min(max((f + 0.5) / 2.0 - 0.5, 0.0), n_c - 1.0)
        for I in range(n_c):
            P[f, I] = max(0.0, 1.0 - abs(y - I))
    return P


@pytest.mark.parametrize("n_c", [1, 2, 3, 8])
def test_interp_matches_hat_functions(n_c):
    assert np.allclose(mg.interp_1d(n_c).toarray(), hat_interp_1d(n_c), atol=0)


@pytest.mark.parametrize("a,b", [(4, 4), (5, 3), (8, 2)])
def test_prolongation_constants_and_linears(a, b):
    P = mg.prolongation(a, b)
    assert P.shape == (4 * a * b, a * b)
    assert np.allclose(P @ np.ones(a * b), 1.0, atol=0)
    # linear in the row index: coarse value at centre (I + 1/2) * 2 fine units
    I, J = np.meshgrid(np.arange(a), np.arange(b), indexing="ij")
    uc = pg.vec(2.0 * (I + 0.5))
    uf = pg.unvec(P @ uc, 2 * a, 2 * b)
    fi = np.arange(2 * a)[:, None] + 0.5
    interior = slice(1, 2 * a - 1)
    assert np.allclose(uf[interior, :], np.broadcast_to(fi, uf.shape)[interior, :], atol=1e-14)
    uc = pg.vec(2.0 * (J + 0.5))
    uf = pg.unvec(P @ uc, 2 * a, 2 * b)
    fj = np.arange(2 * b)[None, :] + 0.5
    interior = slice(1, 2 * b - 1)
    assert np.allclose(uf[:, interior], np.broadcast_to(fj, uf.shape)[:, interior], atol=1e-14)


def _random_hierarchy(n_v, n_h, levels, seed):
    L = ops.gradient(n_v, n_h)
    d = pg.random_weights(ops.n_edges(n_v, n_h), seed)
    GA = sp.diags(pg.rng(seed + 1).uniform(0.5, 2.0, n_v * n_h))
    return mg.build_hierarchy(mg.weighted_laplacian(L, d), GA, n_v, n_h, levels)


def test_galerkin_hierarchy_properties():
    H = _random_hierarchy(16, 8, 4, 11)
    for k, (GL, GA) in enumerate(zip(H.G_L, H.G_A)):
        n = GL.shape[0]
        assert abs(GL - GL.T).max() < 1e-14
        assert abs(GA - GA.T).max() < 1e-14
        assert np.abs(GL @ np.ones(n)).max() < 1e-13 * abs(GL).max()
        if k > 0:
            # cell-centred bilinear Galerkin coarse operators couple cells up
            # to two apart: at most a 5 x 5 stencil
            rows, cols = GL.nonzero()
            a, _ = H.shapes[k]
            di = np.abs(rows % a - cols % a)
            dj = np.abs(rows // a - cols // a)
            assert di.max() <= 2 and dj.max() <= 2


def test_galerkin_equals_dense_hat_product():
    H = _random_hierarchy(8, 8, 3, 5)
    for k in range(2):
        a, b = H.shapes[k + 1]
        P = np.kron(hat_interp_1d(b), hat_interp_1d(a))
        for G, Gc in ((H.G_L[k], H.G_L[k + 1]), (H.G_A[k], H.G_A[k + 1])):
            ref = P.T @ G.toarray() @ P
            assert np.allclose(Gc.toarray(), ref, rtol=0, atol=1e-14 * abs(ref).max())


@pytest.mark.parametrize("smoother", ["l1", "jacobi"])
@pytest.mark.parametrize("lam", [1e-3, 0.1, 10.0])
def test_vcycle_symmetric_positive(smoother, lam):
    H = _random_hierarchy(16, 16, 3, 21)
    V = mg.VCycle(H, lam, nu=2, smoother=smoother)
    g = pg.rng(4)
    for _ in range(3):
        u, v = g.standard_normal(256), g.standard_normal(256)
        a, b = V(u) @ v, u @ V(v)
        assert abs(a - b) <= 1e-12 * max(abs(a), abs(b), 1e-300) * 10 + 1e-14 * np.linalg.norm(u) * np.linalg.norm(v)
        assert V(u) @ u > 0
    B = V.as_matrix()
    assert np.allclose(B, B.T, atol=1e-12 * abs(B).max())
    assert np.linalg.eigvalsh(0.5 * (B + B.T)).min() > 0


def test_one_level_cycle_is_exact_inverse():
    H = _random_hierarchy(6, 6, 1, 3)
    lam = 0.7
    V = mg.VCycle(H, lam)
    K = (lam ** 2 * H.G_L[0] + H.G_A[0]).toarray()
    r = pg.rng(9).standard_normal(36)
    assert np.allclose(K @ V(r), r, atol=1e-12)


def _factor(levels, smoother, lam=30.0, n=16):
    L = ops.gradient(n, n)
    GA = sp.diags(np.full(n * n, 1.0))
    H = mg.build_hierarchy(mg.weighted_laplacian(L, np.ones(ops.n_edges(n, n))), GA, n, n, levels)
    V = mg.VCycle(H, lam, nu=2, smoother=smoother)
    K = (lam ** 2 * H.G_L[0] + H.G_A[0]).toarray()
    return np.abs(np.linalg.eigvals(np.eye(n * n) - V.as_matrix() @ K)).max()


@pytest.mark.parametrize("smoother,bound", [("l1", 0.75 ** 4), ("jacobi", 0.2)])
def test_vcycle_convergence_factor_large_lambda(smoother, bound):
    """D = I, lambda large (diffusion-dominated).  Local Fourier analysis of
    the 5-point Laplacian gives the high-frequency smoothing factor
    mu = max |1 - w x| over x in [1/2, 2]: 3/4 for l1-Jacobi (w = 1/2 here)
    and 2/3 for Jacobi with w = 2/3; two pre- and two post-sweeps give
    mu^4, and a correct coarse-grid correction keeps rho(I - B K) at about
    that value, independently of the number of levels."""
    rhos = [_factor(lv, smoother) for lv in (2, 3, 4)]
    assert max(rhos) <= bound * 1.01, rhos
    assert max(rhos) - min(rhos) <= 0.01, rhos


def test_l1_jacobi_is_convergent():
    H = _random_hierarchy(8, 8, 1, 2)
    K = (0.3 ** 2 * H.G_L[0] + H.G_A[0]).toarray()
    Dl1 = np.abs(K).sum(axis=1)
    S = np.eye(64) - K / Dl1[:, None]
    assert np.abs(np.linalg.eigvals(S)).max() < 1.0


def test_default_levels_rule():
    assert mg.default_levels(256, 256) == 5      # 256 -> 16
    assert mg.default_levels(256, 256, 8) == 6   # 256 -> 8
    assert mg.default_levels(512, 512) == 6      # 512 -> 16
    assert mg.default_levels(32, 32) == 2        # 32 -> 16
    assert mg.default_levels(32, 32, 8) == 3     # 32 -> 8
    assert mg.default_levels(40, 24) == 3        # 40 -> 20 -> 10 (24 -> 12 -> 6)
    assert mg.default_levels(40, 24, 4) == 4     # 40 -> 20 -> 10 -> 5
    assert mg.default_levels(33, 32) == 1        # odd side: no coarsening
    with pytest.raises(ValueError):
        mg.level_shapes(12, 12, 4)               # 12 -> 6 -> 3 -> (odd)


# --------------------------------------------------------------------------
# FP16 storage of the smoother data (the mixed path's rounded cycle)
# --------------------------------------------------------------------------
def test_fp16_round_is_round_to_nearest():
    """Against brute force: the stored value is the FP16 number closest to
    v * scale (ties to even), so no neighbouring FP16 number is closer."""
    g = pg.rng(5)
    v = 10.0 ** g.uniform(-9, 1, 4000) * g.choice([-1.0, 1.0], 4000)
    scale = mg.half_scale(np.abs(v).max())
    h = (mg.fp16_round(v, scale) * scale).astype(np.float16)
    x = v * scale
    up = np.nextafter(h, np.float16(np.inf)).astype(np.float64)
    dn = np.nextafter(h, np.float16(-np.inf)).astype(np.float64)
    err = np.abs(h.astype(np.float64) - x)
    assert np.all(err <= np.abs(up - x)) and np.all(err <= np.abs(dn - x))
    # normal range: 11 significant bits
    big = np.abs(x) >= 2.0 ** -14
    assert np.all(err[big] <= 2.0 ** -11 * np.abs(x[big]))


@pytest.mark.parametrize("mx", [1e-12, 3.1e-3, 1.0, 8192.0, 7.7e5])
def test_half_scale_range(mx):
    s = mg.half_scale(mx)
    assert 4096.0 < mx * s <= 8192.0
    assert np.log2(s) == np.round(np.log2(s))  # a power of two: exact scaling


def _hier16(n_v, n_h, levels, seed):
    L = ops.gradient(n_v, n_h)
    d = pg.random_weights(ops.n_edges(n_v, n_h), seed, d_min=0.02)
    ga = pg.rng(seed + 1).uniform(1e-3, 4e-3, n_v * n_h)
    return mg.build_hierarchy(mg.weighted_laplacian(L, d), sp.diags(ga), n_v, n_h, levels)


@pytest.mark.parametrize("lam", [1e-4, 0.05, 2.0])
def test_fp16_coarse_operator_keeps_row_sums_and_is_close(lam):
    H = _hier16(24, 16, 3, 7)
    for k in (1, 2):
        K = (lam ** 2 * H.G_L[k] + H.G_A[k]).toarray()
        Kh = mg.fp16_coarse_operator(H.G_L[k], H.G_A[k], lam ** 2).toarray()
        s32 = np.asarray(H.G_A[k].sum(axis=1)).ravel().astype(np.float32).astype(np.float64)
        # K^ 1 = fl32(G_A 1): the rounding adds a zero-row-sum term
        assert np.abs(Kh.sum(axis=1) - s32).max() <= 1e-14 * np.abs(s32).max()
        off = ~np.eye(K.shape[0], dtype=bool)
        scale = np.abs(K[off]).max()
        assert np.abs(Kh[off] - K[off]).max() <= 2.0 ** -11 * scale + 1e-300
        # K is symmetric to FP64 rounding: a mirrored pair rounds alike, or
        # (a value at a rounding boundary) one FP16 step apart
        assert np.abs(Kh - Kh.T).max() <= 2.0 ** -10 * scale
        assert np.linalg.eigvalsh(0.5 * (Kh + Kh.T)).min() > 0.0


def test_fp16_fine_operator_structure():
    H = _hier16(20, 12, 2, 3)
    lam2 = 0.3
    K = (lam2 * H.G_L[0] + H.G_A[0]).toarray()
    Kh = mg.fp16_fine_operator(H.G_L[0], H.G_A[0], lam2).toarray()
    ga = H.G_A[0].diagonal()
    gah = mg.fp16_round(ga, mg.half_scale(ga.max()))
    # rows sum to the rounded diag(A^T A); symmetric; off-diagonals within 2^-11
    assert np.abs(Kh.sum(axis=1) - gah).max() <= 1e-15 * np.abs(K).max()
    assert np.array_equal(Kh, Kh.T)
    off = ~np.eye(K.shape[0], dtype=bool)
    assert np.all(np.abs(Kh[off] - K[off]) <= 2.0 ** -11 * np.abs(K[off]) + 1e-300)


@pytest.mark.parametrize("lam", [1e-3, 0.3])
def test_fp16_vcycle_symmetric_positive_and_close(lam):
    H = _hier16(16, 16, 3, 11)
    V = mg.VCycle(H, lam, nu=1, storage="fp16")
    g = pg.rng(13)
    u, v = g.standard_normal(256), g.standard_normal(256)
    Bu, Bv = V(u), V(v)
    assert abs(Bu @ v - u @ Bv) <= 1e-12 * abs(Bu @ v)
    assert Bu @ u > 0
    ref = mg.VCycle(H, lam, nu=1)(u)
    assert np.linalg.norm(Bu - ref) <= 1e-2 * np.linalg.norm(ref)
    with pytest.raises(ValueError):
        mg.VCycle(H, lam, storage="fp8")
