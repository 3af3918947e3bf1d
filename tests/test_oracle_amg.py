"""Pins of the oracle's classical AMG coarsening (oracle.amg, Sec. 3.1)
against textbook results and invariants that follow from the definitions:

  * 1-D Laplacian: every other point is a C point and the interpolation is
    linear (weights 1/2; 1 at a Neumann end, 1/2 at a Dirichlet end);
  * isotropic 5-point Laplacian: red-black coarsening, weights 1/(number of
    neighbours);
  * strong anisotropy: coarsening only along the strong direction (each grid
    line coarsened as in 1-D);
  * the first pass on a small chain worked by hand (the measure increment
    decides it); the first pass gives every F point a strong C connection;
    after the second pass every strong F-F pair shares a strong C connection;
  * for a zero-row-sum matrix (L^T D^2 L) the paper's formula interpolates
    constants exactly;
  * the one-sided products are the Galerkin coarsening of A^T A and of
    L^T D^2 L, and FGMRES with the AMG cycle reaches the dense solution.
"""
import numpy as np
import pytest
import scipy.sparse as sp

import problemgen as pg
from oracle import amg
from oracle import operators as ops
from oracle import multigrid as mg
from oracle import paper_mg as pm
from oracle import krylov


def _lap1d(n, neumann=True):
    K = sp.diags([-np.ones(n - 1), 2 * np.ones(n), -np.ones(n - 1)], [-1, 0, 1]).tolil()
    if neumann:
        K[0, 0] = 1.0
        K[n - 1, n - 1] = 1.0
    return K.tocsr()


@pytest.mark.parametrize("n", [5, 9, 17])
@pytest.mark.parametrize("neumann", [True, False])
def test_1d_laplacian_coarsens_every_other_point_with_linear_interpolation(n, neumann):
    K = _lap1d(n, neumann)
    cf, S = amg.split(K)
    assert cf.tolist() == [i % 2 for i in range(n)]          # F C F C ... F
    P = amg.interpolation(K, S, cf).toarray()
    end = 1.0 if neumann else 0.5
    for i in range(n):
        row = P[i]
        if i % 2:
            assert row[i // 2] == 1.0 and np.count_nonzero(row) == 1
        elif i in (0, n - 1):
            j = 0 if i == 0 else (n - 2) // 2
            assert row[j] == pytest.approx(end, abs=1e-15) and np.count_nonzero(row) == 1
        else:
            assert row[i // 2 - 1] == pytest.approx(0.5, abs=1e-15)
            assert row[i // 2] == pytest.approx(0.5, abs=1e-15)
            assert np.count_nonzero(row) == 2


def test_isotropic_5_point_laplacian_gives_red_black_coarsening():
    n_v, n_h = 10, 8
    K = mg.weighted_laplacian(ops.gradient(n_v, n_h), np.ones(ops.n_edges(n_v, n_h)))
    cf, S = amg.split(K)
    grid = cf.reshape(n_h, n_v)            # column-major: [j][i]
    par = (np.add.outer(np.arange(n_h), np.arange(n_v)) % 2).astype(np.int8)
    assert (grid == par).all() or (grid == 1 - par).all()
    P = amg.interpolation(K, S, cf)
    deg = -(K - sp.diags(K.diagonal())).sum(axis=1).A.ravel()     # neighbours per point
    for i in np.flatnonzero(cf == 0):
        w = P[i].data
        assert np.allclose(w, 1.0 / deg[i], rtol=0, atol=1e-15) and w.size == deg[i]


def test_strong_anisotropy_coarsens_along_the_strong_direction_only():
    """Vertical edges weight 1, horizontal 1e-2 (d^2 = 1e-4): only vertical
    connections are strong, and every grid column is split as the 1-D
    Neumann Laplacian."""
    n_v, n_h = 9, 6
    nvert = n_h * (n_v - 1)
    d = np.concatenate([np.ones(nvert), 1e-2 * np.ones(ops.n_edges(n_v, n_h) - nvert)])
    K = mg.weighted_laplacian(ops.gradient(n_v, n_h), d)
    cf, S = amg.split(K)
    for i in range(K.shape[0]):
        for j in S[i]:
            assert abs(i - j) == 1                                # same column
    for col in cf.reshape(n_h, n_v):
        assert col.tolist() == [i % 2 for i in range(n_v)]


def test_first_pass_measure_increment_on_a_chain_numbered_out_of_order():
    """The path 2 - 0 - 1 - 4 - 3 - 5 (unit weights), by hand: measures
    (strong dependants) [2, 2, 1, 2, 2, 1]; 0 becomes C, 1 and 2 become F;
    the new F point 1 raises its other strong connection 4 to 3, so 4 is the
    next C point (not 3, which a tie would pick), 3 becomes F and raises 5 to
    2, and 5 becomes C: the alternating split F C F C F C along the path."""
    n = 6
    K = np.zeros((n, n))
    for a, b in ((0, 1), (0, 2), (1, 4), (3, 4), (3, 5)):
        K[a, b] = K[b, a] = -1.0
    K[np.arange(n), np.arange(n)] = -K.sum(axis=1)
    S = amg.strength(sp.csr_matrix(K))
    assert amg.first_pass(S, n).tolist() == [1, 0, 0, 0, 1, 1]


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_split_invariants_on_random_weights(seed):
    """On the fine 5-point level and on the first Galerkin level: the second
    pass only moves F points to C (and does move some), and afterwards every
    strong F-F pair shares a strong C connection (pairs exist from level 1)."""
    n_v, n_h = 24, 20
    d = pg.random_weights(ops.n_edges(n_v, n_h), seed, d_min=0.02)
    Ks, _, _ = amg.hierarchy(mg.weighted_laplacian(ops.gradient(n_v, n_h), d), max_levels=2)
    for k, K in enumerate(Ks):
        S = amg.strength(K)
        first = amg.first_pass(S, K.shape[0])
        for i in np.flatnonzero(first == amg.F_PT):
            assert any(first[j] == amg.C_PT for j in S[i])
        cf = amg.second_pass(S, first)
        assert ((first == amg.C_PT) <= (cf == amg.C_PT)).all()
        assert (first != cf).sum() > 0
        pairs = 0
        for i in np.flatnonzero(cf == amg.F_PT):
            Ci = {j for j in S[i] if cf[j] == amg.C_PT}
            for j in S[i]:
                if cf[j] == amg.F_PT:
                    pairs += 1
                    assert Ci.intersection(S[j]), (k, i, j)
        assert pairs > 0 or k == 0


@pytest.mark.parametrize("seed", [4, 5])
def test_interpolation_preserves_constants_of_a_zero_row_sum_operator(seed):
    """sum_j w_ij = 1 follows from the formula when K has zero row sums;
    the cases with strong F neighbours (the F_i^s term) are present."""
    n_v, n_h = 20, 20
    d = pg.random_weights(ops.n_edges(n_v, n_h), seed, d_min=0.02)
    K = mg.weighted_laplacian(ops.gradient(n_v, n_h), d)
    Ks, Ps, cfs = amg.hierarchy(K, max_coarse=16)
    assert len(Ps) >= 2
    for k, P in enumerate(Ps):
        assert np.abs(P @ np.ones(P.shape[1]) - 1.0).max() <= 1e-13
        assert np.abs(Ks[k + 1] @ np.ones(Ks[k + 1].shape[0])).max() <= 1e-12 * abs(Ks[k + 1]).max()
    S = amg.strength(Ks[1])
    cf = cfs[1]
    assert any(cf[j] == amg.F_PT for i in np.flatnonzero(cf == amg.F_PT) for j in S[i])


def test_interpolation_against_a_hand_computed_row():
    """One F point with a strong C neighbour, a strong F neighbour and a
    weak neighbour, worked out from the formula by hand."""
    # points: 0 = i (F), 1 = C, 2 = m (F, strong to i and to 1), 3 = weak C
    K = sp.csr_matrix(np.array([
        [4.0, -2.0, -1.0, -0.1],
        [-2.0, 3.0, -1.0, 0.0],
        [-1.0, -1.0, 2.5, 0.0],
        [-0.1, 0.0, 0.0, 1.0]]))
    S = amg.strength(K)
    assert S[0] == [1, 2]                  # -0.1 <= 0.25 * 2: weak
    cf = np.array([0, 1, 0, 1], dtype=np.int8)
    P = amg.interpolation(K, S, cf).toarray()
    # w_01 = -(k01 + k02 k21 / k21) / (k00 + k03) = -(-2 + -1) / (4 - 0.1)
    assert P[0, 0] == pytest.approx(3.0 / 3.9, rel=1e-15)
    assert P[0, 1] == 0.0 and P[1, 0] == 1.0 and P[3, 1] == 1.0


@pytest.mark.parametrize("method", ["rs", "pmis"])
def test_one_sided_amg_hierarchy_is_the_galerkin_hierarchy(method):
    """A_k^T A_k and M_k^T M_k of the one-sided products are the Galerkin
    hierarchies of A^T A and L^T D^2 L, and the level diagonals dA, dM
    (Sec. 3.2, column sums of squares) are their diagonals, from dense
    products."""
    n_v, n_h = 16, 12
    A = pg.blur_csr(n_v, n_h, pg.gaussian_psf(2, 1.0)).to_scipy()
    Lg = ops.gradient(n_v, n_h)
    d = pg.random_weights(ops.n_edges(n_v, n_h), 8, d_min=0.05)
    h = pm.build_one_sided_amg(A, Lg, d, max_coarse=24, method=method)
    Ks, Ps, _ = amg.hierarchy(mg.weighted_laplacian(Lg, d), max_coarse=24, method=method)
    assert len(h.A) == len(Ks) >= 3
    G = (A.T @ A).tocsr()
    for k in range(len(Ks)):
        AtA = (h.A[k].T @ h.A[k]).toarray()
        MtM = (h.M[k].T @ h.M[k]).toarray()
        assert np.abs(AtA - G.toarray()).max() <= 1e-13 * np.abs(AtA).max()
        assert np.abs(MtM - Ks[k].toarray()).max() <= 1e-12 * np.abs(MtM).max()
        assert np.allclose(h.dM[k], Ks[k].diagonal(), rtol=1e-12, atol=0)
        assert np.allclose(h.dA[k], np.diag(AtA), rtol=1e-12, atol=0)
        assert np.allclose(h.dM[k], np.diag(MtM), rtol=1e-12, atol=0)
        if k < len(Ps):
            G = (Ps[k].T @ G @ Ps[k]).tocsr()


@pytest.mark.parametrize("lam", [1e-2, 0.3, 3.0])
def test_amg_paper_solver_reaches_the_dense_solution(lam):
    n = 16
    A = pg.blur_csr(n, n, pg.gaussian_psf(2, 1.0)).to_scipy()
    Lg = ops.gradient(n, n)
    d = pg.random_weights(ops.n_edges(n, n), 5, d_min=0.05)
    F = ops.ForwardCSR(A)
    c = ops.rhs(F, pg.rng(4).standard_normal(A.shape[0]))
    Kd = (A.T @ A + lam * lam * (Lg.T @ sp.diags(d * d) @ Lg)).toarray()
    x_ref = np.linalg.solve(Kd, c)
    x, it, st, _ = pm.solve(F, Lg, d, n, n, 20, c, lam, tol=1e-12, maxit=500, coarsening="amg", max_coarse=32)
    assert st == krylov.CONVERGED
    assert np.linalg.norm(x - x_ref) <= 10 * np.linalg.cond(Kd) * 1e-12 * np.linalg.norm(x_ref)


def test_splitmix64_reproduces_its_published_outputs():
    """The reference SplitMix64 stream seeded with 0 starts 0xe220a8397b1dcdaf,
    0x6e789e6aa1b965f4, 0x06c45d188009454f; the uniforms are the top 53 bits."""
    u = amg.splitmix64_uniform(0, 3)
    for x, z in zip(u, (0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4, 0x06C45D188009454F)):
        assert x == (z >> 11) * 2.0 ** -53


def _path(n, edges):
    K = np.zeros((n, n))
    for a, b in edges:
        K[a, b] = K[b, a] = -1.0
    K[np.arange(n), np.arange(n)] = -K.sum(axis=1)
    return sp.csr_matrix(K)


def test_pmis_one_round_by_hand():
    """Path 0-1-2-3-4, rand (.1 .9 .2 .8 .3): measures 1.1 2.9 2.2 2.8 1.3;
    1 and 3 exceed their unsorted neighbours and become C; 0, 2, 4 depend on
    them and become F."""
    K = _path(5, [(0, 1), (1, 2), (2, 3), (3, 4)])
    S = amg.strength(K)
    cf = amg.pmis_split(S, 5, np.array([0.1, 0.9, 0.2, 0.8, 0.3]))
    assert cf.tolist() == [0, 1, 0, 1, 0]


def test_pmis_two_rounds_by_hand():
    """Path 0-..-5, measures 1.5 2.1 2.9 2.3 2.2 1.05: round 1 makes 2 C and
    1, 3 F; round 2: 0 has no unsorted neighbour left (C), 4 exceeds 5 (C),
    then 5 depends on 4 (F)."""
    K = _path(6, [(0, 1), (1, 2), (2, 3), (3, 4), (4, 5)])
    S = amg.strength(K)
    cf = amg.pmis_split(S, 6, np.array([0.5, 0.1, 0.9, 0.3, 0.2, 0.05]))
    assert cf.tolist() == [1, 0, 1, 0, 1, 0]


@pytest.mark.parametrize("seed", [1, 2])
def test_pmis_invariants_on_random_weights(seed):
    """Every point is sorted; an F point either has no strong connections at
    all or a strong connection to a C point; the hierarchy interpolates
    constants exactly."""
    n_v, n_h = 24, 20
    d = pg.random_weights(ops.n_edges(n_v, n_h), seed, d_min=0.02)
    K = mg.weighted_laplacian(ops.gradient(n_v, n_h), d)
    S = amg.strength(K)
    ST = amg.transpose_sets(S, K.shape[0])
    cf = amg.pmis_split(S, K.shape[0], amg.splitmix64_uniform(amg.PMIS_SEED, K.shape[0]))
    assert set(cf.tolist()) <= {0, 1}
    for i in np.flatnonzero(cf == amg.F_PT):
        assert (not ST[i] and not S[i]) or any(cf[j] == amg.C_PT for j in S[i])
    Ks, Ps, _ = amg.hierarchy(K, max_coarse=16, method="pmis")
    assert len(Ps) >= 2
    for P in Ps:
        assert np.abs(P @ np.ones(P.shape[1]) - 1.0).max() <= 1e-13


@pytest.mark.parametrize("n,S,expected", [
    # |S^T| = (0, 2, 1): point 1 wins, and 0 and 2 depend on it.
    (3, [[1, 2], [], [1]], [amg.F_PT, amg.C_PT, amg.F_PT]),
    # |S^T| = (1, 2, 0, 2, 1).  Round 1: 3 beats 1 (equal measure, larger
    # index) and 2; 0 loses to its dependant 4 (equal measure, larger
    # index); 1 and 2 depend on 3 and become F.  Round 2: 4 beats 0.
    # Round 3: 0 has no unsorted neighbour left and becomes C.
    (5, [[], [3, 4], [3], [1], [0, 1]], [amg.C_PT, amg.F_PT, amg.F_PT, amg.C_PT, amg.C_PT]),
    # two mutually strong points of equal measure: the larger index is C
    (2, [[1], [0]], [amg.F_PT, amg.C_PT]),
])
def test_pmis_asymmetric_strength_by_hand(n, S, expected):
    """PMIS with zero random parts, worked by hand: the measure is |S_i^T|
    (not |S_i|), a point competes with every unsorted point it is strongly
    connected to in either direction, (measure, index) pairs compare with
    ties to the larger index, and a point becomes F through its own strong
    connections S_i to a new C point."""
    assert amg.pmis_split(S, n, np.zeros(n)).tolist() == expected


def test_hierarchy_limits_and_pmis_seeds():
    """The hierarchy's stated stopping rules and seeds: coarsening stops at
    max_levels levels and at a level of at most max_coarse points (a level
    of exactly max_coarse points is not split); with PMIS, level k draws its
    random parts from the SplitMix64 stream seeded with 2306 + k."""
    K = mg.weighted_laplacian(ops.gradient(24, 20), pg.random_weights(ops.n_edges(24, 20), 5)) \
        + sp.identity(480) * 1e-3
    n = K.shape[0]
    for L in (1, 2, 3):
        Ks, Ps, _ = amg.hierarchy(K, max_levels=L, max_coarse=2)
        assert len(Ks) == L and len(Ps) == L - 1
    assert len(amg.hierarchy(K, max_coarse=n)[0]) == 1
    Ks, _, _ = amg.hierarchy(K, max_coarse=n - 1, max_levels=2)
    assert len(Ks) == 2
    m1 = Ks[1].shape[0]
    assert len(amg.hierarchy(K, max_coarse=m1, max_levels=3)[0]) == 2
    assert len(amg.hierarchy(K, max_coarse=m1 - 1, max_levels=3)[0]) == 3
    Ks, Ps, cfs = amg.hierarchy(K, max_levels=3, max_coarse=2, method="pmis")
    assert amg.PMIS_SEED == 2306
    for k in range(2):
        S = amg.strength(Ks[k])
        nk = Ks[k].shape[0]
        assert np.array_equal(cfs[k], amg.pmis_split(S, nk, amg.splitmix64_uniform(2306 + k, nk)))
        assert not np.array_equal(cfs[k], amg.pmis_split(S, nk, amg.splitmix64_uniform(2306 + k + 1, nk)))


def test_paper_solver_coarsening_selects_the_split():
    """solve(coarsening="pmis") is FGMRES on the hierarchy built with the
    PMIS split, and "amg" on the one built with the two passes (replayed
    bit for bit); on this problem the two splits differ."""
    n = 16
    A = pg.blur_csr(n, n, pg.gaussian_psf(2, 1.0)).to_scipy()
    Lg = ops.gradient(n, n)
    d = pg.random_weights(ops.n_edges(n, n), 5, d_min=0.05)
    F = ops.ForwardCSR(A)
    c = ops.rhs(F, pg.rng(4).standard_normal(A.shape[0]))
    lam = 0.3
    hs = {}
    for coarsening, method in (("amg", "rs"), ("pmis", "pmis")):
        h = pm.build_one_sided_amg(A, Lg, d, 20, 32, method)
        V = pm.PaperVCycle(h, lam, 2, 1)
        ref = pm.fgmres(lambda v: V.K(0, v), c, None, V, 1e-10, 500, 200, "mgs")
        out = pm.solve(F, Lg, d, n, n, 20, c, lam, tol=1e-10, maxit=500, coarsening=coarsening, max_coarse=32)
        assert np.array_equal(out[0], ref[0]) and out[1] == ref[1]
        hs[method] = h
    assert [a.shape for a in hs["rs"].A] != [a.shape for a in hs["pmis"].A] or \
        any((a != b).nnz for a, b in zip(hs["rs"].A, hs["pmis"].A))
