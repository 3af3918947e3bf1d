"""The autotuner (params.autotune) and the one-column SpMV configurations it
chooses from (params.spmv_variant), against the oracle."""
import numpy as np
import pytest
import scipy.sparse as sp

import problemgen as pg
from oracle import operators as ops
from oracle import multigrid as mg
from oracle import krylov
from paper_2306_11067_gb300 import Solver, lcmg as L

pytestmark = pytest.mark.gpu


def _rel(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def _oracle_x(P, d, levels, lam, tol=1e-12):
    F = ops.ForwardCSR(P.A.to_scipy())
    Lg = ops.gradient(P.n_v, P.n_h)
    H = mg.build_hierarchy(mg.weighted_laplacian(Lg, d), sp.diags(F.diag_AtA()), P.n_v, P.n_h, levels)
    c = ops.rhs(F, P.b[:, 0])
    x, *_ = krylov.pcg(lambda v: ops.normal_apply(F, Lg, d, lam, v), c, None, mg.VCycle(H, lam),
                       tol=tol, maxit=20000)
    return x


@pytest.mark.parametrize("variant", [1, 2, 3])
@pytest.mark.parametrize("precision,bound", [(L.PREC_FP64, 1e-8), (L.PREC_MIXED, 1e-6)])
def test_every_spmv_variant_reaches_oracle(variant, precision, bound):
    """Each configuration the autotuner may pick, on both passes (and the
    true-residual and rho passes), gives the oracle's solution."""
    P = pg.make_problem("ct256", size=48)
    d = pg.random_weights(ops.n_edges(48, 48), 3, d_min=0.05)
    s = Solver(48, 48, levels=3, spmv_variant=variant, precision=precision, tol=1e-12, maxit=20000)
    s.set_forward_csr(P.A)
    s.set_weights(d)
    out = s.solve([0.1], P.b[:, 0])
    st = s.stats()
    s.close()
    assert (st["tuned_spmv_a"], st["tuned_spmv_at"]) == (variant, variant)
    assert out["status"][0, 0] == 0
    assert _rel(out["x"][0, 0], _oracle_x(P, d, 3, 0.1)) <= bound
    rho = np.linalg.norm(P.A.to_scipy() @ out["x"][0, 0] - P.b[:, 0])
    assert abs(out["rho"][0, 0] - rho) <= 1e-10 * rho


@pytest.mark.parametrize("nlam,mode", [(1, L.MODE_SEQUENTIAL), (3, L.MODE_SEQUENTIAL), (3, L.MODE_BATCHED)])
def test_autotuned_solves_reach_oracle_and_keep_their_choice(nlam, mode):
    """One-column batches (any lambda count in the chain) tune the SpMV
    configurations; a batch of 3 lambdas keeps the batched SpMM."""
    P = pg.make_problem("ct256", size=64)
    d = np.ones(ops.n_edges(64, 64))
    lams = np.array([0.05, 0.3, 2.0])[:nlam]
    s = Solver(64, 64, autotune=1, precision=L.PREC_MIXED, tol=1e-12, maxit=20000, mode=mode)
    s.set_forward_csr(P.A)
    out = s.solve(lams, P.b[:, 0])
    st1 = s.stats()
    out2 = s.solve(lams, P.b[:, 0])
    st2 = s.stats()
    levels = L.lcmg_num_levels(s.ctx)
    s.close()
    if mode == L.MODE_SEQUENTIAL:
        assert st1["tuned_spmv_a"] in (1, 2, 3) and st1["tuned_spmv_at"] in (1, 2, 3, 4, 5, 6)
    else:
        assert (st1["tuned_spmv_a"], st1["tuned_spmv_at"]) == (0, 0)
    assert st1["tuned_vfuse"] in (0, 1)
    # tuned once per width: the second solve reuses the choice and repeats
    # the first one's arithmetic exactly
    assert [st2[k] for k in ("tuned_spmv_a", "tuned_spmv_at", "tuned_vfuse")] == \
        [st1[k] for k in ("tuned_spmv_a", "tuned_spmv_at", "tuned_vfuse")]
    assert np.array_equal(out["x"], out2["x"])
    for j, lam in enumerate(lams):
        assert out["status"][0, j] == 0
        assert _rel(out["x"][0, j], _oracle_x(P, d, levels, lam)) <= 1e-6
