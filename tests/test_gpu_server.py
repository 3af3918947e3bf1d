"""The serving layer (lcmg_server_*): continuous admission of lambda-sweep
and Algorithm 2 requests of mixed problems and sizes.

Each served request must give the same result alone and in the mix: the
server runs every request on a context of its own with the same kernels and
reduction order as a fresh lcmg_solve / lcmg_lcurve_run, so results are
compared to that and, for one request, to the oracle.
"""
import time

import numpy as np
import pytest
import scipy.sparse as sp

import problemgen as pg
from oracle import operators as ops
from oracle import multigrid as mg
from oracle import krylov
from paper_2306_11067_gb300 import Server, Solver, LcmgError, lcmg as L

pytestmark = pytest.mark.gpu


def _rel(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def _problems():
    """(name, n_v, n_h, kind, operator, b) for a mix of CT and blur problems
    of different sizes, FP32 and FP64 CSR values and a PSF stencil."""
    out = []
    for N in (32, 48):
        P = pg.make_problem("ct256", size=N)
        out.append(("ct%d" % N, N, N, "csr", P.A, P.b[:, 0]))
    P = pg.make_problem("deblur32_csr")
    out.append(("blur32csr", 32, 32, "csr", P.A, P.b[:, 0]))
    P = pg.make_problem("deblur512", size=40, n_rhs=1)
    out.append(("blur40psf", P.n_v, P.n_h, "psf", P.psf, P.b[:, 0]))
    return out


def _alone(n_v, n_h, kind, op, b, lams, max_outer, params):
    s = Solver(n_v, n_h, **params)
    if kind == "csr":
        s.set_forward_csr(op)
    else:
        s.set_forward_stencil(op)
    if max_outer == 0:
        r = s.solve(lams, b)
        out = dict(x=r["x"][0], rho=r["rho"][0], iters=r["iters"][0], status=r["status"][0])
    else:
        r = s.lcurve_run(lams, b, max_outer=max_outer)
        out = dict(x=r["x"], history=[int(h) for h in r["history"]])
    s.close()
    return out


def _add(srv, n_v, n_h, kind, op):
    return srv.add_csr(n_v, n_h, op) if kind == "csr" else srv.add_psf(n_v, n_h, op)


@pytest.mark.parametrize("mode", [L.MODE_BATCHED, L.MODE_SEQUENTIAL])
def test_served_mix_equals_alone(mode):
    params = dict(mode=mode, precision=L.PREC_MIXED, tol=1e-8, maxit=5000)
    probs = _problems()
    srv = Server(hbm_budget=16 << 30, slots=3, **params)
    ids = [_add(srv, n_v, n_h, kind, op) for _, n_v, n_h, kind, op, _ in probs]
    g = pg.rng(17)
    reqs = []
    for k in range(10):
        i = k % len(probs)
        nl = [3, 5, 8, 4][k % 4]
        lams = np.sort(10.0 ** g.uniform(-2, 0.5, nl))
        mo = 3 if k in (3, 8) else 0
        if mo:
            lams = np.logspace(-3, 0.5, 10)
        reqs.append((i, lams, mo, srv.submit(ids[i], lams, probs[i][5], max_outer=mo)))
    results = [srv.wait(t) for *_, t in reqs]
    st = srv.stats()
    srv.close()
    assert st["completed"] == len(reqs) and st["peak_running"] >= 2
    for (i, lams, mo, _), r in zip(reqs, results):
        assert r["state"] == L.LCMG_OK, r.get("error")
        assert r["t_submit"] <= r["t_admit"] <= r["t_done"]
        _, n_v, n_h, kind, op, b = probs[i]
        ref = _alone(n_v, n_h, kind, op, b, lams, mo, params)
        if mo == 0:
            # the same outcome (converged or not) and the same iterates
            assert np.array_equal(r["status"], ref["status"])
            for j in range(len(lams)):
                assert _rel(r["x"][j], ref["x"][j]) <= 1e-12
            assert np.array_equal(r["iters"], ref["iters"])
        else:
            assert r["history"] == ref["history"]
            assert _rel(r["x"], ref["x"]) <= 1e-12


def test_budget_for_one_context_serialises_and_evicts():
    params = dict(precision=L.PREC_FP64, tol=1e-8)
    probs = _problems()[:2]
    srv = Server(hbm_budget=1 << 40, slots=2, **params)
    ids = [_add(srv, n_v, n_h, kind, op) for _, n_v, n_h, kind, op, _ in probs]
    need = max(srv.footprint(i, 4) for i in ids)
    srv.close()
    # room for one context at a time: requests of alternating problems
    # must run one after another and evict each other's contexts
    srv = Server(hbm_budget=int(need * 1.3), slots=2, **params)
    ids = [_add(srv, n_v, n_h, kind, op) for _, n_v, n_h, kind, op, _ in probs]
    lams = np.array([0.01, 0.1, 1.0, 3.0])
    tickets = [(k % 2, srv.submit(ids[k % 2], lams, probs[k % 2][5])) for k in range(4)]
    res = [(i, srv.wait(t)) for i, t in tickets]
    st = srv.stats()
    srv.close()
    assert st["peak_running"] == 1 and st["evictions"] >= 3
    spans = sorted((r["t_admit"], r["t_done"]) for _, r in res)
    for (a0, d0), (a1, d1) in zip(spans, spans[1:]):
        assert a1 >= d0
    for i, r in res:
        _, n_v, n_h, kind, op, b = probs[i]
        ref = _alone(n_v, n_h, kind, op, b, lams, 0, params)
        for j in range(len(lams)):
            assert _rel(r["x"][j], ref["x"][j]) <= 1e-12


def test_oversized_request_fails_nomem_and_queued_request_cancels():
    name, n_v, n_h, kind, op, b = _problems()[1]
    srv = Server(hbm_budget=1 << 40, slots=1, tol=1e-8)
    pid = _add(srv, n_v, n_h, kind, op)
    need = srv.footprint(pid, 3)
    srv.close()
    srv = Server(hbm_budget=need // 2, slots=1, tol=1e-8)
    pid = _add(srv, n_v, n_h, kind, op)
    r = srv.wait(srv.submit(pid, [0.1, 0.3, 1.0], b))
    assert r["state"] == L.LCMG_ERR_NOMEM
    srv.close()
    srv = Server(hbm_budget=1 << 40, slots=1, tol=1e-10)
    pid = _add(srv, n_v, n_h, kind, op)
    long = [srv.submit(pid, np.logspace(-3, 0, 8), b) for _ in range(3)]
    last = srv.submit(pid, [0.1, 1.0], b)
    assert srv.cancel(last) == L.LCMG_OK
    with pytest.raises(LcmgError):
        srv.wait(last)
    for t in long:
        assert srv.wait(t)["state"] == L.LCMG_OK
    srv.close()


def test_warm_start_from_resident_solutions():
    name, n_v, n_h, kind, op, b = _problems()[0]
    lams = np.array([0.02, 0.2, 2.0])
    srv = Server(hbm_budget=1 << 40, slots=1, tol=1e-9, precision=L.PREC_FP64)
    pid = _add(srv, n_v, n_h, kind, op)
    r1 = srv.wait(srv.submit(pid, lams, b))
    r2 = srv.wait(srv.submit(pid, lams, b, warm=1))
    st = srv.stats()
    srv.close()
    assert st["reuses"] >= 1
    assert r2["iters"].sum() < r1["iters"].sum() // 4
    for j in range(len(lams)):
        assert _rel(r2["x"][j], r1["x"][j]) <= 1e-7


def test_served_request_matches_oracle():
    """One CT request, FP64 to 1e-12, against the oracle's PCG."""
    N = 32
    P = pg.make_problem("ct256", size=N)
    lams = np.array([0.05, 0.5])
    srv = Server(hbm_budget=1 << 40, slots=2, precision=L.PREC_FP64, tol=1e-12, maxit=20000)
    pid = srv.add_csr(N, N, P.A)
    r = srv.wait(srv.submit(pid, lams, P.b[:, 0]))
    srv.close()
    F = ops.ForwardCSR(P.A.to_scipy())
    Lg = ops.gradient(N, N)
    d = np.ones(ops.n_edges(N, N))
    H = mg.build_hierarchy(mg.weighted_laplacian(Lg, d), sp.diags(F.diag_AtA()), N, N,
                           mg.default_levels(N, N))
    c = ops.rhs(F, P.b[:, 0])
    for j, lam in enumerate(lams):
        x, *_ = krylov.pcg(lambda v: ops.normal_apply(F, Lg, d, lam, v), c, None, mg.VCycle(H, lam),
                           tol=1e-12, maxit=20000)
        assert _rel(r["x"][j], x) <= 1e-8
