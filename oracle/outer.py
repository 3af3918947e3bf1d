"""Algorithm 2 end to end (oracle; test infrastructure).

For each outer iteration l: choose the lambda window (full sweep at l = 1,
Sec. 3.4), build the multigrid hierarchy for the current weights D^(l)
(once, reused for every lambda, Sec. 3.2), solve eq. (normal) for each
lambda in the window from the largest to the smallest, each warm-started
from the previous lambda's solution and the first from x^(*, l-1) (zero at
l = 1) (Sec. 3.3), evaluate the L-curve and select its corner, stop when
three consecutive selections agree (Sec. 3.5; or, with stop_rule = 1, when
||L x*||_2 decreases between outer iterations, the heuristic Sec. 3.5
compares against), else update the weights by eq. (g).  D^(1) = I (Sec. 2).
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np
import scipy.sparse as sp

from . import operators as ops
from . import multigrid as mg
from . import krylov
from . import lcurve


@dataclass
class Params:
    nu: int = 2
    smoother: str = "l1"
    omega: float = 2.0 / 3.0
    levels: int | None = None
    coarse_max: int = 16
    q: float = 2.0
    d_min: float = 1e-3
    tol: float = 1e-6
    maxit: int = 10000
    stop_rule: int = 0     # 0: three equal selections (Sec. 3.5); 1: ||L x*|| decreases


@dataclass
class Setup:
    """Quantities fixed by the forward problem (independent of lambda and D)."""
    F: object
    L: sp.csr_matrix
    n_v: int
    n_h: int
    diag_AtA: np.ndarray


def setup(problem) -> Setup:
    F = ops.make_forward(problem)
    L = ops.gradient(problem.n_v, problem.n_h)
    return Setup(F, L, problem.n_v, problem.n_h, F.diag_AtA())


def hierarchy(S: Setup, d, params: Params):
    levels = params.levels or mg.default_levels(S.n_v, S.n_h, params.coarse_max)
    G_L0 = mg.weighted_laplacian(S.L, d)
    G_A0 = sp.diags(S.diag_AtA).tocsr()
    return mg.build_hierarchy(G_L0, G_A0, S.n_v, S.n_h, levels)


def solve(S: Setup, hier, d, c, lam, x0, params: Params, precondition=True):
    V = mg.VCycle(hier, lam, params.nu, params.smoother, params.omega) if precondition else None
    K = lambda v: ops.normal_apply(S.F, S.L, d, lam, v)
    return krylov.pcg(K, c, x0, V, params.tol, params.maxit)


@dataclass
class OuterRecord:
    window: tuple
    lambdas: np.ndarray
    rho: np.ndarray
    eta: np.ndarray
    iters: np.ndarray
    status: np.ndarray
    selected: int          # 1-based index into the full lambda list
    d: np.ndarray | None = None   # the weights D^(l) of this outer iteration
    x: list | None = None         # the solutions, x[j] for lambda index lo + j
    hier: object = None           # the hierarchy built for D^(l)


@dataclass
class RunResult:
    x: np.ndarray
    history: list
    records: list = field(default_factory=list)
    d: np.ndarray | None = None
    lx: list = field(default_factory=list)   # ||L x*||_2 per outer iteration


def lcurve_run(problem, params: Params, rhs_index: int = 0, max_outer: int = 15,
               lambdas=None) -> RunResult:
    S = setup(problem)
    lam_all = np.asarray(problem.lambdas if lambdas is None else lambdas, dtype=np.float64)
    m = len(lam_all)
    b = problem.b[:, rhs_index]
    c = ops.rhs(S.F, b)
    d = np.ones(ops.n_edges(S.n_v, S.n_h))
    x_star = np.zeros(S.F.n)
    hist, recs, lx = [], [], []
    for ell in range(1, max_outer + 1):
        lo, hi = lcurve.lambda_window(m, hist[-1] if hist else 0)
        hier = hierarchy(S, d, params)
        k = hi - lo + 1
        xs = [None] * k
        rho, eta = np.zeros(k), np.zeros(k)
        its, sts = np.zeros(k, int), np.zeros(k, int)
        x_prev = x_star
        for i in range(hi, lo - 1, -1):              # largest lambda first
            j = i - lo
            x, it, st, _ = solve(S, hier, d, c, lam_all[i - 1], x_prev, params)
            xs[j], its[j], sts[j] = x, it, st
            rho[j], eta[j] = lcurve.lcurve_values(S.F, S.L, d, b, x)
            x_prev = x
        sel = lo + lcurve.corner(rho, eta)
        hist.append(sel)
        x_star = xs[sel - lo]
        recs.append(OuterRecord((lo, hi), lam_all[lo - 1:hi], rho, eta, its, sts, sel, d, xs, hier))
        lx.append(float(np.linalg.norm(S.L @ x_star)))
        if params.stop_rule == 1 and lcurve.should_stop_lx(lx):
            break
        if params.stop_rule == 0 and lcurve.should_stop(hist):
            break
        d = lcurve.update_weights(d, S.L, x_star, params.q, params.d_min)
    return RunResult(x_star, hist, recs, d, lx)
