"""The paper's own preconditioner and Krylov method (oracle; test infrastructure).

Sec. 3.2 builds the multigrid hierarchy on the whole normal operator

    K(lam) = A^T A + lam^2 M^T M,    M = D L

without forming A^T A: the interpolation operators P_k define the
one-sided coarse operators A_1 = A, A_{k+1} = A_k P_k and M_1 = D L,
M_{k+1} = M_k P_k (numbered here from 0: A_0 = A, M_0 = D L), so the Galerkin
coarse operator of level k is applied in two stages as
K_k x = A_k^T (A_k x) + lam^2 M_k^T (M_k x).  The hierarchy does not depend
on lambda and is reused for every lambda of an outer iteration.  Stored per
level: the diagonals of A_k^T A_k (column sums of squares of A_k) and of
M_k^T M_k.  Relaxation is diagonally preconditioned CG: each relaxation
call runs a few CG steps on K_k e = b_k from the current iterate with the
preconditioner diag(A_k^T A_k) + lam^2 diag(M_k^T M_k); two steps before
and one after the coarse-grid correction (the paper's V(2,1)).  The
coarsest level is solved exactly.  Because CG relaxation makes the cycle a
nonlinear operator, the outer solver is flexible GMRES (Sec. 3.3).

Readings taken where the paper is silent:
  * P_k is either the cell-centred bilinear interpolation of the geometric
    hierarchy (oracle.multigrid.prolongation) or the paper's classical AMG
    interpolation of G_L = L^T D^2 L (oracle.amg, Sec. 3.1), which depends
    on D and so is rebuilt for every weight vector;
  * restriction R_k = P_k^T, gamma = 1, zero initial guess on coarse levels;
  * FGMRES is right-preconditioned with Givens rotations and modified
    Gram-Schmidt Arnoldi (orth="mgs"), or classical Gram-Schmidt applied
    twice (orth="cgs2"; the two agree in exact arithmetic, and at small
    lambda their step counts differ by ~5-10% through rounding alone); the tolerance is the relative residual
    ||c - K x||_2 <= tol ||c||_2 of the normal equations, judged on the
    Arnoldi estimate and confirmed on the true residual, from which the
    iteration restarts if it is not met; the basis is restarted after
    `restart` vectors (the paper runs without restart: restart >= maxit).

Status codes as in oracle.krylov: 0 converged, 1 iteration limit,
2 breakdown, 3 non-finite values.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np
import scipy.linalg as sla
import scipy.sparse as sp

from . import multigrid as mg
from . import amg
from .krylov import CONVERGED, MAXIT, BREAKDOWN, NONFINITE


def explicit_forward(F) -> sp.csr_matrix:
    """A as an explicit sparse matrix (a PSF operator assembled column by
    column from unit vectors: small grids only)."""
    if hasattr(F, "A"):
        return sp.csr_matrix(F.A, dtype=np.float64)
    n = F.n
    cols = [sp.csr_matrix(F.matvec(e).reshape(-1, 1)) for e in np.eye(n)]
    return sp.hstack(cols).tocsr()


@dataclass
class OneSided:
    shapes: list      # (n_v, n_h) per level
    A: list           # A_k, CSR
    M: list           # M_k, CSR
    P: list           # P[k]: level k+1 -> level k
    dA: np.ndarray    # list of diag(A_k^T A_k)
    dM: np.ndarray    # list of diag(M_k^T M_k)


def build_one_sided(A, L, d, n_v, n_h, levels) -> OneSided:
    """A_{k+1} = A_k P_k and M_{k+1} = M_k P_k with M_0 = diag(d) L (Sec. 3.2)."""
    shapes = mg.level_shapes(n_v, n_h, levels)
    As = [sp.csr_matrix(A, dtype=np.float64)]
    Ms = [(sp.diags(np.asarray(d, dtype=np.float64)) @ L).tocsr()]
    Ps = []
    for k in range(levels - 1):
        P = mg.prolongation(*shapes[k + 1])
        Ps.append(P)
        As.append((As[-1] @ P).tocsr())
        Ms.append((Ms[-1] @ P).tocsr())
    dA = [np.asarray(Ak.multiply(Ak).sum(axis=0)).ravel() for Ak in As]
    dM = [np.asarray(Mk.multiply(Mk).sum(axis=0)).ravel() for Mk in Ms]
    return OneSided(shapes, As, Ms, Ps, dA, dM)


def build_one_sided_amg(A, L, d, max_levels=20, max_coarse=256, method="rs") -> OneSided:
    """As build_one_sided with the classical AMG interpolation of
    G_L = L^T D^2 L (Sec. 3.2; split by the paper's two passes or by PMIS);
    level shapes are (n_k, 1)."""
    Ks, Ps, _ = amg.hierarchy(mg.weighted_laplacian(L, np.asarray(d, dtype=np.float64)), max_levels, max_coarse,
                              method=method)
    As = [sp.csr_matrix(A, dtype=np.float64)]
    Ms = [(sp.diags(np.asarray(d, dtype=np.float64)) @ L).tocsr()]
    for P in Ps:
        As.append((As[-1] @ P).tocsr())
        Ms.append((Ms[-1] @ P).tocsr())
    dA = [np.asarray(Ak.multiply(Ak).sum(axis=0)).ravel() for Ak in As]
    dM = [np.asarray(Mk.multiply(Mk).sum(axis=0)).ravel() for Mk in Ms]
    return OneSided([(K.shape[0], 1) for K in Ks], As, Ms, Ps, dA, dM)


def pcg_steps(apply_K, dinv, x, b, steps):
    """`steps` steps of Jacobi-preconditioned CG on K e = b from x."""
    r = b - apply_K(x)
    z = dinv * r
    p = z.copy()
    rz = r @ z
    for s in range(steps):
        if not rz > 0.0:
            break
        q = apply_K(p)
        pq = p @ q
        if not pq > 0.0:
            break
        a = rz / pq
        x = x + a * p
        r = r - a * q
        if s + 1 < steps:
            z = dinv * r
            rz_new = r @ z
            p = z + (rz_new / rz) * p
            rz = rz_new
    return x


class PaperVCycle:
    """One V(nu1, nu2) cycle of Algorithm 1 on K(lam) with the one-sided
    hierarchy and CG relaxation, zero initial guess: r -> approx K^{-1} r."""

    def __init__(self, h: OneSided, lam: float, nu1: int = 2, nu2: int = 1):
        self.h, self.nu1, self.nu2 = h, nu1, nu2
        self.lam2 = lam * lam
        self.dinv = [1.0 / (dA + self.lam2 * dM) for dA, dM in zip(h.dA, h.dM)]
        Ac, Mc = h.A[-1].toarray(), h.M[-1].toarray()
        self.chol = sla.cho_factor(Ac.T @ Ac + self.lam2 * (Mc.T @ Mc), lower=True)

    def K(self, k, x):
        return self.h.A[k].T @ (self.h.A[k] @ x) + self.lam2 * (self.h.M[k].T @ (self.h.M[k] @ x))

    def cycle(self, k, b):
        if k == len(self.h.A) - 1:
            return sla.cho_solve(self.chol, b)
        Kk = lambda v: self.K(k, v)
        x = pcg_steps(Kk, self.dinv[k], np.zeros_like(b), b, self.nu1)   # pre-relaxation
        r = b - Kk(x)
        ec = self.cycle(k + 1, self.h.P[k].T @ r)                         # coarse correction
        x = x + self.h.P[k] @ ec
        return pcg_steps(Kk, self.dinv[k], x, b, self.nu2)                # post-relaxation

    def __call__(self, r):
        return self.cycle(0, np.asarray(r, dtype=np.float64))


def fgmres(apply_K, c, x0=None, apply_M=None, tol=1e-6, maxit=10000, restart=200, orth="mgs"):
    """Right-preconditioned flexible GMRES.  Returns (x, iterations, status,
    relres); ``iterations`` counts applications of K inside the Arnoldi
    loop (initial and true residuals excluded)."""
    c = np.asarray(c, dtype=np.float64)
    x = np.zeros_like(c) if x0 is None else np.array(x0, dtype=np.float64)
    M = (lambda v: v) if apply_M is None else apply_M
    cn = np.linalg.norm(c)
    if cn == 0.0:
        return np.zeros_like(c), 0, CONVERGED, 0.0
    it = 0
    while True:
        r = c - apply_K(x)
        beta = np.linalg.norm(r)
        if not np.isfinite(beta):
            return x, it, NONFINITE, np.nan
        if beta / cn <= tol:
            return x, it, CONVERGED, beta / cn
        if it >= maxit:
            return x, it, MAXIT, beta / cn
        m = min(restart, maxit - it)
        n = c.size
        V = np.zeros((n, m + 1))
        Z = np.zeros((n, m))
        H = np.zeros((m + 1, m))
        g = np.zeros(m + 1)
        cs, sn = np.zeros(m), np.zeros(m)
        V[:, 0] = r / beta
        g[0] = beta
        j_done = 0
        breakdown = False
        for j in range(m):
            Z[:, j] = M(V[:, j])
            w = apply_K(Z[:, j])
            it += 1
            if orth == "mgs":                            # modified Gram-Schmidt
                for i in range(j + 1):
                    H[i, j] = V[:, i] @ w
                    w = w - H[i, j] * V[:, i]
            else:                                        # classical, twice
                for _ in range(2):
                    h = V[:, : j + 1].T @ w
                    w = w - V[:, : j + 1] @ h
                    H[: j + 1, j] += h
            H[j + 1, j] = np.linalg.norm(w)
            if not np.all(np.isfinite(H[: j + 2, j])):
                return x, it, NONFINITE, np.nan
            if H[j + 1, j] > 0.0:
                V[:, j + 1] = w / H[j + 1, j]
            for i in range(j):                           # earlier rotations
                t = cs[i] * H[i, j] + sn[i] * H[i + 1, j]
                H[i + 1, j] = -sn[i] * H[i, j] + cs[i] * H[i + 1, j]
                H[i, j] = t
            den = np.hypot(H[j, j], H[j + 1, j])
            if den == 0.0:
                breakdown = True
                break
            cs[j], sn[j] = H[j, j] / den, H[j + 1, j] / den
            H[j, j], H[j + 1, j] = den, 0.0
            g[j + 1] = -sn[j] * g[j]
            g[j] = cs[j] * g[j]
            j_done = j + 1
            if abs(g[j + 1]) / cn <= tol:
                break
        if j_done > 0:
            y = sla.solve_triangular(H[:j_done, :j_done], g[:j_done])
            x = x + Z[:, :j_done] @ y
        if breakdown and j_done == 0:
            r = c - apply_K(x)
            return x, it, BREAKDOWN, np.linalg.norm(r) / cn


def solve(F, L, d, n_v, n_h, levels, c, lam, x0=None, tol=1e-6, maxit=10000, nu1=2, nu2=1,
          restart=200, coarsening="geometric", max_coarse=256, orth="mgs"):
    """FGMRES with the paper's V-cycle on eq. (normal) for one lambda;
    with coarsening="amg" (the paper's split) or "pmis", `levels` is the
    largest number of levels."""
    A = explicit_forward(F)
    if coarsening in ("amg", "pmis"):
        h = build_one_sided_amg(A, L, d, levels, max_coarse, "pmis" if coarsening == "pmis" else "rs")
    else:
        h = build_one_sided(A, L, d, n_v, n_h, levels)
    V = PaperVCycle(h, lam, nu1, nu2)
    K = lambda v: V.K(0, v)
    return fgmres(K, c, x0, V, tol, maxit, restart, orth)
