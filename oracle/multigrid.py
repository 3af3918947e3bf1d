"""V-cycle preconditioner (oracle; test infrastructure).

Multigrid cycle of Algorithm 1 (Sec. 3.1) with gamma = 1 (a V-cycle), zero
initial guess, nu pre- and nu post-smoothing sweeps, restriction R_k = P_k^T
and Galerkin coarse operators K_{k+1} = P_k^T K_k P_k (Sec. 3.1).  The
operator it is built on is

    K_pre(lam) = lam^2 L^T D^2 L + diag(A^T A)

(the diffusion-type term of eq. (normal) plus the diagonal of the data
term, Sec. 3.2).  The hierarchy of G_L^k = P^T G_L^{k-1} P and
G_A^k = P^T G_A^{k-1} P is independent of lambda and is built once per
weight vector D and reused for every lambda (Sec. 3.2), and
K_k(lam) = lam^2 G_L^k + G_A^k.

Readings where the paper leaves the choice open (the paper itself uses
classical AMG with diagonally preconditioned CG smoothing and FGMRES):
  * coarsening is geometric, cell-centred, factor 2 in each direction;
    P_k = P_h (x) P_v with the 1-D cell-centred linear interpolation
    (fine cell 2I <- 3/4 coarse I + 1/4 coarse I-1, fine cell 2I+1 <-
    3/4 coarse I + 1/4 coarse I+1; a neighbour outside the domain gives its
    weight to coarse I, so P 1 = 1);
  * the smoother is stationary l1-Jacobi, z <- z + D_l1^{-1}(r - K z) with
    D_l1 = diag(sum_j |k_ij|) (or damped Jacobi with weight omega), so the
    V(nu, nu) cycle is a symmetric operator and CG applies;
  * the coarsest level is solved exactly by a dense Cholesky factorisation.

The mixed-precision path may store the smoother data of every level above
the coarsest in FP16 (storage="fp16"; a fixed SPD perturbation of the
cycle, not of the system solved): each array is scaled by the power of two
that puts its largest magnitude in (4096, 8192] (``half_scale``) and
rounded to the nearest FP16 number (``fp16_round``).  On the finest level
the rounded quantities are the edge weights of G_L^0 = L^T W L and
diag(A^T A), so the level operator is lam^2 L^T W^ L + diag(ga^).  On a
coarse level they are the off-diagonal entries of K_k(lam) = lam^2 G_L^k +
G_A^k (one scale per level and lambda, from lam^2 max|G_L^k| + max|G_A^k|
over off-diagonal entries), and the diagonal is rebuilt as the row sum of
G_A^k (the rows of G_L^k sum to zero), rounded to FP32, minus the rounded
off-diagonals, so the rounded operator keeps K_k 1 = G_A^k 1.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np
import scipy.linalg as sla
import scipy.sparse as sp


def interp_1d(n_c: int) -> sp.csr_matrix:
    """(2 n_c) x n_c cell-centred linear interpolation, constants preserved."""
    rows, cols, vals = [], [], []
    for I in range(n_c):
        for f, nb in ((2 * I, I - 1), (2 * I + 1, I + 1)):
            if 0 <= nb < n_c:
                rows += [f, f]; cols += [I, nb]; vals += [0.75, 0.25]
            else:
                rows += [f]; cols += [I]; vals += [1.0]
    return sp.csr_matrix((vals, (rows, cols)), shape=(2 * n_c, n_c))


def prolongation(n_v_c: int, n_h_c: int) -> sp.csr_matrix:
    """P = P_h (x) P_v from a coarse n_v_c x n_h_c grid to the 2x finer grid
    (column-major vectors, so P_v acts on the row index)."""
    return sp.kron(interp_1d(n_h_c), interp_1d(n_v_c)).tocsr()


def weighted_laplacian(L: sp.spmatrix, d: np.ndarray) -> sp.csr_matrix:
    """G_L = L^T D^2 L (Sec. 3.2)."""
    return (L.T @ sp.diags(d * d) @ L).tocsr()


def level_shapes(n_v: int, n_h: int, levels: int):
    shapes = [(n_v, n_h)]
    for _ in range(levels - 1):
        a, b = shapes[-1]
        if a % 2 or b % 2:
            raise ValueError("grid side not divisible by 2 for the requested levels")
        shapes.append((a // 2, b // 2))
    return shapes


def default_levels(n_v: int, n_h: int, coarse_max: int = 16) -> int:
    """Coarsen by 2 while both sides are even and some side exceeds coarse_max."""
    lv, a, b = 1, n_v, n_h
    while (a > coarse_max or b > coarse_max) and a % 2 == 0 and b % 2 == 0:
        a, b, lv = a // 2, b // 2, lv + 1
    return lv


@dataclass
class Hierarchy:
    shapes: list          # (n_v, n_h) per level
    G_L: list             # assembled CSR per level
    G_A: list             # assembled CSR per level
    P: list               # P[k]: level k+1 -> level k


def build_hierarchy(G_L0, G_A0, n_v, n_h, levels) -> Hierarchy:
    """Galerkin hierarchy G^{k+1} = P_k^T G^k P_k for both parts (Sec. 3.1)."""
    shapes = level_shapes(n_v, n_h, levels)
    GL, GA, Ps = [sp.csr_matrix(G_L0)], [sp.csr_matrix(G_A0)], []
    for k in range(levels - 1):
        P = prolongation(*shapes[k + 1])
        Ps.append(P)
        GL.append((P.T @ GL[-1] @ P).tocsr())
        GA.append((P.T @ GA[-1] @ P).tocsr())
    return Hierarchy(shapes, GL, GA, Ps)


def half_scale(mx: float) -> float:
    """The power of two that puts mx (> 0) in (4096, 8192]."""
    if not mx > 0.0:
        return 1.0
    return 2.0 ** math.floor(math.log2(8192.0 / mx))


def fp16_round(v, scale: float):
    """v rounded as stored: nearest FP16 number of v * scale, divided back."""
    return (np.asarray(v, dtype=np.float64) * scale).astype(np.float16).astype(np.float64) / scale


def _offdiag(M):
    M = sp.coo_matrix(M)
    off = M.row != M.col
    return M.row[off], M.col[off], M.data[off]


def fp16_fine_operator(G_L0, G_A0, lam2):
    """lam^2 L^T W^ L + diag(ga^) with the edge weights (minus the
    off-diagonal entries of G_L^0) and diag(A^T A) rounded as stored."""
    r, c, v = _offdiag(G_L0)
    n = G_L0.shape[0]
    w = fp16_round(-v, half_scale(np.max(np.abs(v)) if v.size else 0.0))
    Wo = sp.csr_matrix((-w, (r, c)), shape=(n, n))
    GLh = Wo - sp.diags(np.asarray(Wo.sum(axis=1)).ravel())
    ga = G_A0.diagonal()
    gah = fp16_round(ga, half_scale(np.max(np.abs(ga))))
    return (lam2 * GLh + sp.diags(gah)).tocsr()


def fp16_coarse_operator(G_L, G_A, lam2):
    """K_k(lam) with its off-diagonal entries rounded as stored and the
    diagonal rebuilt from the FP32 row sums of G_A."""
    n = G_L.shape[0]
    K = (lam2 * G_L + G_A).tocsr()
    r, c, v = _offdiag(K)
    _, _, vl = _offdiag(G_L)
    _, _, va = _offdiag(G_A)
    bound = lam2 * (np.max(np.abs(vl)) if vl.size else 0.0) + (np.max(np.abs(va)) if va.size else 0.0)
    vh = fp16_round(v, half_scale(bound))
    Ko = sp.csr_matrix((vh, (r, c)), shape=(n, n))
    s = np.asarray(G_A.sum(axis=1)).ravel().astype(np.float32).astype(np.float64)
    return (Ko + sp.diags(s - np.asarray(Ko.sum(axis=1)).ravel())).tocsr()


class VCycle:
    """B(lam) r: one V(nu, nu) cycle of Algorithm 1 with zero initial guess
    (storage="fp16": the smoothers of every level above the coarsest work on
    the rounded operators described in the module docstring)."""

    def __init__(self, hier: Hierarchy, lam: float, nu: int = 2,
                 smoother: str = "l1", omega: float = 2.0 / 3.0, storage: str = "fp64"):
        self.h, self.nu = hier, nu
        lam2 = lam * lam
        self.K = [(lam2 * gl + ga).tocsr() for gl, ga in zip(hier.G_L, hier.G_A)]
        if storage == "fp16":
            last = len(self.K) - 1
            for k in range(last):
                self.K[k] = (fp16_fine_operator(hier.G_L[0], hier.G_A[0], lam2) if k == 0
                             else fp16_coarse_operator(hier.G_L[k], hier.G_A[k], lam2))
        elif storage != "fp64":
            raise ValueError(storage)
        self.Dinv = []
        for K in self.K:
            if smoother == "l1":
                self.Dinv.append(1.0 / np.asarray(abs(K).sum(axis=1)).ravel())
            elif smoother == "jacobi":
                self.Dinv.append(omega / K.diagonal())
            else:
                raise ValueError(smoother)
        self.chol = sla.cho_factor(self.K[-1].toarray(), lower=True)

    def smooth(self, k, x, b):
        for _ in range(self.nu):
            x = x + self.Dinv[k] * (b - self.K[k] @ x)
        return x

    def cycle(self, k, b):
        if k == len(self.K) - 1:
            return sla.cho_solve(self.chol, b)
        x = self.smooth(k, np.zeros_like(b), b)          # pre-smoothing
        r = b - self.K[k] @ x                            # residual
        rc = self.h.P[k].T @ r                           # restriction R = P^T
        ec = self.cycle(k + 1, rc)                       # coarse correction
        x = x + self.h.P[k] @ ec                         # prolongation
        return self.smooth(k, x, b)                      # post-smoothing

    def __call__(self, r):
        return self.cycle(0, r)

    def as_matrix(self):
        n = self.K[0].shape[0]
        return np.column_stack([self(e) for e in np.eye(n)])
