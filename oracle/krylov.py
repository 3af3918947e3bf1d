"""Preconditioned conjugate gradients (oracle; test infrastructure).

Solves K x = c for the symmetric positive definite normal-equations matrix
K = A^T A + lam^2 L^T D^2 L of eq. (normal) (Sec. 3.2), c = A^T b, with the
Hestenes-Stiefel recurrences.  Convergence is the relative residual of the
normal equations, ||c - K x||_2 / ||c||_2 <= tol (the paper bounds the l2
norm of this residual, Sec. 3.3; the tolerance is read as relative).  The
test is made on the recursively updated residual; when it passes, the true
residual c - K x is formed and the iteration restarts from it if the true
residual is still above tol.

Status codes: 0 converged, 1 iteration limit, 2 breakdown (p^T K p <= 0 or
r^T z <= 0), 3 non-finite values.
"""
from __future__ import annotations

import numpy as np

CONVERGED, MAXIT, BREAKDOWN, NONFINITE = 0, 1, 2, 3


def pcg(apply_K, c, x0=None, apply_B=None, tol=1e-6, maxit=10000, callback=None):
    """Returns (x, iterations, status, relres).  ``iterations`` counts
    applications of K inside the loop (the initial residual excluded)."""
    c = np.asarray(c, dtype=np.float64)
    x = np.zeros_like(c) if x0 is None else np.array(x0, dtype=np.float64)
    B = (lambda v: v) if apply_B is None else apply_B
    cn = np.linalg.norm(c)
    if cn == 0.0:
        return np.zeros_like(c), 0, CONVERGED, 0.0
    r = c - apply_K(x)
    if np.linalg.norm(r) / cn <= tol:
        return x, 0, CONVERGED, np.linalg.norm(r) / cn
    z = B(r)
    p = z.copy()
    rz = r @ z
    it = 0
    while it < maxit:
        if not np.isfinite(rz):
            return x, it, NONFINITE, np.nan
        if rz <= 0:
            return x, it, BREAKDOWN, np.linalg.norm(r) / cn
        q = apply_K(p)
        pq = p @ q
        it += 1
        if not np.isfinite(pq):
            return x, it, NONFINITE, np.nan
        if pq <= 0:
            return x, it, BREAKDOWN, np.linalg.norm(r) / cn
        alpha = rz / pq
        x = x + alpha * p
        r = r - alpha * q
        if callback is not None:
            callback(x, r)
        if np.linalg.norm(r) / cn <= tol:
            r = c - apply_K(x)                        # true residual at exit
            rel = np.linalg.norm(r) / cn
            if rel <= tol:
                return x, it, CONVERGED, rel
            z = B(r)                                  # restart from it
            p = z.copy()
            rz = r @ z
            continue
        z = B(r)
        rz_new = r @ z
        beta = rz_new / rz
        p = z + beta * p
        rz = rz_new
    r = c - apply_K(x)
    return x, it, MAXIT, np.linalg.norm(r) / cn
