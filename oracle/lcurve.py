"""Outer-loop ingredients (oracle; test infrastructure).

* lcurve_values: rho = ||A x - b||_2 and eta = ||D L x||_2, the coordinates
  (before the logarithm) of the L-curve point for x (Sec. 1).
* corner: the point of maximum positive curvature of the discrete L-curve
  (Sec. 1).  The paper does not give the discrete procedure; the reading
  used here is the signed Menger curvature of three consecutive points
  (log10 rho, log10 eta) taken in order of increasing lambda:
      kappa_i = 2 cross(P_i - P_{i-1}, P_{i+1} - P_i)
                / (|P_i - P_{i-1}| |P_{i+1} - P_i| |P_{i+1} - P_{i-1}|),
  positive where the curve turns from its steep leg to its flat leg.  The
  chosen index maximises kappa over interior points with kappa > 0 (ties,
  relative difference below 1e-12, go to the smaller lambda); with no
  positive kappa it maximises kappa over interior points.  Endpoints are
  never chosen.
* update_weights: eq. (g): g = |D L x| / ||D L x||_inf, d = 1 - g^q, and the
  new weights diag(d) D.  d is clamped below at d_min so the weights stay in
  (0, 1]; if D L x = 0 the weights are unchanged (d = 1, Sec. 3.4).
* lambda_window: the trimmed index range of Algorithm 2: all of 1..m at the
  first outer iteration, else [max(min(i-2, m-9), 1), min(max(i+7, 10), m)]
  (1-based, lambdas increasing).
* should_stop: Algorithm 2's outer stopping rule, three equal consecutive
  selected lambdas (Sec. 3.5).
"""
from __future__ import annotations

import numpy as np


def lcurve_values(F, L, d, b, x):
    rho = np.linalg.norm(F.matvec(x) - b)
    eta = np.linalg.norm(d * (L @ x))
    return rho, eta


def menger_curvature(rho, eta):
    u = np.log10(np.asarray(rho, dtype=np.float64))
    v = np.log10(np.asarray(eta, dtype=np.float64))
    k = len(u)
    kap = np.full(k, -np.inf)
    for i in range(1, k - 1):
        a = np.array([u[i] - u[i - 1], v[i] - v[i - 1]])
        b = np.array([u[i + 1] - u[i], v[i + 1] - v[i]])
        c = np.array([u[i + 1] - u[i - 1], v[i + 1] - v[i - 1]])
        cross = a[0] * b[1] - a[1] * b[0]
        den = np.linalg.norm(a) * np.linalg.norm(b) * np.linalg.norm(c)
        kap[i] = 2.0 * cross / den if den > 0 else 0.0
    return kap


def corner(rho, eta) -> int:
    """0-based index of the selected L-curve point (needs >= 3 points)."""
    k = len(rho)
    if k < 3:
        raise ValueError("the L-curve corner needs at least three points")
    kap = menger_curvature(rho, eta)
    interior = list(range(1, k - 1))
    pos = [i for i in interior if kap[i] > 0]
    cand = pos if pos else interior
    best = cand[0]
    for i in cand[1:]:
        # strictly larger by more than a relative 1e-12 -> take it;
        # otherwise keep the earlier (smaller lambda) index
        if kap[i] > kap[best] + 1e-12 * abs(kap[best]):
            best = i
    return best


def update_weights(d_prev, L, x, q=2.0, d_min=1e-3):
    """D^(l+1) = diag(d) D^(l) with d from eq. (g) evaluated on D^(l) L x."""
    v = d_prev * (L @ x)
    vmax = np.max(np.abs(v)) if v.size else 0.0
    if vmax == 0.0:
        return d_prev.copy()
    g = np.abs(v) / vmax
    d = np.maximum(1.0 - g ** q, d_min)
    return d * d_prev


def lambda_window(m: int, i_prev: int):
    """(lo, hi), 1-based inclusive; i_prev = 0 marks the first outer iteration."""
    if i_prev <= 0:
        return 1, m
    lo = max(min(i_prev - 2, m - 9), 1)
    hi = min(max(i_prev + 7, 10), m)
    return lo, hi


def should_stop(history) -> bool:
    """history: selected 1-based lambda indices, one per outer iteration."""
    return len(history) >= 3 and history[-1] == history[-2] == history[-3]


def should_stop_lx(lx_history) -> bool:
    """The heuristic of Gazzola et al. that Sec. 3.5 compares against: stop
    once ||L x^(*,l)||_2 has decreased from outer iteration l-1 to l.
    lx_history: ||L x*||_2 per outer iteration."""
    return len(lx_history) >= 2 and lx_history[-1] < lx_history[-2]
