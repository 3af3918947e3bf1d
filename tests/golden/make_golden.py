"""Writes the fixtures in this directory from the oracle alone (run from the
repository root: python tests/golden/make_golden.py).  Inputs come from the
seeded generators of problemgen; expected values only from oracle/.

  corners.txt        L-curve corner (Sec. 1; signed Menger curvature of
                     (log10 rho, log10 eta), the reading of oracle.lcurve)
                     of 30 seeded random L-curves
  windows.txt        the lambda window of Algorithm 2 for the paper's grid
                     of 30 lambdas (Sec. 4), every previous selection
  rs_amg_12x10.txt   classical AMG of Sec. 3.1 (theta = 0.25) on
                     L^T D^2 L of a 12 x 10 grid with seeded weights: the
                     C/F split and the interpolation P of the first level
"""
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import problemgen as pg  # noqa: E402
from oracle import amg, lcurve, multigrid as mg, operators as ops  # noqa: E402


def corners():
    g = pg.rng(2024)
    lines = ["# L-curve corner (Sec. 1): k, then rho_0..rho_{k-1}, eta_0..eta_{k-1} (increasing lambda),",
             "# then the oracle's corner index (0-based).  Written by tests/golden/make_golden.py."]
    for _ in range(30):
        k = int(g.integers(3, 21))
        rho = np.sort(10.0 ** g.uniform(-2, 3, k))
        eta = np.sort(10.0 ** g.uniform(-2, 3, k))[::-1]
        idx = lcurve.corner(rho, eta)
        lines.append(" ".join([str(k)] + ["%.17g" % v for v in rho] + ["%.17g" % v for v in eta] + [str(idx)]))
    return lines


def windows():
    m = 30
    lines = ["# Algorithm 2's lambda window for m = 30 lambdas (the grid of Sec. 4): i_prev lo hi",
             "# (1-based, inclusive; i_prev = 0 marks the first outer iteration).  Written by make_golden.py."]
    for i in range(0, m + 1):
        lo, hi = (1, m) if i == 0 else lcurve.lambda_window(m, i)
        lines.append("%d %d %d" % (i, lo, hi))
    return lines


def rs_amg():
    n_v, n_h = 12, 10
    d = pg.random_weights(ops.n_edges(n_v, n_h), 31, d_min=0.02)
    K = mg.weighted_laplacian(ops.gradient(n_v, n_h), d).tocsr()
    K.sort_indices()
    cf, S = amg.split(K)
    P = amg.interpolation(K, S, cf).tocsr()
    P.sort_indices()
    lines = ["# Classical AMG (Sec. 3.1, theta = 0.25) on L^T D^2 L, 12 x 10 grid,",
             "# d = problemgen.random_weights(n_edges, seed 31, d_min 0.02).  Written by make_golden.py.",
             "K %d %d" % (K.shape[0], K.nnz),
             "rp " + " ".join(str(v) for v in K.indptr),
             "ci " + " ".join(str(v) for v in K.indices),
             "v " + " ".join("%.17g" % v for v in K.data),
             "cf " + "".join(str(int(v)) for v in cf),
             "P %d %d %d" % (P.shape[0], P.shape[1], P.nnz),
             "prp " + " ".join(str(v) for v in P.indptr),
             "pci " + " ".join(str(v) for v in P.indices),
             "pv " + " ".join("%.17g" % v for v in P.data)]
    return lines


if __name__ == "__main__":
    for name, fn in (("corners.txt", corners), ("windows.txt", windows), ("rs_amg_12x10.txt", rs_amg)):
        with open(os.path.join(HERE, name), "w") as f:
            f.write("\n".join(fn()) + "\n")
        print("wrote", name)
