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

Full-size fixtures (python tests/golden/make_golden.py full; minutes of
CPU): sampled outputs at the sizes of the benchmark workloads, which the
GPU tests compare with the library at those sizes.
  ct256_full.txt     256 x 256 CT (180 x 363 rays): one V(1,1) cycle and
                     the PCG solution at tol 1e-12 for lambda = 1, 0.05
                     with seeded weights; sampled entries, norms, rho, eta
  ct128_alg2.txt     Algorithm 2 on the 128 x 128 CT recipe at tol 1e-9:
                     the selected lambda indices
  deblur64_alg2.txt  Algorithm 2 on the 512 x 512 blur recipe's 64 x 64
                     form (19 x 19 PSF, its 24 lambdas >= 1e-4, at most 5
                     outer iterations) at tol 1e-9, right-hand sides 0, 1
  deblur512_solve.txt  512 x 512, 19 x 19 Gaussian sigma 3, 4 right-hand
                     sides, lambda = 0.05, 0.5, tol 1e-12, 6 levels
  deblur2048_ops.txt   2048 x 2048, 31 x 31 Gaussian sigma 5: K(lambda) p
                     and one V(1,1) cycle (10 levels) on seeded vectors
  ct256_vcycle16.txt, deblur2048_vcycle16.txt   the same cycles with the
                     smoother data stored in FP16 (oracle.multigrid,
                     storage="fp16"), the mixed path's one-lambda cycle
"""
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import problemgen as pg  # noqa: E402
from oracle import amg, krylov, lcurve, multigrid as mg, operators as ops, outer  # noqa: E402
import scipy.sparse as sp  # noqa: E402

# samples per full-size vector and their seed
N_SAMPLES = 512


def sample_index(n, seed):
    return np.sort(pg.rng(seed).choice(n, N_SAMPLES, replace=False))


def _vec_lines(tag, idx, v):
    return ["%s %.17g %s" % (tag, np.linalg.norm(v), " ".join("%.17g" % x for x in v[idx]))]


def _pcg(F, Lg, d, H, lam, c, tol):
    return krylov.pcg(lambda v: ops.normal_apply(F, Lg, d, lam, v), c, None, mg.VCycle(H, lam, nu=1), tol=tol,
                      maxit=50000)


def ct256_full():
    P = pg.make_problem("ct256")
    n = P.n
    F = ops.make_forward(P)
    Lg = ops.gradient(P.n_v, P.n_h)
    d = pg.random_weights(ops.n_edges(P.n_v, P.n_h), 41, d_min=0.05)
    levels = mg.default_levels(P.n_v, P.n_h)
    H = mg.build_hierarchy(mg.weighted_laplacian(Lg, d), sp.diags(F.diag_AtA()), P.n_v, P.n_h, levels)
    idx = sample_index(n, 43)
    r = pg.rng(42).standard_normal(n)
    c = ops.rhs(F, P.b[:, 0])
    lines = ["# ct256 (256 x 256, 180 x 363 rays): d = random_weights(n_edges, 41, d_min 0.05), levels %d," % levels,
             "# V(1,1) l1-Jacobi.  vcycle: B(lam) r for r = rng(42).standard_normal(n); solve: PCG from zero to",
             "# tol 1e-12 on b = the workload's b.  Lines: 'lam', then 'vcycle'/'x' with the norm and the values",
             "# at the sample indices (rng(43).choice(n, 512)), then 'rho_eta_its'.  Written by make_golden.py.",
             "idx " + " ".join(str(i) for i in idx)]
    for lam in (1.0, 0.05):
        z = mg.VCycle(H, lam, nu=1)(r)
        x, it, st, rel = _pcg(F, Lg, d, H, lam, c, 1e-12)
        assert st == 0, (lam, st, rel)
        rho, eta = lcurve.lcurve_values(F, Lg, d, P.b[:, 0], x)
        lines += ["lam %.17g" % lam] + _vec_lines("vcycle", idx, z) + _vec_lines("x", idx, x)
        lines.append("rho_eta_its %.17g %.17g %d" % (rho, eta, it))
        print("ct256", lam, it, flush=True)
    return lines


def deblur64_alg2():
    P = pg.make_problem("deblur512", size=64)
    lams = P.lambdas[8:]
    prm = outer.Params(nu=1, tol=1e-9, maxit=50000, levels=P.levels)
    lines = ["# Algorithm 2 on the deblur512 recipe at 64 x 64 (19 x 19 Gaussian sigma 3, zero boundary, %d" % P.levels,
             "# levels), the recipe's lambdas from the 9th on (%d lambdas, %.3g .. 1: the smaller ones do not reach" % (
                 len(lams), lams[0]),
             "# tol 1e-9 within 50,000 PCG iterations), V(1,1), tol 1e-9, three-equal stop, at most %d outer" % (
                 P.meta["max_outer"]),
             "# iterations, right-hand sides 0 and 1: the selected 1-based lambda indices per right-hand side."]
    for r in (0, 1):
        res = outer.lcurve_run(P, prm, rhs_index=r, max_outer=P.meta["max_outer"], lambdas=lams)
        lines.append("history %d " % r + " ".join(str(h) for h in res.history))
        for rec in res.records:
            kap = np.sort(lcurve.menger_curvature(rec.rho, rec.eta))[::-1]
            lines.append("kappa_top2 %d %.6g %.6g" % (r, kap[0], kap[1]))
            lines.append("iterations %d %s status %s" % (r, " ".join(str(int(v)) for v in rec.iters), " ".join(str(int(v)) for v in rec.status)))
        print("deblur64 history", r, res.history, flush=True)
    return lines


def ct128_alg2():
    P = pg.make_problem("ct256", size=128)
    prm = outer.Params(nu=1, tol=1e-9, maxit=50000)
    res = outer.lcurve_run(P, prm, max_outer=15)
    lines = ["# Algorithm 2 on the ct256 recipe at 128 x 128 (%d angles x %d bins), 20 lambdas" % (
                 round(180 * 128 / 256), P.A.m // round(180 * 128 / 256)),
             "# logspace(-4, 0), V(1,1), tol 1e-9, three-equal stop, max 15 outer iterations: the selected",
             "# 1-based lambda indices; then per outer iteration the two largest curvatures (near-tie check).",
             "history " + " ".join(str(h) for h in res.history)]
    for rec in res.records:
        kap = np.sort(lcurve.menger_curvature(rec.rho, rec.eta))[::-1]
        lines.append("kappa_top2 %.6g %.6g" % (kap[0], kap[1]))
    print("ct128 history", res.history, flush=True)
    return lines


def deblur512_solve():
    P = pg.make_problem("deblur512")
    n = P.n
    F = ops.make_forward(P)
    Lg = ops.gradient(P.n_v, P.n_h)
    d = pg.random_weights(ops.n_edges(P.n_v, P.n_h), 51, d_min=0.05)
    H = mg.build_hierarchy(mg.weighted_laplacian(Lg, d), sp.diags(F.diag_AtA()), P.n_v, P.n_h, P.levels)
    idx = sample_index(n, 53)
    lines = ["# deblur512 (512 x 512, 19 x 19 Gaussian sigma 3, 4 right-hand sides), d = random_weights(n_edges,",
             "# 51, d_min 0.05), %d levels, V(1,1), PCG from zero to tol 1e-12.  Lines 'case rhs lam', then" % P.levels,
             "# 'x' (norm, values at rng(53).choice(n, 512)) and 'rho_eta_its'.  Written by make_golden.py.",
             "idx " + " ".join(str(i) for i in idx)]
    for r in range(P.b.shape[1]):
        c = ops.rhs(F, P.b[:, r])
        for lam in (0.05, 0.5):
            x, it, st, rel = _pcg(F, Lg, d, H, lam, c, 1e-12)
            assert st == 0, (r, lam, st, rel)
            rho, eta = lcurve.lcurve_values(F, Lg, d, P.b[:, r], x)
            lines += ["case %d %.17g" % (r, lam)] + _vec_lines("x", idx, x)
            lines.append("rho_eta_its %.17g %.17g %d" % (rho, eta, it))
            print("deblur512", r, lam, it, flush=True)
    return lines


def deblur2048_ops():
    N = 2048
    psf = pg.gaussian_psf(15, 5.0)
    F = ops.ForwardPSF(psf, N, N)
    Lg = ops.gradient(N, N)
    n = N * N
    d = pg.random_weights(ops.n_edges(N, N), 61, d_min=0.05)
    idx = sample_index(n, 63)
    p = pg.rng(62).standard_normal(n)
    lines = ["# 2048 x 2048, 31 x 31 Gaussian sigma 5, d = random_weights(n_edges, 61, d_min 0.05).",
             "# 'apply lam': K(lam) p for p = rng(62).standard_normal(n); 'vcycle lam': one V(1,1) cycle of 10",
             "# levels on the same p.  Each: norm, then values at rng(63).choice(n, 512).  Written by make_golden.py.",
             "idx " + " ".join(str(i) for i in idx)]
    for lam in (1e-3, 0.1):
        q = ops.normal_apply(F, Lg, d, lam, p)
        lines += _vec_lines("apply %.17g" % lam, idx, q)
        print("deblur2048 apply", lam, flush=True)
    H = mg.build_hierarchy(mg.weighted_laplacian(Lg, d), sp.diags(F.diag_AtA()), N, N, 10)
    for lam in (1e-3, 0.1):
        z = mg.VCycle(H, lam, nu=1)(p)
        lines += _vec_lines("vcycle %.17g" % lam, idx, z)
        print("deblur2048 vcycle", lam, flush=True)
    return lines


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


def ct256_vcycle16():
    P = pg.make_problem("ct256")
    F = ops.make_forward(P)
    Lg = ops.gradient(P.n_v, P.n_h)
    d = pg.random_weights(ops.n_edges(P.n_v, P.n_h), 41, d_min=0.05)
    levels = mg.default_levels(P.n_v, P.n_h)
    H = mg.build_hierarchy(mg.weighted_laplacian(Lg, d), sp.diags(F.diag_AtA()), P.n_v, P.n_h, levels)
    idx = sample_index(P.n, 43)
    r = pg.rng(42).standard_normal(P.n)
    lines = ["# ct256 as ct256_full.txt: one V(1,1) cycle with the smoother data in FP16 (storage fp16).",
             "# Lines 'vcycle lam' with the norm and the values at the sample indices.  Written by make_golden.py.",
             "idx " + " ".join(str(i) for i in idx)]
    for lam in (1.0, 0.05):
        lines += _vec_lines("vcycle %.17g" % lam, idx, mg.VCycle(H, lam, nu=1, storage="fp16")(r))
    return lines


def deblur2048_vcycle16():
    N = 2048
    psf = pg.gaussian_psf(15, 5.0)
    F = ops.ForwardPSF(psf, N, N)
    Lg = ops.gradient(N, N)
    d = pg.random_weights(ops.n_edges(N, N), 61, d_min=0.05)
    idx = sample_index(N * N, 63)
    p = pg.rng(62).standard_normal(N * N)
    H = mg.build_hierarchy(mg.weighted_laplacian(Lg, d), sp.diags(F.diag_AtA()), N, N, 10)
    lines = ["# deblur2048 as deblur2048_ops.txt: one V(1,1) cycle (10 levels) with the smoother data in FP16",
             "# (storage fp16).  Lines 'vcycle lam', norm, values at the sample indices.  Written by make_golden.py.",
             "idx " + " ".join(str(i) for i in idx)]
    for lam in (1e-3, 0.1):
        lines += _vec_lines("vcycle %.17g" % lam, idx, mg.VCycle(H, lam, nu=1, storage="fp16")(p))
        print("deblur2048 vcycle16", lam, flush=True)
    return lines


FULL = {"ct256_full.txt": ct256_full, "ct128_alg2.txt": ct128_alg2, "deblur64_alg2.txt": deblur64_alg2,
        "deblur512_solve.txt": deblur512_solve,
        "deblur2048_ops.txt": deblur2048_ops, "ct256_vcycle16.txt": ct256_vcycle16,
        "deblur2048_vcycle16.txt": deblur2048_vcycle16}

if __name__ == "__main__":
    if len(sys.argv) > 1 and sys.argv[1] == "full":
        names = sys.argv[2:] or list(FULL)
        for name in names:
            lines = FULL[name]()  # computed first: a file appears only when complete
            with open(os.path.join(HERE, name), "w") as f:
                f.write("\n".join(lines) + "\n")
            print("wrote", name, flush=True)
        sys.exit(0)
    for name, fn in (("corners.txt", corners), ("windows.txt", windows), ("rs_amg_12x10.txt", rs_amg)):
        with open(os.path.join(HERE, name), "w") as f:
            f.write("\n".join(fn()) + "\n")
        print("wrote", name)
