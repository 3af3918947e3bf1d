#!/usr/bin/env python
"""Throughput of multigrid-preconditioned CG on the regularized normal
equations (eq. (normal)) for the L-curve sweep of Algorithm 2.

Headline workload (the largest single-GPU problem): 2048 x 2048
deblurring, Gaussian PSF sigma 5 applied as a 31 x 31 separable stencil
with zero boundary, a piecewise-constant phantom with 2% noise, 64 lambdas
logspace(-6, 0).  Setup (untimed): the first outer iteration of Algorithm 2
(D = I, all 64 lambdas) gives the corner x*^(1) and, by one weight update
of eq. (g), D^(2).  One step = Algorithm 2's second outer iteration: the
hierarchy for D^(2), the trimmed window of 10 lambdas around the first
corner solved largest-first, each warm-started from the previous one (the
first from x*^(1)), to a relative normal-equations residual of 1e-6, the
L-curve values, the corner and the weight update.  The metric is
lambda-solves per second: systems that reached rel-res 1e-6, divided by
the wall time of the steps.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                  [--workload deblur2048|ct256]

--workload ct256 times Algorithm 2 end to end on the 256 x 256 CT matrix
(the previous headline).  Under torchrun each rank runs its own replica
(the right-hand sides differ by the noise draw); there is no collective on
the data path; the job's value is the lambda-solves of all ranks divided by
the slowest rank's time.  --impl reference times the CPU oracle instead.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "lambda-solves/s at rel-res 1e-6"
NU = 1  # V(nu, nu) sweeps: the library's default, and what the oracle arms run
DESC = {
    "deblur2048": ("deblur2048: 2048x2048 deblurring, Gaussian PSF sigma 5 as a 31x31 separable stencil (zero "
                   "boundary), piecewise-constant phantom (20 seeded rectangles/ellipses), 2% noise, 64 lambdas "
                   "logspace(-6, 0); D^(2) from one weight update (eq. (g), q = 2, d_min 1e-3) of the first "
                   "sweep's corner; one step = Algorithm 2's second outer iteration: hierarchy for D^(2), the "
                   "trimmed window of 10 lambdas, largest first, warm-started from the previous solution (the first "
                   "from x*^(1)), rel-res 1e-6, L-curve corner, weight update; 10-level V(1,1) l1-Jacobi"),
    "ct256": ("ct256: 256x256 parallel-beam CT, 180 angles x 363 bins exact ray-length CSR (FP32 values, int32 "
              "indices), 10 seeded ellipses, 1% noise, 20 lambdas logspace(-4, 0), Algorithm 2 (max 15 outer "
              "iterations, three-equal stop, largest-lambda-first warm-start chain), rel-res 1e-6, 5-level V(1,1) "
              "l1-Jacobi"),
}
SETUP_MAXIT = 1000  # the first sweep only draws D^(2) and the window: its small-lambda solves are capped
MAXIT = 10000
KERNEL_SRC = os.path.join(ROOT, "paper_2306_11067_gb300", "csrc", "kernels.cuh")
LAUNCH_SRC = os.path.join(ROOT, "paper_2306_11067_gb300", "csrc", "launch_spmm.cu")
TRAFFIC_FILE = os.path.join(ROOT, "profiles", "k_spmv1_ct256_traffic.txt")
CSRC = os.path.join(ROOT, "paper_2306_11067_gb300", "csrc")
# ncu DRAM records of the deblur2048 kernels: (file, source files whose
# contents the record is valid for)
RECORDS = {
    "k_band": (os.path.join(ROOT, "profiles", "k_band_deblur2048_traffic.txt"),
               ("separable.cuh", "separable.cu", "kernels.cuh", "common.cuh")),
    "vcycle": (os.path.join(ROOT, "profiles", "vcycle_deblur2048_traffic.txt"),
               ("vfine.cuh", "vcoarse.cuh", "vfused.cuh", "compact.cuh", "kernels.cuh", "launch_level.cu",
                "common.cuh")),
}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="deblur2048", choices=["deblur2048", "ct256"])
    ap.add_argument("--precision", default="mixed", choices=["mixed", "fp64"])
    ap.add_argument("--mode", default="sequential", choices=["sequential", "batched"])
    ap.add_argument("--no-plain", action="store_true", help="skip the plain FP64 comparison run")
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU oracle baseline")
    ap.add_argument("--oracle-sample", default=None, help=argparse.SUPPRESS)
    ap.add_argument("--no-serve", action="store_true", help="skip the served-mix latency leg")
    ap.add_argument("--no-rhs", action="store_true", help="skip the right-hand-side-batched 512^2 leg")
    ap.add_argument("--rhs-only", action="store_true", help="run only the right-hand-side-batched 512^2 leg")
    ap.add_argument("--serve-only", action="store_true",
                    help="only the served mix: --serve-requests per rate at each --serve-rates fraction of capacity")
    ap.add_argument("--serve-requests", type=int, default=200)
    ap.add_argument("--serve-rates", type=float, nargs="+", default=[0.5, 1.0, 1.5])
    ap.add_argument("--compare-precond", action="store_true",
                    help="time the lambda sweep of one outer iteration with the default preconditioner (FP64 and "
                         "mixed) and the paper's own (geometric and classical AMG interpolation, FP64) at 64^2, "
                         "128^2, 256^2 CT; one JSON line per arm, no bench line")
    ap.add_argument("--compare-algorithm2", action="store_true",
                    help="one full Algorithm 2 run of the CT workload per solver arm (default preconditioner mixed "
                         "and FP64, the paper's method with geometric P and with classical AMG split by the "
                         "paper's two passes or by PMIS): "
                         "lambda-solves/s and the selected lambda indices; one JSON line per arm")
    ap.add_argument("--profile-iters", type=int, default=0,
                    help="profiler workload: one lambda of the workload, this many PCG iterations, no JSON line")
    ap.add_argument("--profile-precond", type=int, default=0, choices=[0, 1, 2],
                    help="profiler workload's solver (ct256): 0 the default PCG (mixed), 1 the paper's method with "
                         "geometric P, 2 with classical AMG (FP64; --profile-iters FGMRES steps)")
    return ap.parse_args()


def host_info() -> dict:
    """CPU model and core count of this machine (for the CPU baselines)."""
    model = None
    try:
        for line in open("/proc/cpuinfo"):
            k = line.split(":")[0].strip().lower()
            if k in ("model name", "cpu model") and model is None:
                model = line.split(":", 1)[1].strip()
    except OSError:
        pass
    if model is None:
        try:
            out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
            for line in out.splitlines():
                if line.lower().startswith("model name"):
                    model = line.split(":", 1)[1].strip()
                    break
        except Exception:
            pass
    mem = None
    try:
        for line in open("/proc/meminfo"):
            if line.startswith("MemAvailable"):
                mem = int(line.split()[1]) * 1024
    except OSError:
        pass
    return {"cpu_model": model or "unknown", "nproc": os.cpu_count(), "mem_available_bytes": mem}


# ---------------------------------------------------------------------------
# CPU oracle samples (1-thread subprocesses; the reference arm)
# ---------------------------------------------------------------------------
def oracle_sample_2048(spec: dict) -> dict:
    """Time the oracle's pieces of one deblur2048 step on this machine's host
    cores: one application of K(lambda) = A^T A + lambda^2 L^T D^2 L (the
    2-D correlation with the 31 x 31 PSF and its transpose), the Galerkin
    hierarchy of 10 levels, the per-lambda V-cycle setup and one V(1,1)
    cycle.  The weights are read from spec['d'] (an .npy path) when given,
    else D = I: the cost does not depend on their values."""
    import numpy as np
    import scipy.sparse as sp
    import problemgen as pg
    from oracle import operators as ops
    from oracle import multigrid as mg
    P = pg.make_problem("deblur2048")
    F = ops.make_forward(P)
    Lg = ops.gradient(P.n_v, P.n_h)
    d = np.load(spec["d"]) if spec.get("d") else np.ones(ops.n_edges(P.n_v, P.n_h))
    lam = float(spec.get("lam", 0.01))
    x = pg.rng(5).standard_normal(P.n)
    t0 = time.perf_counter()
    ops.normal_apply(F, Lg, d, lam, x)
    t_k = time.perf_counter() - t0
    t0 = time.perf_counter()
    H = mg.build_hierarchy(mg.weighted_laplacian(Lg, d), sp.diags(F.diag_AtA()), P.n_v, P.n_h, P.levels)
    t_h = time.perf_counter() - t0
    t0 = time.perf_counter()
    V = mg.VCycle(H, lam, nu=NU)
    t_s = time.perf_counter() - t0
    t0 = time.perf_counter()
    V(x)
    t_v = time.perf_counter() - t0
    return dict(t_apply=t_k, t_hierarchy=t_h, t_vsetup=t_s, t_vcycle=t_v,
                threads=int(os.environ.get("OMP_NUM_THREADS", "1")))


def oracle_sample_ct256(budget_s: float, n_solves_max: int = 2) -> dict:
    """Time the oracle on the first outer iteration of the CT workload:
    solves from the largest lambda down, each warm-started from the previous
    one, until n_solves_max solves or the time budget is spent."""
    import numpy as np
    import problemgen as pg
    from oracle import outer
    from oracle import operators as ops
    P = pg.make_problem("ct256")
    prm = outer.Params(tol=1e-6, maxit=10000, nu=NU)
    t0 = time.perf_counter()
    S = outer.setup(P)
    c = ops.rhs(S.F, P.b[:, 0])
    d = np.ones(ops.n_edges(P.n_v, P.n_h))
    hier = outer.hierarchy(S, d, prm)
    t_setup = time.perf_counter() - t0
    its = 0
    solves = 0
    x = None
    t1 = time.perf_counter()
    for lam in P.lambdas[::-1]:
        x, it, st, _ = outer.solve(S, hier, d, c, lam, x, prm)
        its += it
        solves += int(st == 0)
        if solves >= n_solves_max or time.perf_counter() - t1 > budget_s:
            break
    t_solve = time.perf_counter() - t1
    return dict(solves=solves, iterations=its, solve_s=t_solve, setup_s=t_setup,
                threads=int(os.environ.get("OMP_NUM_THREADS", "1")))


def _oracle_env():
    env = dict(os.environ)
    for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        env[k] = "1"
    return env


def run_oracle_subprocess(spec: dict) -> dict:
    code = ("import json,sys; sys.path.insert(0, %r); import bench; "
            "print(json.dumps(bench.oracle_dispatch(json.loads(sys.argv[1]))))" % ROOT)
    out = subprocess.run([sys.executable, "-c", code, json.dumps(spec)], capture_output=True, text=True,
                         env=_oracle_env(), cwd=ROOT, timeout=1200)
    if out.returncode != 0:
        raise RuntimeError(out.stderr[-2000:])
    return json.loads(out.stdout.strip().splitlines()[-1])


def run_oracle_concurrent(spec: dict, procs: int) -> list:
    """procs 1-thread oracle samples at the same time (all cores busy)."""
    code = ("import json,sys; sys.path.insert(0, %r); import bench; "
            "print(json.dumps(bench.oracle_dispatch(json.loads(sys.argv[1]))))" % ROOT)
    ps = [subprocess.Popen([sys.executable, "-c", code, json.dumps(spec)], stdout=subprocess.PIPE,
                           stderr=subprocess.PIPE, text=True, env=_oracle_env(), cwd=ROOT) for _ in range(procs)]
    res = []
    for p in ps:
        out, err = p.communicate(timeout=1800)
        if p.returncode != 0:
            raise RuntimeError(err[-2000:])
        res.append(json.loads(out.strip().splitlines()[-1]))
    return res


def oracle_sample_small(spec: dict) -> dict:
    """The oracle on the 32 x 32 CSR blur case (9 x 9 PSF sigma 1.5 as an
    FP64 CSR matrix, lambda = 0.05, tol 1e-10, 3 levels): hierarchy and PCG
    solve from zero, timed whole, repeated for about a second."""
    import numpy as np
    import scipy.sparse as sp
    import problemgen as pg
    from oracle import operators as ops, multigrid as mg, krylov
    P = pg.make_problem("deblur32_csr")
    F = ops.ForwardCSR(P.A.to_scipy())
    Lg = ops.gradient(P.n_v, P.n_h)
    d = np.ones(ops.n_edges(P.n_v, P.n_h))
    lam = float(P.lambdas[0])
    n, its, t0 = 0, 0, time.perf_counter()
    while n < 3 or time.perf_counter() - t0 < 1.0:
        H = mg.build_hierarchy(mg.weighted_laplacian(Lg, d), sp.diags(F.diag_AtA()), P.n_v, P.n_h, P.levels)
        _, it, st, _ = krylov.pcg(lambda v: ops.normal_apply(F, Lg, d, lam, v), ops.rhs(F, P.b[:, 0]), None,
                                  mg.VCycle(H, lam, nu=NU), tol=P.tol, maxit=20000)
        n, its = n + 1, it
    return dict(seconds_per_solve=(time.perf_counter() - t0) / n, iterations=int(its), solves=n,
                threads=int(os.environ.get("OMP_NUM_THREADS", "1")))


def oracle_sample_512(spec: dict) -> dict:
    """The oracle's pieces on the 512 x 512 blur workload (19 x 19 PSF sigma 3,
    6 levels): one K(lambda) application, the hierarchy, one V-cycle setup
    and one V(1,1) cycle, with the weights of the right-hand-side leg."""
    import numpy as np
    import scipy.sparse as sp
    import problemgen as pg
    from oracle import operators as ops, multigrid as mg
    P = pg.make_problem("deblur512")
    F = ops.make_forward(P)
    Lg = ops.gradient(P.n_v, P.n_h)
    d = pg.random_weights(ops.n_edges(P.n_v, P.n_h), 52, d_min=0.05)
    lam = float(spec.get("lam", 0.01))
    x = pg.rng(5).standard_normal(P.n)
    t0 = time.perf_counter()
    ops.normal_apply(F, Lg, d, lam, x)
    t_k = time.perf_counter() - t0
    t0 = time.perf_counter()
    H = mg.build_hierarchy(mg.weighted_laplacian(Lg, d), sp.diags(F.diag_AtA()), P.n_v, P.n_h, P.levels)
    t_h = time.perf_counter() - t0
    t0 = time.perf_counter()
    V = mg.VCycle(H, lam, nu=NU)
    t_s = time.perf_counter() - t0
    t0 = time.perf_counter()
    V(x)
    t_v = time.perf_counter() - t0
    return dict(t_apply=t_k, t_hierarchy=t_h, t_vsetup=t_s, t_vcycle=t_v,
                threads=int(os.environ.get("OMP_NUM_THREADS", "1")))


def cpu_configs(device, rhs_leg):
    """The oracle, one thread, on the 32^2 CSR case (timed whole) and on the
    512^2 blur sweep of the right-hand-side leg (one right-hand side, the 32
    lambdas of one outer iteration: extrapolated from its timed pieces with
    the GPU one-column chain's iterations), beside the GPU's figures."""
    import numpy as np
    import problemgen as pg
    from paper_2306_11067_gb300 import lcmg as L
    out = {}
    try:
        o = run_oracle_subprocess({"kind": "small"})
        P = pg.make_problem("deblur32_csr")
        gpu = {}
        for prec, nm in ((L.PREC_FP64, "fp64"), (L.PREC_MIXED, "mixed")):
            sv = L.Solver(P.n_v, P.n_h, device=device, precision=prec, tol=P.tol, maxit=20000, levels=P.levels)
            sv.set_forward_csr(P.A)
            sv.solve(P.lambdas, P.b[:, 0])
            t0, n = time.perf_counter(), 0
            while n < 5 or time.perf_counter() - t0 < 0.5:
                r = sv.solve(P.lambdas, P.b[:, 0])
                n += 1
            gpu[nm] = {"solves_per_s": n / (time.perf_counter() - t0), "iterations": int(r["iters"][0, 0])}
            sv.close()
        out["deblur32_csr"] = {"workload": "32x32 blur, 9x9 PSF sigma 1.5 as FP64 CSR, lambda 0.05, tol 1e-10, "
                                           "3 levels, one solve from zero (hierarchy included)",
                               "oracle_solves_per_s_1thread": 1.0 / o["seconds_per_solve"],
                               "oracle_iterations": o["iterations"], "gpu": gpu}
    except Exception as ex:  # reported, not fatal
        out["deblur32_csr"] = {"failed": str(ex)}
    try:
        if rhs_leg and "one_column_chains" in rhs_leg:
            o = run_oracle_subprocess({"kind": "512"})
            its = float(np.mean(rhs_leg["iterations_per_rhs_one_column"]))
            t = its * (o["t_apply"] + o["t_vcycle"]) + 32 * o["t_vsetup"] + o["t_hierarchy"]
            out["deblur512_sweep"] = {
                "workload": "512x512 blur (19x19 PSF sigma 3), one right-hand side, the 32 lambdas of one outer "
                            "iteration in the chain",
                "oracle_lambda_solves_per_s_1thread": 32.0 / t, "kind": "extrapolation",
                "how": "oracle time per PCG iteration (one K application + one V-cycle) x the GPU one-column "
                       "chain's mean iterations per right-hand side (%.0f) + 32 V-cycle setups + one hierarchy"
                       % its,
                "timings_s": o,
                "gpu_one_column_lambda_solves_per_s": rhs_leg["one_column_chains"]["value"],
                "gpu_batched_lambda_solves_per_s": rhs_leg["batched"]["value"]}
    except Exception as ex:  # reported, not fatal
        out["deblur512_sweep"] = {"failed": str(ex)}
    return out


def oracle_dispatch(spec: dict) -> dict:
    if spec["kind"] == "deblur2048":
        return oracle_sample_2048(spec)
    if spec["kind"] == "small":
        return oracle_sample_small(spec)
    if spec["kind"] == "512":
        return oracle_sample_512(spec)
    return oracle_sample_ct256(float(spec.get("budget", 8.0)), int(spec.get("solves", 1)))


def oracle_rate_2048(o: dict, its_per_solve: float, window: int) -> float:
    """lambda-solves/s of the oracle on the step, extrapolated from its
    timed pieces: every lambda-solve takes its_per_solve PCG iterations (one
    K application and one V-cycle each) and its V-cycle setup; the hierarchy
    is built once per window of `window` solves."""
    per_solve = its_per_solve * (o["t_apply"] + o["t_vcycle"]) + o["t_vsetup"] + o["t_hierarchy"] / window
    return 1.0 / per_solve


# ---------------------------------------------------------------------------
# clocks during the timed region
# ---------------------------------------------------------------------------
class ClockSampler:
    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device: int):
        self.device = device
        self.proc = None
        self.path = os.path.join("/tmp", f"lcmg_clocks_{os.getpid()}.csv")

    def start(self):
        try:
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.device), f"--query-gpu={self.QUERY}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.f.close()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            p = [v.strip() for v in line.split(",")]
            if len(p) < 9:
                continue
            try:
                sm.append(float(p[1])); mx.append(float(p[2]))
            except ValueError:
                continue
            for nm, v in zip(names, p[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        os.unlink(self.path)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "samples": len(sm), "reasons": sorted(reasons)}


def measured_hbm_peak():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        return float(json.load(open(p))["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


def kernel_fingerprint():
    """sha256[:16] of the one-column SpMV kernel and of the launcher that
    picks its configuration: a recorded ncu traffic figure is only used
    while both are unchanged."""
    src = open(KERNEL_SRC).read()
    i = src.index("    k_spmv1(")
    j = src.index("\n}\n", i)
    lsrc = open(LAUNCH_SRC).read()
    a = lsrc.index("static int run1c(")
    b = lsrc.index("\n}\n", lsrc.index("static int run1(", a))
    return hashlib.sha256((src[i:j] + lsrc[a:b]).encode()).hexdigest()[:16]


def source_fingerprint(kind):
    """sha256[:16] over the source files a deblur2048 DRAM record covers."""
    h = hashlib.sha256()
    for name in RECORDS[kind][1]:
        h.update(open(os.path.join(CSRC, name), "rb").read())
    return h.hexdigest()[:16]


def recorded(kind):
    """The key: value pairs of a committed deblur2048 ncu record, if it was
    taken on the current sources; else None."""
    path = RECORDS[kind][0]
    if not os.path.exists(path):
        return None
    kv = {}
    for line in open(path):
        if ":" in line and not line.startswith("#"):
            k, v = line.split(":", 1)
            kv[k.strip()] = v.strip()
    if kv.get("source_sha256_16") != source_fingerprint(kind):
        return None
    return kv


def recorded_float(kind, key):
    kv = recorded(kind)
    try:
        return float(kv[key]) if kv else None
    except (KeyError, ValueError):
        return None


def recorded_traffic():
    """DRAM bytes per launch of the operator passes from the committed ncu
    summary, if it was taken on the current kernel source; else None."""
    if not os.path.exists(TRAFFIC_FILE):
        return None
    kv = {}
    for line in open(TRAFFIC_FILE):
        if ":" in line:
            k, v = line.split(":", 1)
            kv[k.strip()] = v.strip()
    if kv.get("k_spmv1_source_sha256_16") != kernel_fingerprint():
        return None
    try:
        return float(kv["dram_bytes_per_pass"])
    except (KeyError, ValueError):
        return None

# Served mix (the mixed blur and CT request stream, in the sizes that generate in

# Served mix (configs[3]'s request stream in the sizes that generate in
# seconds): 60% deblurring at 128^2, 256^2, 512^2, 1024^2 (PSF 9 x 9, sigma
# 1.5) and 40% CT at 128^2, 256^2, 512^2 (angles 0.7 x side, bins 1.42 x side;
# the 1024^2 CT matrix, ~1G nonzeros, takes minutes to generate on the host
# and is left out); each request a 16-lambda sweep logspace(-5, 0, 16) of its
# own seeded phantom at its own noise level U[0.5%, 5%], solved as the
# paper's warm-start chain (mixed precision, rel-res 1e-6), arriving as a
# seeded Poisson process at given fractions of the capacity measured on a
# burst of the same mix.
SERVE_CT = ((128, 90, 182), (256, 179, 364), (512, 358, 727))   # side, angles, bins
SERVE_BLUR = (128, 256, 512, 1024)                               # side; PSF 9 x 9, sigma 1.5
SERVE_SLOTS = 4
SERVE_MAXIT = 10000


def serving_leg(device, n_requests=40, rates=(1.0,)):
    """p50 / p99 latency (submit -> result) and throughput of the served
    mix, per arrival rate (a fraction of the burst capacity)."""
    import numpy as np
    import problemgen as pg
    from paper_2306_11067_gb300 import lcmg as L
    g = pg.rng(7)
    srv = L.Server(device=device, hbm_budget=96 << 30, slots=SERVE_SLOTS, precision=L.PREC_MIXED,
                   mode=L.MODE_SEQUENTIAL, tol=1e-6, maxit=SERVE_MAXIT)
    psf = pg.gaussian_psf(4, 1.5)
    probs = []  # (pid, kind, N, forward)
    t0 = time.perf_counter()
    for N, na, nb in SERVE_CT:
        A = pg.ct_csr(N, na, nb)
        probs.append((srv.add_csr(N, N, A), "ct", N, A.to_scipy()))
    for N in SERVE_BLUR:
        probs.append((srv.add_psf(N, N, psf), "blur", N, None))
    t_gen = time.perf_counter() - t0
    lams = np.logspace(-5, 0, 16)

    def make_request(k):
        ct = g.uniform() < 0.4
        cand = [p for p in probs if (p[1] == "ct") == ct]
        pid, kind, N, A = cand[int(g.integers(len(cand)))]
        img = pg.phantom_mixed(N, N, 10, 3000 + k, lo=0.1, hi=1.0)
        b = (A @ img.ravel(order="F")) if kind == "ct" else pg.blur_apply(img, psf).ravel(order="F")
        return pid, N, kind, pg.add_noise(b, float(g.uniform(0.005, 0.05)), 5000 + k)

    # capacity on a burst of 2 x slots requests
    burst = [make_request(k) for k in range(2 * SERVE_SLOTS)]
    t0 = time.perf_counter()
    tick = [srv.submit(pid, lams, b) for pid, _, _, b in burst]
    for t in tick:
        srv.wait(t)
    cap = len(burst) / (time.perf_counter() - t0)
    out = {"burst_capacity_per_s": cap, "slots": SERVE_SLOTS, "requests_per_rate": n_requests,
           "problem_setup_s": round(t_gen, 1), "rates": []}
    for ri, frac in enumerate(rates):
        rate = frac * cap
        reqs = [make_request(1000 * (ri + 1) + k) for k in range(n_requests)]
        gaps = g.exponential(1.0 / rate, n_requests)
        t0 = time.perf_counter()
        tick, t_next = [], t0
        for (pid, _, _, b), gap in zip(reqs, gaps):
            t_next += gap
            delay = t_next - time.perf_counter()
            if delay > 0:
                time.sleep(delay)
            tick.append(srv.submit(pid, lams, b))
        res = [srv.wait(t) for t in tick]
        wall = time.perf_counter() - t0
        lat = np.array([r["t_done"] - r["t_submit"] for r in res]) * 1e3
        full = np.array([r["n_converged"] == len(lams) for r in res])
        conv = int(sum(r["n_converged"] for r in res))
        lat_c = lat[full] if full.any() else lat
        out["rates"].append({
            "fraction_of_capacity": frac, "arrival_rate_per_s": rate,
            "p50_ms": float(np.percentile(lat_c, 50)), "p99_ms": float(np.percentile(lat_c, 99)),
            "p50_ms_all": float(np.percentile(lat, 50)), "p99_ms_all": float(np.percentile(lat, 99)),
            "lambda_solves_per_s": conv / wall, "converged_systems": conv, "systems": len(lams) * n_requests,
            "converged_fraction": conv / (len(lams) * n_requests),
            "requests_fully_converged": int(full.sum())})
    st = srv.stats()
    srv.close()
    out.update({"peak_running": st["peak_running"], "context_reuses": st["reuses"], "evictions": st["evictions"],
                "mix": "60% deblurring (128^2..1024^2, PSF 9x9 sigma 1.5) / 40% CT (128^2: 90x182 rays, 256^2: "
                       "179x364, 512^2: 358x727); 16 lambda = logspace(-5, 0, 16) per request, noise U[0.5%, 5%]; "
                       "seeded Poisson arrivals; the paper's warm-start chain, mixed precision, tol 1e-6, maxit "
                       + str(SERVE_MAXIT) + "; p50/p99 over fully converged requests (the _all values over all)"})
    return out


def profile_workload(args):
    """A short run for profiler captures: the workload's operator and
    hierarchy, one lambda (the middle of the grid) solved from zero for
    args.profile_iters PCG iterations (mixed precision, one column).  For
    deblur2048 the solver is the timed step's (same sizes, levels, kernels
    and launch shapes) with seeded stand-in edge weights in place of D^(2)."""
    import problemgen as pg
    from paper_2306_11067_gb300 import lcmg as L
    if args.workload == "deblur2048":
        P = pg.make_problem("deblur2048")
        prec = L.PREC_MIXED if args.precision == "mixed" else L.PREC_FP64
        s = L.Solver(P.n_v, P.n_h, precision=prec, mode=L.MODE_SEQUENTIAL, nu=NU, tol=1e-30,
                     maxit=args.profile_iters, levels=P.levels)
        s.set_forward_stencil(P.psf)
        s.set_weights(pg.random_weights(P.n_h * (P.n_v - 1) + (P.n_h - 1) * P.n_v, 3, d_min=0.05))
        lam = P.lambdas[len(P.lambdas) // 2: len(P.lambdas) // 2 + 1]
        s.solve(lam, P.b[:, 0])
        s.close()
        return
    P = pg.make_problem("ct256")
    kw = {0: dict(precision=L.PREC_MIXED),
          1: dict(precision=L.PREC_FP64, precond=1),
          2: dict(precision=L.PREC_FP64, precond=1, coarsening=1)}[args.profile_precond]
    s = L.Solver(P.n_v, P.n_h, mode=L.MODE_SEQUENTIAL, tol=1e-30, maxit=args.profile_iters, **kw)
    s.set_forward_csr(P.A)
    lam = P.lambdas[len(P.lambdas) // 2: len(P.lambdas) // 2 + 1]
    s.solve(lam, P.b[:, 0])
    s.close()


def compare_precond():
    """Sequential chain over the workload's lambdas (tol 1e-6, one
    right-hand side) for each preconditioner arm in FP64, and the default
    one in mixed precision (the benchmark's path): sweep time after a
    warm-up solve that builds the hierarchies, FGMRES / PCG steps, time per
    step."""
    import numpy as np
    import problemgen as pg
    from paper_2306_11067_gb300 import lcmg as L
    F64, MIX = L.PREC_FP64, L.PREC_MIXED
    arms = [("pcg-default", dict(precond=0, precision=F64)), ("paper-geometric", dict(precond=1, precision=F64)),
            ("paper-amg", dict(precond=1, coarsening=1, precision=F64)),
            ("paper-amg-pmis", dict(precond=1, coarsening=2, precision=F64)),
            ("pcg-default-mixed", dict(precond=0, precision=MIX))]
    for N in (64, 128, 256):
        P = pg.make_problem("ct256", size=None if N == 256 else N)
        b = P.b[:, 0]
        for name, kw in arms:
            s = L.Solver(N, N, mode=L.MODE_SEQUENTIAL, tol=1e-6, maxit=10000, **kw)
            s.set_forward_csr(P.A)
            t0 = time.perf_counter()
            s.solve(P.lambdas[-2:], b)
            t_warm = time.perf_counter() - t0
            t0 = time.perf_counter()
            out = s.solve(P.lambdas, b)
            dt = time.perf_counter() - t0
            st = s.stats()
            its = out["iters"][0]
            levels = (L.lcmg_amg_levels(s.ctx).tolist() if kw.get("coarsening") else L.lcmg_num_levels(s.ctx))
            print(json.dumps({"arm": name, "n": N, "precision": "fp64" if kw["precision"] == F64 else "mixed", "lambdas": int(len(P.lambdas)), "sweep_s": round(dt, 3),
                              "warmup_s": round(t_warm, 3), "steps": int(its.sum()),
                              "us_per_step": round(st["iterate_ms"] * 1e3 / max(st["batch_iterations"], 1), 1),
                              "status": sorted(set(int(v) for v in out["status"][0])), "levels": levels}),
                  flush=True)
            s.close()


def compare_algorithm2():
    """Algorithm 2 end to end on the workload (tol 1e-6, the paper's chain)
    with each solver arm: one untimed run, then one timed run (wall clock,
    the weights, hierarchies and every solve included)."""
    import problemgen as pg
    from paper_2306_11067_gb300 import lcmg as L
    P = pg.make_problem("ct256")
    b = P.b[:, 0]
    max_outer = P.meta.get("max_outer", 15)
    arms = [("pcg-default-mixed", dict(precond=0, precision=L.PREC_MIXED)),
            ("pcg-default-fp64", dict(precond=0, precision=L.PREC_FP64)),
            ("paper-geometric", dict(precond=1, precision=L.PREC_FP64)),
            ("paper-amg", dict(precond=1, coarsening=1, precision=L.PREC_FP64)),
            ("paper-amg-pmis", dict(precond=1, coarsening=2, precision=L.PREC_FP64))]
    for name, kw in arms:
        s = L.Solver(P.n_v, P.n_h, mode=L.MODE_SEQUENTIAL, tol=1e-6, maxit=10000, nu=NU, **kw)
        s.set_forward_csr(P.A)
        s.lcurve_run(P.lambdas, b, max_outer=max_outer)
        t0 = time.perf_counter()
        r = s.lcurve_run(P.lambdas, b, max_outer=max_outer)
        dt = time.perf_counter() - t0
        s.close()
        print(json.dumps({"arm": name, "workload": "ct256", "seconds": round(dt, 3),
                          "lambda_solves": int(r["n_converged"]), "lambda_solves_per_s": round(r["n_converged"] / dt, 3),
                          "outer_iterations": len(r["history"]), "selected_lambda_indices": [int(h) for h in r["history"]]}),
              flush=True)



def job_aggregate(conv: float, elapsed: float, world: int, device=None):
    """Whole-job totals of a replicas run: the converged lambda-solves of all
    ranks (sum) and the slowest rank's time (max), over the default process
    group (NCCL on GPUs, gloo on CPUs); a single rank returns its own."""
    if world <= 1:
        return float(conv), float(elapsed)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(conv), float(elapsed)], dtype=torch.float64, device=device)
    tot = t[:1].clone()
    dist.all_reduce(tot, op=dist.ReduceOp.SUM)
    mx = t[1:].clone()
    dist.all_reduce(mx, op=dist.ReduceOp.MAX)
    return float(tot[0]), float(mx[0])


def replica_rhs(P, rank: int):
    """Right-hand side of a rank's replica: the workload's own b on rank 0;
    the same operator and phantom with the rank's own noise draw elsewhere."""
    import problemgen as pg
    if rank == 0:
        return P.b[:, 0]
    return pg.add_noise(P.A.to_scipy() @ P.x_true[:, 0], P.meta["noise"], P.meta["noise_seed"] + 7919 * rank)




def rhs_batched_leg(device):
    """The right-hand-side-batched chain on the 512^2 workload (19 x 19 PSF,
    sigma 3, as a separable stencil; 4 seeded phantoms; 32 lambdas
    logspace(-5, 0); 6 levels; one outer iteration of Algorithm 2 with a
    seeded D shared by the four images): at each lambda, largest first,
    the four right-hand sides advance as one batch (B = 4, each column
    warm-started from its own previous-lambda solution), against four
    one-column chains on the same operator.  Mixed precision, rel-res 1e-6."""
    import numpy as np
    import problemgen as pg
    from paper_2306_11067_gb300 import lcmg as L
    P = pg.make_problem("deblur512")
    nrhs, nlam = P.b.shape[1], len(P.lambdas)
    d = pg.random_weights(P.n_h * (P.n_v - 1) + (P.n_h - 1) * P.n_v, 52, d_min=0.05)
    s = L.Solver(P.n_v, P.n_h, device=device, precision=L.PREC_MIXED, mode=L.MODE_SEQUENTIAL, nu=NU, tol=P.tol,
                 maxit=MAXIT, levels=P.levels, timing=1)
    s.set_forward_stencil(P.psf)
    s.set_weights(d)
    B = np.ascontiguousarray(P.b.T)
    s.solve(P.lambdas[-2:], B)  # warm-up: hierarchy, graphs
    t0 = time.perf_counter()
    out = s.solve(P.lambdas, B)
    t_b = time.perf_counter() - t0
    st_b = s.stats()  # the statistics of the last solve call
    its_b = out["iters"]
    conv_b = int((out["status"] == 0).sum())
    its_s = np.zeros_like(its_b)
    status_s = np.zeros_like(out["status"])
    conv_s = 0
    keys = ("vcycle_ms", "vcycle_count", "vcycle_bytes", "iterate_ms", "batch_iterations")
    st_s = {k: 0 for k in keys}
    t0 = time.perf_counter()
    for r in range(nrhs):
        o = s.solve(P.lambdas, B[r])
        its_s[r] = o["iters"][0]
        status_s[r] = o["status"][0]
        conv_s += int((o["status"][0] == 0).sum())
        st = s.stats()
        for k in keys:
            st_s[k] += st[k]
    t_s = time.perf_counter() - t0
    s.close()
    peak, _ = measured_hbm_peak()

    def vc(st):
        gbs = (st["vcycle_bytes"] / (st["vcycle_ms"] / 1e3) / 1e9) if st["vcycle_ms"] > 0 else None
        return {"us_per_cycle": st["vcycle_ms"] * 1e3 / max(st["vcycle_count"], 1), "gb_s": gbs,
                "frac_of_measured_hbm": gbs / peak if gbs else None,
                "us_per_pcg_iteration": st["iterate_ms"] * 1e3 / max(st["batch_iterations"], 1)}

    # per right-hand side: the iterations of the lambdas both forms brought
    # to the tolerance, batched against one-column
    both = (out["status"] == 0) & (status_s == 0)
    tot_b = np.where(both, its_b, 0).sum(axis=1)
    tot_s = np.where(both, its_s, 0).sum(axis=1)
    rel = np.abs(tot_b - tot_s) / np.maximum(tot_s, 1)
    return {"workload": "deblur512: 512x512, PSF 19x19 sigma 3 (separable), 4 phantoms, 1% noise, 32 lambdas "
                        "logspace(-5, 0), 6 levels, shared seeded D, rel-res 1e-6, mixed precision",
            "batched": {"value": conv_b / t_b, "unit": "lambda-solves/s", "seconds": t_b, "converged": conv_b,
                        "solves": nrhs * nlam, "pcg_iterations": int(its_b.sum()), "vcycle": vc(st_b)},
            "one_column_chains": {"value": conv_s / t_s, "unit": "lambda-solves/s", "seconds": t_s,
                                  "converged": conv_s, "pcg_iterations": int(its_s.sum()), "vcycle": vc(st_s)},
            "speedup": (conv_b / t_b) / (conv_s / t_s) if conv_s and t_b > 0 else None,
            "iterations_per_rhs_batched": tot_b.tolist(), "iterations_per_rhs_one_column": tot_s.tolist(),
            "lambdas_converged_in_both": int(both.sum()),
            "iterations_rel_diff_max": float(rel.max()),
            "iterations_batched": its_b.tolist(), "iterations_one_column": its_s.tolist()}


def fp64_peak(device: int):
    from paper_2306_11067_gb300 import lcmg as L
    try:
        return {"fp64_tflops": L.lcmg_fma_peak(device, L.PREC_FP64), "fp32_tflops": L.lcmg_fma_peak(device, L.PREC_MIXED),
                "how": "lcmg_fma_peak: 8 independent multiply-add chains per thread on every SM, best of 5 launches"}
    except Exception as ex:  # reported, not fatal
        return {"failed": str(ex)}


class Deblur2048:
    """The headline workload: setup (Algorithm 2's first outer iteration)
    and the timed step (its second outer iteration), through the C ABI."""

    def __init__(self, dev, local, stream, P, b):
        import numpy as np
        import torch
        from paper_2306_11067_gb300 import lcmg as L
        self.L, self.np, self.torch = L, np, torch
        self.dev, self.local, self.stream = dev, local, stream
        self.P = P
        self.n, self.ne = P.n, P.n_h * (P.n_v - 1) + (P.n_h - 1) * P.n_v
        self.m_lam = len(P.lambdas)
        with torch.cuda.stream(stream):
            self.b_dev = torch.tensor(b, dtype=torch.float64, device=dev).reshape(1, -1)
        stream.synchronize()
        self.b_host = b

    def solver(self, precision, timing):
        L = self.L
        s = L.Solver(self.P.n_v, self.P.n_h, device=self.local, stream=self.stream, precision=precision,
                     mode=L.MODE_SEQUENTIAL, nu=NU, tol=self.P.tol, maxit=MAXIT, levels=self.P.levels, timing=timing)
        s.set_forward_stencil(self.P.psf)
        return s

    def prepare(self, s):
        """Algorithm 2's first outer iteration (D = I, every lambda) with
        PCG capped at SETUP_MAXIT: its corner i1 and solution x*^(1), and
        D^(2) = the weight update of eq. (g) from x*^(1)."""
        L, torch = self.L, self.torch
        with torch.cuda.stream(self.stream):
            self.x1 = torch.empty(self.n, dtype=torch.float64, device=self.dev)
        s.set_params(maxit=SETUP_MAXIT)
        t0 = time.perf_counter()
        r = L.lcmg_lcurve_run_dev(s.ctx, self.P.lambdas, self.b_dev, 1, self.x1)
        self.setup_s = time.perf_counter() - t0
        self.setup_solves, self.setup_conv = r["n_solves"], r["n_converged"]
        self.i1 = int(r["history"][0])
        L.lcmg_update_weights_dev(s.ctx, self.x1, 2.0, 1e-3)
        self.d2 = L.lcmg_get_weights(s.ctx, self.ne)
        s.set_params(maxit=MAXIT)
        self.lo, self.hi = L.lcmg_cull_lambdas(self.m_lam, self.i1)
        self.lam_win = self.np.ascontiguousarray(self.P.lambdas[self.lo - 1:self.hi])
        k = len(self.lam_win)
        with torch.cuda.stream(self.stream):
            self.d2_dev = torch.tensor(self.d2, dtype=torch.float64, device=self.dev)
            self.x0 = torch.zeros(k, self.n, dtype=torch.float64, device=self.dev)
            self.x0[k - 1].copy_(self.x1)  # the chain starts at the window's largest lambda from x*^(1)
            self.x = torch.empty(k, self.n, dtype=torch.float64, device=self.dev)
            self.rho = torch.empty(1, k, dtype=torch.float64, device=self.dev)
            self.eta = torch.empty(1, k, dtype=torch.float64, device=self.dev)
            self.its = torch.empty(1, k, dtype=torch.int32, device=self.dev)
            self.st = torch.empty(1, k, dtype=torch.int32, device=self.dev)
        self.stream.synchronize()
        self.x0_host = self.x0.cpu().numpy()

    def step_dev(self, s):
        """One timed step with every input resident in device memory."""
        L = self.L
        L.lcmg_set_weights_dev(s.ctx, self.d2_dev, self.ne)
        L.lcmg_solve_dev(s.ctx, self.lam_win, self.b_dev, self.x, self.x0, self.rho, self.eta, self.its, self.st)
        stats = s.stats()
        rho, eta = self.rho.cpu().numpy()[0], self.eta.cpu().numpy()[0]
        st, its = self.st.cpu().numpy()[0], self.its.cpu().numpy()[0]
        sel = self.lo + L.lcmg_lcurve_corner(rho, eta)
        L.lcmg_update_weights_dev(s.ctx, self.x[sel - self.lo], 2.0, 1e-3)
        return {"converged": int((st == 0).sum()), "solves": len(st), "iterations": int(its.sum()),
                "selected": int(sel), "its": [int(v) for v in its], "stats": stats}

    def step_host(self, s, d2_pin, b_pin, x0_pin):
        """The same step through the host-pointer calls (inputs copied in
        from pinned host memory, the solutions and the new weights read back)."""
        L = self.L
        L.lcmg_set_weights(s.ctx, d2_pin)
        out = L.lcmg_solve(s.ctx, self.lam_win, b_pin, x0_pin)
        sel = self.lo + L.lcmg_lcurve_corner(out["rho"][0], out["eta"][0])
        L.lcmg_update_weights(s.ctx, out["x"][0, sel - self.lo], 2.0, 1e-3, self.ne)
        return int((out["status"][0] == 0).sum())

    def bytes_host(self):
        k = len(self.lam_win)
        h2d = self.ne * 8 + self.n * 8 + k * self.n * 8 + self.n * 8
        d2h = k * self.n * 8 + k * (8 + 8 + 4 + 4) + self.ne * 8
        return h2d, d2h


def main_deblur(args, world, rank, local):
    import numpy as np
    import torch
    import torch.distributed as dist
    import problemgen as pg
    from paper_2306_11067_gb300 import lcmg as L

    if world > 1:
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    stream = torch.cuda.Stream(device=dev)
    P = pg.make_problem("deblur2048")
    b = P.b[:, 0] if rank == 0 else pg.add_noise(pg.vec(pg.blur_apply(pg.unvec(P.x_true[:, 0], P.n_v, P.n_h), P.psf)),
                                                 P.meta["noise"], P.meta["noise_seed"] + 7919 * rank)
    W = Deblur2048(dev, local, stream, P, b)
    prec = L.PREC_MIXED if args.precision == "mixed" else L.PREC_FP64
    solver = W.solver(prec, 1)
    W.prepare(solver)
    levels = L.lcmg_num_levels(solver.ctx)

    for _ in range(args.warmup):
        W.step_dev(solver)

    # ---------------- timed region (inputs resident in HBM) ---------------
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize(dev)
    clk = ClockSampler(local)
    clk.start()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    t0 = time.perf_counter()
    results = [W.step_dev(solver) for _ in range(args.steps)]
    e1.record(stream)
    torch.cuda.synchronize(dev)
    wall = time.perf_counter() - t0
    if world > 1:
        dist.barrier()
    clocks = clk.stop()
    dev_ms = e0.elapsed_time(e1)
    elapsed = max(dev_ms / 1e3, wall)
    conv = sum(r["converged"] for r in results)
    solves = sum(r["solves"] for r in results)
    col_its = sum(r["iterations"] for r in results)
    st = [r["stats"] for r in results]
    launches = sum(s_["kernel_launches"] for s_ in st)
    conv_all, elapsed_all = job_aggregate(conv, elapsed, world, dev)
    value = conv_all / elapsed_all

    # ---------------- end to end through the host API ---------------------
    h2d, d2h = W.bytes_host()
    d2_pin = torch.empty(W.ne, dtype=torch.float64, pin_memory=True)
    d2_pin.copy_(torch.from_numpy(W.d2))
    b_pin = torch.empty((1, P.n), dtype=torch.float64, pin_memory=True)
    b_pin.copy_(torch.from_numpy(np.ascontiguousarray(b)).reshape(1, -1))
    x0_pin = torch.empty(W.x0.shape, dtype=torch.float64, pin_memory=True)
    x0_pin.copy_(torch.from_numpy(W.x0_host))
    e2e_conv, e2e_t = 0, 0.0
    for _ in range(max(1, min(args.steps, 3))):
        t1 = time.perf_counter()
        e2e_conv += W.step_host(solver, d2_pin.numpy(), b_pin.numpy(), x0_pin.numpy())
        e2e_t += time.perf_counter() - t1
    e2e_value = e2e_conv / e2e_t * (conv_all / max(conv, 1))

    # ---------------- rooflines of the operator passes and the V-cycle ----
    peak, peak_kind = measured_hbm_peak()
    op_ms = sum(s_["op_ms_a"] + s_["op_ms_at"] for s_ in st)
    op_launches = sum(s_["op_launches"] for s_ in st)
    op_bytes = sum(s_["op_bytes"] for s_ in st)
    v_ms = sum(s_["vcycle_ms"] for s_ in st)
    v_cnt = sum(s_["vcycle_count"] for s_ in st)
    v_bytes = sum(s_["vcycle_bytes"] for s_ in st)
    it_ms = sum(s_["iterate_ms"] for s_ in st)
    b_its = sum(s_["batch_iterations"] for s_ in st)
    band = {
        "kernel": "k_band (separable A^T A: u = (I (x) T_v) p along i, then q = (T_h (x) I) u + lam^2 L^T W L p "
                  "with p.q along j; 61 taps each, FP32)",
        "bound": "hbm", "unit": "GB/s", "peak": peak, "peak_source": f"{peak_kind} (MEASURED_PEAKS.json hbm_gbs)",
        "achieved": (op_bytes / (op_ms / 1e3) / 1e9) if op_ms > 0 else None,
        "algorithmic_bytes_per_apply": (op_bytes * 2 / op_launches) if op_launches else None,
        "avg_us_pass_v": (sum(s_["op_ms_a"] for s_ in st) * 2e3 / op_launches) if op_launches else None,
        "avg_us_pass_h": (sum(s_["op_ms_at"] for s_ in st) * 2e3 / op_launches) if op_launches else None,
        "fp32_gflop_per_apply": 2.0 * P.n * 2 * 61 / 1e9,
        "share_of_iteration_time": ((op_ms * 2 / op_launches) * b_its / it_ms) if (it_ms > 0 and op_launches) else None,
        "traffic": recorded_float("k_band", "dram_bytes_per_apply") if prec == L.PREC_MIXED else None,
        "traffic_unit": "DRAM bytes per apply (both passes), ncu, profiles/k_band_deblur2048_traffic.txt",
    }
    band["frac"] = band["achieved"] / peak if band["achieved"] else None
    vcyc = {
        "kernel": "V(1,1) cycle, 10 levels: k_vdown / k_vup per level (FP16 smoother data) + k_coarse_solve",
        "bound": "hbm", "unit": "GB/s", "peak": peak, "peak_source": f"{peak_kind} (MEASURED_PEAKS.json hbm_gbs)",
        "achieved": (v_bytes / (v_ms / 1e3) / 1e9) if v_ms > 0 else None,
        "algorithmic_bytes_per_cycle": (v_bytes / v_cnt) if v_cnt else None,
        "avg_us_per_cycle": (v_ms * 1e3 / v_cnt) if v_cnt else None,
        "share_of_iteration_time": ((v_ms / v_cnt) * b_its / it_ms) if (it_ms > 0 and v_cnt) else None,
        "traffic": recorded_float("vcycle", "dram_bytes_per_cycle") if prec == L.PREC_MIXED else None,
        "traffic_unit": "DRAM bytes per cycle (all its kernels), ncu, profiles/vcycle_deblur2048_traffic.txt",
    }
    vrec = recorded("vcycle") if prec == L.PREC_MIXED else None
    if vrec:  # per-level DRAM GB/s of the cycle's kernels (ncu, cold cache, serialised)
        vcyc["levels_ncu"] = {k[len("level_"):]: v for k, v in vrec.items() if k.startswith("level_")}
    vcyc["frac"] = vcyc["achieved"] / peak if vcyc["achieved"] else None
    dominant, other = (vcyc, band) if (vcyc["share_of_iteration_time"] or 0) >= (band["share_of_iteration_time"] or 0) \
        else (band, vcyc)

    # ---------------- plain FP64 one-lambda-at-a-time comparison ----------
    plain = None
    if not args.no_plain and rank == 0:
        ps = W.solver(L.PREC_FP64, 1)
        W.step_dev(ps)  # warm-up
        torch.cuda.synchronize(dev)
        t1 = time.perf_counter()
        rp = W.step_dev(ps)
        torch.cuda.synchronize(dev)
        tp = time.perf_counter() - t1
        s64 = rp["stats"]
        ob = s64["op_bytes"]
        plain = {"value": rp["converged"] / tp, "unit": "lambda-solves/s", "precision": "fp64", "mode": "sequential",
                 "step_s": tp, "converged": rp["converged"], "pcg_iterations": rp["iterations"],
                 "us_per_iteration": s64["iterate_ms"] * 1e3 / max(s64["batch_iterations"], 1),
                 "avg_us_pass_v": s64["op_ms_a"] * 2e3 / max(s64["op_launches"], 1),
                 "avg_us_pass_h": s64["op_ms_at"] * 2e3 / max(s64["op_launches"], 1),
                 "fp64_gflop_per_apply": 2.0 * P.n * 2 * 61 / 1e9, "selected": rp["selected"]}
        ps.close()

    # ---------------- CPU oracle baseline (rank 0, N = 1 only) ------------
    cpu = None
    its_per_solve = col_its / max(conv, 1)
    if rank == 0 and world == 1 and not args.no_cpu:
        cpu = cpu_baseline_2048(W, its_per_solve)

    serving = None
    if rank == 0 and world == 1 and not args.no_serve:
        try:
            serving = serving_leg(local)
        except Exception as ex:  # reported, not fatal
            serving = {"failed": str(ex)}

    rhs_batched = None
    if rank == 0 and world == 1 and not args.no_rhs:
        try:
            rhs_batched = rhs_batched_leg(local)
        except Exception as ex:  # reported, not fatal
            rhs_batched = {"failed": str(ex)}
    cpu_cfg = None
    if rank == 0 and world == 1 and not args.no_cpu:
        cpu_cfg = cpu_configs(local, rhs_batched)

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": "lambda-solves/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": elapsed_all * 1e3 / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32 (f16 smoother data; f64 dots, recurrences, true residuals, coarse solve)"
            if prec == L.PREC_MIXED else "f64",
            "data": "synthetic (seeded piecewise-constant phantom, Gaussian blur, Gaussian noise)",
            "config": {"workload": DESC["deblur2048"], "precision": args.precision, "levels": levels,
                       "parallelism": f"replicas x{world}" if world > 1 else "single GPU",
                       "l2": "inputs larger than L2 (the 10 window solutions and warm starts: 671 MB; one FP64 "
                             "vector 33.5 MB, the FP32 iteration's vectors and smoother data 150 MB)",
                       "first_sweep": {"corner": W.i1, "solves": W.setup_solves, "converged": W.setup_conv,
                                       "maxit": SETUP_MAXIT, "seconds": round(W.setup_s, 2)},
                       "window": [W.lo, W.hi], "lambda_solves_per_step": conv / args.steps,
                       "systems_per_step": solves / args.steps, "pcg_iterations_per_step": col_its / args.steps,
                       "iterations_per_lambda": results[-1]["its"],
                       "selected_lambda_index": results[-1]["selected"],
                       "us_per_pcg_iteration": it_ms * 1e3 / max(b_its, 1)},
            "e2e": {"value": e2e_value, "unit": "lambda-solves/s", "h2d_bytes_per_step": h2d,
                    "d2h_bytes_per_step": d2h},
            "gpu_launches": launches,
            "roofline": dominant,
            "roofline_other": other,
            "cpu_baseline": cpu,
            "plain_fp64": plain,
            "fma_peaks": fp64_peak(local) if rank == 0 else None,
            "serving": serving,
            "rhs_batched_512": rhs_batched,
            "cpu_baseline_configs": cpu_cfg,
            "clocks": clocks,
        }
        print(json.dumps(line))
    solver.close()
    if world > 1:
        dist.destroy_process_group()


def cpu_baseline_2048(W, its_per_solve):
    """The oracle's pieces timed on one core and on every core at once
    (independent processes), extrapolated to the step's lambda-solves/s."""
    import numpy as np
    hi = host_info()
    res = {"unit": "lambda-solves/s", "kind": "oracle", **hi}
    try:
        with tempfile.NamedTemporaryFile(suffix=".npy", delete=False) as f:
            path = f.name
        np.save(path, W.d2)
        spec = {"kind": "deblur2048", "d": path, "lam": float(W.lam_win[-1])}
        o = run_oracle_subprocess(spec)
        window = len(W.lam_win)
        v1 = oracle_rate_2048(o, its_per_solve, window)
        res.update({"value": v1, "cores": 1, "timings_s": o,
                    "sample": ("oracle (scipy 2-D correlation with the 31x31 PSF, sparse Galerkin hierarchy, V(1,1)) "
                               "on the same 2048x2048 workload and D^(2), 1 thread: one K(lambda) application, the "
                               "10-level hierarchy, one V-cycle setup and one V-cycle, timed; extrapolated to "
                               "lambda-solves/s with this run's %.1f PCG iterations per converged lambda-solve and "
                               "one hierarchy per window of %d lambdas" % (its_per_solve, window))})
        procs = hi["nproc"] or 1
        if hi["mem_available_bytes"]:
            procs = max(1, min(procs, int(hi["mem_available_bytes"] // (6 << 30))))
        t0 = time.perf_counter()
        many = run_oracle_concurrent(spec, procs)
        wall = time.perf_counter() - t0
        rates = [oracle_rate_2048(m, its_per_solve, window) for m in many]
        res["all_cores"] = {"value": sum(rates), "cores": procs, "processes": procs, "wall_s": wall,
                            "sample": "the same sample in %d concurrent 1-thread processes (independent lambda "
                                      "solves on every core); value = the sum of their extrapolated rates" % procs}
        os.unlink(path)
    except Exception as ex:  # reported, not fatal
        res.update({"value": None, "cores": 1, "sample": f"failed: {ex}"})
    return res


def main_ct256(args, world, rank, local):
    """Algorithm 2 end to end on the 256 x 256 CT workload (one step = one
    full run: weights, hierarchies, every window's chain, corners, weight
    updates and the three-equal stop)."""

    import numpy as np
    import torch
    import torch.distributed as dist
    import problemgen as pg
    from paper_2306_11067_gb300 import lcmg as L

    if world > 1:
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    stream = torch.cuda.Stream(device=dev)

    P = pg.make_problem("ct256")
    b = replica_rhs(P, rank)
    n, m = P.n, P.m
    prec = L.PREC_MIXED if args.precision == "mixed" else L.PREC_FP64
    mode = L.MODE_SEQUENTIAL if args.mode == "sequential" else L.MODE_BATCHED
    max_outer = P.meta.get("max_outer", 15)

    def make_solver(precision, timing, md=mode):
        s = L.Solver(P.n_v, P.n_h, device=local, stream=stream, precision=precision, mode=md, nu=NU,
                     tol=1e-6, maxit=10000, timing=timing)
        s.set_forward_csr(P.A)
        return s

    solver = make_solver(prec, 1)
    levels = L.lcmg_num_levels(solver.ctx)
    with torch.cuda.stream(stream):
        b_dev = torch.tensor(b, dtype=torch.float64, device=dev)
        x_dev = torch.empty(n, dtype=torch.float64, device=dev)
    stream.synchronize()

    def step():
        r = L.lcmg_lcurve_run_dev(solver.ctx, P.lambdas, b_dev, max_outer, x_dev)
        return r, solver.stats()

    for _ in range(args.warmup):
        step()

    # ---------------- timed region (inputs resident in HBM) ---------------
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize(dev)
    clk = ClockSampler(local)
    clk.start()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    t0 = time.perf_counter()
    results = [step() for _ in range(args.steps)]
    e1.record(stream)
    torch.cuda.synchronize(dev)
    wall = time.perf_counter() - t0
    if world > 1:
        dist.barrier()
    clocks = clk.stop()
    dev_ms = e0.elapsed_time(e1)
    elapsed = max(dev_ms / 1e3, wall)  # the steps synchronise; both clocks agree closely
    conv = sum(r["n_converged"] for r, _ in results)
    solves = sum(r["n_solves"] for r, _ in results)
    col_its = sum(s["column_iterations"] for _, s in results)
    launches = sum(s["kernel_launches"] for _, s in results)
    op_ms = sum(s["op_ms_a"] + s["op_ms_at"] for _, s in results)
    op_ms_a = sum(s["op_ms_a"] for _, s in results)
    op_ms_at = sum(s["op_ms_at"] for _, s in results)
    op_launches = sum(s["op_launches"] for _, s in results)
    op_bytes = sum(s["op_bytes"] for _, s in results)
    batch_its = sum(s["batch_iterations"] for _, s in results)
    history = results[-1][0]["history"]

    # whole-job aggregate over ranks
    conv_all, elapsed_all = job_aggregate(conv, elapsed, world, dev)
    value = conv_all / elapsed_all

    # ---------------- end to end through the host API ---------------------
    b_pin = torch.empty(m, dtype=torch.float64, pin_memory=True)
    b_pin.copy_(torch.from_numpy(b))
    b_host = b_pin.numpy()
    e2e_conv, e2e_t = 0, 0.0
    for _ in range(max(1, min(args.steps, 3))):
        t1 = time.perf_counter()
        r = solver.lcurve_run(P.lambdas, b_host, max_outer=max_outer)
        e2e_t += time.perf_counter() - t1
        e2e_conv += r["n_converged"]
    e2e_value = e2e_conv / e2e_t * (conv_all / max(conv, 1))  # other ranks run the same

    # ---------------- plain FP64 one-lambda-at-a-time comparison ----------
    plain = None
    if not args.no_plain and rank == 0:
        ps = make_solver(L.PREC_FP64, 0, L.MODE_SEQUENTIAL)
        L.lcmg_lcurve_run_dev(ps.ctx, P.lambdas, b_dev, max_outer, x_dev)  # warm-up
        t1 = time.perf_counter()
        rp = L.lcmg_lcurve_run_dev(ps.ctx, P.lambdas, b_dev, max_outer, x_dev)
        tp = time.perf_counter() - t1
        plain = {"value": rp["n_converged"] / tp, "unit": "lambda-solves/s", "precision": "fp64",
                 "mode": "sequential", "history": [int(h) for h in rp["history"]],
                 "column_iterations": ps.stats()["column_iterations"]}
        ps.close()

    # ---------------- roofline of the dominant kernel ---------------------
    peak, peak_kind = measured_hbm_peak()
    # algorithmic bytes of one apply by the per-nonzero count of the matrix
    # in CSR (8 B: FP32 value + int32 column, both passes) plus the vectors:
    # 2 * 8 nnz + 2 s (m + n) for s = 4 (FP32) vectors
    sv = 4 if args.precision == "mixed" else 8
    bytes_8b_apply = 2 * 8 * P.A.nnz + 2 * sv * (P.A.m + P.A.n)
    apply_s = (op_ms * 2 / op_launches / 1e3) if op_launches else None
    achieved = (bytes_8b_apply / apply_s / 1e9) if apply_s else None
    achieved_stored = (op_bytes / (op_ms / 1e3) / 1e9) if op_ms > 0 else None
    roofline = {
        "kernel": (("k_spmv1 (the one-column SpMV, both operator passes: y = A p with int32 columns, then "
                    "q = A^T y + lam^2 L^T W L p with p.q and 16-bit column offsets)")
                   if mode == L.MODE_SEQUENTIAL
                   else "k_spmm (the batched SpMM, both operator passes over the active columns)"),
        "bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
        "frac": (achieved / peak) if achieved else None, "peak_source": f"{peak_kind} (MEASURED_PEAKS.json hbm_gbs)",
        "algorithmic_bytes_per_apply": bytes_8b_apply,
        "bytes_basis": "8 B per nonzero and pass (FP32 value + int32 column) + 2 s (m + n)",
        "achieved_stored_format": achieved_stored,
        "stored_format_note": "GB/s by the bytes the passes read as stored (16-bit column offsets in the "
                              "transposed pass: 6 B per nonzero)",
        "traffic": recorded_traffic() if mode == L.MODE_SEQUENTIAL else None,
        "stored_bytes_per_pass": (op_bytes / op_launches) if op_launches else None,
        "avg_pass_us": (op_ms * 1e3 / op_launches) if op_launches else None,
        "avg_us_A": (op_ms_a * 2e3 / op_launches) if op_launches else None,
        "avg_us_At": (op_ms_at * 2e3 / op_launches) if op_launches else None,
        # the passes are timed on a sample of the iterations: scale the mean
        # per-iteration time by every iteration of the timed steps
        "share_of_device_time": ((op_ms * 2 / op_launches) * batch_its / dev_ms)
        if (dev_ms > 0 and op_launches) else None,
    }

    # ---------------- CPU oracle baseline (rank 0, N = 1 only) ------------
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu:
        try:
            o = run_oracle_subprocess({"kind": "ct256", "budget": 20.0, "solves": 2})
            it_rate = o["iterations"] / o["solve_s"]
            solves_per_it = conv / max(col_its, 1)
            cpu = {"value": it_rate * solves_per_it, "unit": "lambda-solves/s", "cores": o["threads"],
                   "kind": "oracle",
                   "sample": ("oracle PCG (scipy CSR, 1 thread) on the same ct256 workload: the first %d solves "
                              "of the first outer iteration's largest-first chain (%d PCG iterations in %.1f s); "
                              "iterations/s scaled by this run's lambda-solves per PCG iteration (%d / %d)"
                              % (o["solves"], o["iterations"], o["solve_s"], conv, col_its)),
                   "sample_solves_per_s": o["solves"] / o["solve_s"]}
        except Exception as ex:  # reported, not fatal
            cpu = {"value": None, "unit": "lambda-solves/s", "cores": 1, "kind": "oracle", "sample": f"failed: {ex}"}

    # ---------------- served mix: p50 / p99 latency (rank 0, N = 1) -------
    serving = None
    if rank == 0 and world == 1 and not args.no_serve:
        try:
            serving = serving_leg(local)
        except Exception as ex:  # reported, not fatal
            serving = {"failed": str(ex)}

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": "lambda-solves/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": elapsed_all * 1e3 / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32 (f64 dots, recurrences, true residuals, coarse solve)" if prec == L.PREC_MIXED else "f64",
            "data": "synthetic (seeded phantoms, ray-length CT matrix, Gaussian noise)",
            "config": {"workload": DESC["ct256"], "precision": args.precision, "mode": args.mode,
                       "levels": levels, "parallelism": f"replicas x{world}" if world > 1 else "single GPU",
                       "l2": "inputs larger than L2 (A and A^T CSR: 240 MB per operator application)",
                       "lambda_solves_per_step": conv / args.steps, "systems_per_step": solves / args.steps,
                       "pcg_iterations_per_step": col_its / args.steps,
                       "selected_lambda_indices": [int(h) for h in history]},
            "e2e": {"value": e2e_value, "unit": "lambda-solves/s", "h2d_bytes_per_step": m * 8,
                    "d2h_bytes_per_step": n * 8 + 4 * max_outer},
            "gpu_launches": launches,
            "roofline": roofline,
            "cpu_baseline": cpu,
            "plain_fp64": plain,
            "serving": serving,
            "clocks": clocks,
        }
        print(json.dumps(line))
    solver.close()
    if world > 1:
        dist.destroy_process_group()



# measured on GB300 by this benchmark (its config.pcg_iterations_per_step /
# lambda_solves_per_step: 1,184 / 10): the reference arm's extrapolation to
# lambda-solves
REF_ITS_PER_SOLVE = 118.4


def oracle_steps_2048(spec: dict) -> dict:
    """The reference arm's samples: the oracle's hierarchy and V-cycle setup
    once, then spec['n'] samples of one PCG iteration's work (one K(lambda)
    application and one V(1,1) cycle), each timed."""
    import numpy as np
    import scipy.sparse as sp
    import problemgen as pg
    from oracle import operators as ops
    from oracle import multigrid as mg
    P = pg.make_problem("deblur2048")
    F = ops.make_forward(P)
    Lg = ops.gradient(P.n_v, P.n_h)
    d = np.ones(ops.n_edges(P.n_v, P.n_h))
    lam = float(spec.get("lam", 0.01))
    x = pg.rng(5).standard_normal(P.n)
    t0 = time.perf_counter()
    H = mg.build_hierarchy(mg.weighted_laplacian(Lg, d), sp.diags(F.diag_AtA()), P.n_v, P.n_h, P.levels)
    t_h = time.perf_counter() - t0
    t0 = time.perf_counter()
    V = mg.VCycle(H, lam, nu=NU)
    t_s = time.perf_counter() - t0
    steps = []
    for _ in range(int(spec["n"])):
        t0 = time.perf_counter()
        q = ops.normal_apply(F, Lg, d, lam, x)
        V(q)
        steps.append(time.perf_counter() - t0)
    return dict(t_hierarchy=t_h, t_vsetup=t_s, steps=steps, threads=int(os.environ.get("OMP_NUM_THREADS", "1")))


def reference_arm(args, world, rank):
    """The CPU oracle, timed as it stands, on a bounded sample per step."""
    if rank != 0:
        return
    hi = host_info()
    if args.workload == "ct256":
        steps = []
        for i in range(args.warmup + args.steps):
            o = run_oracle_subprocess({"kind": "ct256", "budget": 8.0, "solves": 1})
            if i >= args.warmup:
                steps.append(o)
        solves = sum(o["solves"] for o in steps)
        t = sum(o["solve_s"] for o in steps)
        value = solves / t
        ms = t * 1e3 / args.steps
        sample = ("per step: oracle PCG (scipy CSR, 1 thread) solving the largest lambda of the first outer "
                  "iteration of the ct256 workload to rel-res 1e-6 (%d PCG iterations)" % steps[-1]["iterations"])
    else:
        code = ("import json,sys; sys.path.insert(0, %r); import bench; "
                "print(json.dumps(bench.oracle_steps_2048(json.loads(sys.argv[1]))))" % ROOT)
        out = subprocess.run([sys.executable, "-c", code, json.dumps({"n": args.warmup + args.steps})],
                             capture_output=True, text=True, env=_oracle_env(), cwd=ROOT, timeout=3600)
        if out.returncode != 0:
            raise RuntimeError(out.stderr[-2000:])
        o = json.loads(out.stdout.strip().splitlines()[-1])
        st = o["steps"][args.warmup:]
        t_it = sum(st) / len(st)
        window = 10
        per_solve = REF_ITS_PER_SOLVE * t_it + o["t_vsetup"] + o["t_hierarchy"] / window
        value = 1.0 / per_solve
        ms = t_it * 1e3
        sample = ("per step: one PCG iteration's work of the oracle (scipy 2-D correlation with the 31x31 PSF and its "
                  "transpose, V(1,1) on the sparse Galerkin hierarchy; 1 thread) on the 2048x2048 workload; "
                  "lambda-solves/s extrapolated with %.0f PCG iterations per lambda-solve (this benchmark's GPU "
                  "measurement), the V-cycle setup per solve and one hierarchy (%.1f s) per window of %d lambdas"
                  % (REF_ITS_PER_SOLVE, o["t_hierarchy"], window))
    line = {"metric": METRIC, "value": value, "unit": "lambda-solves/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": DESC[args.workload]}, "impl": "reference",
            "cpu_baseline": {"value": value, "unit": "lambda-solves/s", "kind": "oracle",
                             "cores": 1, "sample": sample, **hi},
            "e2e": {"value": value, "unit": "lambda-solves/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


def main():
    args = parse()
    if args.oracle_sample is not None:
        print(json.dumps(oracle_dispatch(json.loads(args.oracle_sample))))
        return
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        return reference_arm(args, world, rank)
    if args.profile_iters > 0:
        return profile_workload(args)
    if args.compare_precond:
        return compare_precond()
    if args.compare_algorithm2:
        return compare_algorithm2()
    if args.rhs_only:
        print(json.dumps(rhs_batched_leg(local)))
        return
    if args.serve_only:
        print(json.dumps(serving_leg(local, n_requests=args.serve_requests, rates=tuple(args.serve_rates))))
        return
    if args.workload == "ct256":
        return main_ct256(args, world, rank, local)
    return main_deblur(args, world, rank, local)


if __name__ == "__main__":
    main()
