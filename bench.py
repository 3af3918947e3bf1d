#!/usr/bin/env python
"""Throughput of multigrid-preconditioned CG on the regularized normal
equations, swept over lambda and outer iterations (Algorithm 2).

One step = one full run of Algorithm 2 on the 256 x 256 CT workload:
lambda window, weights -> fine operator, Galerkin hierarchy, coarsest
factorisations, PCG solves (largest lambda first, each warm-started from
the previous lambda's solution), L-curve values, corner, weight update and
the three-equal stopping rule.  The metric is lambda-solves per second:
systems brought to a relative normal-equations residual of 1e-6, divided by
the wall time of the steps.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Under torchrun each rank runs its own replica of the workload (the right-
hand sides differ by the noise seed); there is no collective on the data
path; the job's value is the lambda-solves of all ranks divided by the
slowest rank's time.  --impl reference times the CPU oracle instead.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

WORKLOAD = "ct256"
WORKLOAD_DESC = ("ct256: 256x256 parallel-beam CT, 180 angles x 363 bins exact ray-length CSR "
                 "(FP32 values, int32 indices), 10 seeded ellipses, 1% noise, 20 lambdas "
                 "logspace(-4, 0), Algorithm 2 (max 15 outer iterations, three-equal stop, "
                 "largest-lambda-first warm-start chain), rel-res 1e-6, 5-level V(1,1) l1-Jacobi")
METRIC = "lambda-solves/s at rel-res 1e-6"
NU = 1  # V(nu, nu) sweeps: the library's default, and what the oracle arms run
KERNEL_SRC = os.path.join(ROOT, "paper_2306_11067_gb300", "csrc", "kernels.cuh")
LAUNCH_SRC = os.path.join(ROOT, "paper_2306_11067_gb300", "csrc", "launch_spmm.cu")
TRAFFIC_FILE = os.path.join(ROOT, "profiles", "k_spmv1_ct256_traffic.txt")


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--precision", default="mixed", choices=["mixed", "fp64"])
    ap.add_argument("--mode", default="sequential", choices=["sequential", "batched"])
    ap.add_argument("--no-plain", action="store_true", help="skip the plain FP64 comparison run")
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU oracle baseline")
    ap.add_argument("--oracle-sample", type=float, default=None, help=argparse.SUPPRESS)
    ap.add_argument("--no-serve", action="store_true", help="skip the served-mix latency leg")
    ap.add_argument("--serve-only", action="store_true", help=argparse.SUPPRESS)
    ap.add_argument("--compare-precond", action="store_true",
                    help="time the lambda sweep of one outer iteration with the default preconditioner (FP64 and "
                         "mixed) and the paper's own (geometric and classical AMG interpolation, FP64) at 64^2, "
                         "128^2, 256^2; one JSON line per arm, no bench line")
    ap.add_argument("--compare-algorithm2", action="store_true",
                    help="one full Algorithm 2 run of the workload per solver arm (default preconditioner mixed "
                         "and FP64, the paper's method with geometric P and with classical AMG split by the "
                         "paper's two passes or by PMIS): "
                         "lambda-solves/s and the selected lambda indices; one JSON line per arm")
    ap.add_argument("--profile-iters", type=int, default=0,
                    help="profiler workload: one lambda of the workload, this many PCG iterations, no JSON line")
    ap.add_argument("--profile-precond", type=int, default=0, choices=[0, 1, 2],
                    help="profiler workload's solver: 0 the default PCG (mixed), 1 the paper's method with "
                         "geometric P, 2 with classical AMG (FP64; --profile-iters FGMRES steps)")
    return ap.parse_args()


# ---------------------------------------------------------------------------
# CPU oracle sample (runs in a 1-thread subprocess, or as the reference arm)
# ---------------------------------------------------------------------------
def oracle_sample(budget_s: float, n_solves_max: int = 2) -> dict:
    """Time the oracle on the first outer iteration of the same workload:
    solves from the largest lambda down, each warm-started from the previous
    one, until n_solves_max solves or the time budget is spent."""
    import numpy as np
    import problemgen as pg
    from oracle import outer
    from oracle import operators as ops
    P = pg.make_problem(WORKLOAD)
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


def run_oracle_subprocess(budget_s: float, n_solves_max: int) -> dict:
    env = dict(os.environ)
    for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        env[k] = "1"
    code = ("import json,sys; sys.path.insert(0, %r); import bench; "
            "print(json.dumps(bench.oracle_sample(%f, %d)))" % (ROOT, budget_s, n_solves_max))
    out = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, env=env, cwd=ROOT,
                         timeout=600)
    if out.returncode != 0:
        raise RuntimeError(out.stderr[-2000:])
    return json.loads(out.stdout.strip().splitlines()[-1])


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


# Served mix (a reduced form of the Poisson request stream): 40% CT and 60%
# deblurring, image sides drawn uniformly from the sizes below, each request
# a 16-lambda sweep logspace(-5, 0, 16) of its own seeded phantom at its own
# noise level U[0.5%, 5%], arriving as a seeded Poisson process at 0.8x the
# capacity measured on a burst of the same mix.
SERVE_CT = ((128, 90, 182), (256, 179, 364))   # side, angles, bins
SERVE_BLUR = (128, 256, 512)                    # side; PSF 9 x 9, sigma 1.5
SERVE_REQUESTS = 24
SERVE_SLOTS = 4
SERVE_MAXIT = 2000   # per system; lambda = 1e-5 deblurring rarely reaches 1e-6: it is reported, not counted


def serving_leg(device):
    """p50 / p99 latency (submit -> result) and throughput of the served mix."""
    import numpy as np
    import problemgen as pg
    from paper_2306_11067_gb300 import lcmg as L
    g = pg.rng(7)
    srv = L.Server(device=device, hbm_budget=64 << 30, slots=SERVE_SLOTS, precision=L.PREC_MIXED,
                   mode=L.MODE_BATCHED, tol=1e-6, maxit=SERVE_MAXIT)
    psf = pg.gaussian_psf(4, 1.5)
    probs = []  # (pid, kind, N, forward)
    for N, na, nb in SERVE_CT:
        A = pg.ct_csr(N, na, nb)
        probs.append((srv.add_csr(N, N, A), "ct", N, A.to_scipy()))
    for N in SERVE_BLUR:
        probs.append((srv.add_psf(N, N, psf), "blur", N, None))
    lams = np.logspace(-5, 0, 16)

    def make_request(k):
        ct = g.uniform() < 0.4
        cand = [p for p in probs if (p[1] == "ct") == ct]
        pid, kind, N, A = cand[int(g.integers(len(cand)))]
        img = pg.phantom_mixed(N, N, 10, 3000 + k, lo=0.1, hi=1.0)
        b = (A @ img.ravel(order="F")) if kind == "ct" else pg.blur_apply(img, psf).ravel(order="F")
        return pid, pg.add_noise(b, float(g.uniform(0.005, 0.05)), 5000 + k)

    # capacity on a burst of 2 x slots requests
    burst = [make_request(k) for k in range(2 * SERVE_SLOTS)]
    t0 = time.perf_counter()
    tick = [srv.submit(pid, lams, b) for pid, b in burst]
    done = [srv.wait(t) for t in tick]
    cap = len(done) / (time.perf_counter() - t0)
    # the Poisson stream
    rate = 0.8 * cap
    reqs = [make_request(100 + k) for k in range(SERVE_REQUESTS)]
    gaps = g.exponential(1.0 / rate, SERVE_REQUESTS)
    t0 = time.perf_counter()
    tick, t_next = [], t0
    for (pid, b), gap in zip(reqs, gaps):
        t_next += gap
        delay = t_next - time.perf_counter()
        if delay > 0:
            time.sleep(delay)
        tick.append(srv.submit(pid, lams, b))
    res = [srv.wait(t) for t in tick]
    wall = time.perf_counter() - t0
    st = srv.stats()
    srv.close()
    lat = np.array([r["t_done"] - r["t_submit"] for r in res]) * 1e3
    conv = int(sum(r["n_converged"] for r in res))
    return {"requests": SERVE_REQUESTS, "p50_ms": float(np.percentile(lat, 50)),
            "p99_ms": float(np.percentile(lat, 99)), "mean_ms": float(lat.mean()),
            "lambda_solves_per_s": conv / wall, "converged": conv, "systems": 16 * SERVE_REQUESTS,
            "arrival_rate_per_s": rate, "burst_capacity_per_s": cap, "slots": SERVE_SLOTS,
            "peak_running": st["peak_running"], "context_reuses": st["reuses"],
            "mix": "40% CT (128^2: 90x182 rays, 256^2: 179x364) / 60% deblurring (128^2, 256^2, 512^2; "
                   "PSF 9x9 sigma 1.5); 16 lambda = logspace(-5, 0, 16) per request, noise U[0.5%, 5%]; "
                   "seeded Poisson arrivals at 0.8x burst capacity; mixed precision, batched, tol 1e-6, "
                   "maxit " + str(SERVE_MAXIT)}


def profile_workload(args):
    """A short run for profiler captures: the workload's operator and
    hierarchy, one lambda (the middle of the grid) solved from zero for
    args.profile_iters PCG iterations (mixed precision, one column)."""
    import problemgen as pg
    from paper_2306_11067_gb300 import lcmg as L
    P = pg.make_problem(WORKLOAD)
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
        P = pg.make_problem(WORKLOAD, size=None if N == 256 else N)
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
    P = pg.make_problem(WORKLOAD)
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
        print(json.dumps({"arm": name, "workload": WORKLOAD, "seconds": round(dt, 3),
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


# ---------------------------------------------------------------------------
def main():
    args = parse()
    if args.oracle_sample is not None:
        print(json.dumps(oracle_sample(args.oracle_sample)))
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
    if args.serve_only:
        print(json.dumps(serving_leg(int(os.environ.get("LOCAL_RANK", "0")))))
        return

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

    P = pg.make_problem(WORKLOAD)
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
    achieved = (op_bytes / (op_ms / 1e3) / 1e9) if op_ms > 0 else None
    roofline = {
        "kernel": (("k_spmv1 (the one-column SpMV, both operator passes: y = A p with int32 columns, then "
                    "q = A^T y + lam^2 L^T W L p with p.q and 16-bit column offsets)") if mode == L.MODE_SEQUENTIAL
                   else "k_spmm (the batched SpMM, both operator passes over the active columns)"),
        "bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
        "frac": (achieved / peak) if achieved else None, "peak_source": f"{peak_kind} (MEASURED_PEAKS.json hbm_gbs)",
        "traffic": recorded_traffic() if mode == L.MODE_SEQUENTIAL else None,
        "algorithmic_bytes_per_pass": (op_bytes / op_launches) if op_launches else None,
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
            o = run_oracle_subprocess(20.0, 2)
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
            "config": {"workload": WORKLOAD_DESC, "precision": args.precision, "mode": args.mode,
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


def reference_arm(args, world, rank):
    """The CPU oracle, timed as it stands, on a bounded sample per step."""
    if rank != 0:
        return
    steps = []
    for i in range(args.warmup + args.steps):
        o = run_oracle_subprocess(8.0, 1)
        if i >= args.warmup:
            steps.append(o)
    solves = sum(o["solves"] for o in steps)
    t = sum(o["solve_s"] for o in steps)
    value = solves / t
    sample = ("per step: oracle PCG (scipy CSR, 1 thread) solving the largest lambda of the first outer "
              "iteration of the ct256 workload to rel-res 1e-6 (%d PCG iterations)" % steps[-1]["iterations"])
    line = {"metric": METRIC, "value": value, "unit": "lambda-solves/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": t * 1e3 / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD_DESC}, "impl": "reference",
            "cpu_baseline": {"value": value, "unit": "lambda-solves/s", "kind": "oracle",
                             "cores": steps[-1]["threads"], "sample": sample},
            "e2e": {"value": value, "unit": "lambda-solves/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


if __name__ == "__main__":
    main()
