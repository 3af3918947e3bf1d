"""The multi-rank path of bench.py on CPU ranks (gloo, world size 2):
replicas, no collective on the data path; the job's value is the
lambda-solves of all ranks over the slowest rank's time."""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

import bench
import problemgen as pg


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, q):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        conv, t = (70.0, 5.5) if rank == 0 else (64.0, 6.25)
        q.put((rank, bench.job_aggregate(conv, t, world)))
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_job_aggregate_sums_solves_and_takes_the_slowest_rank():
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    out = dict(q.get(timeout=120) for _ in range(world))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for r in range(world):
        assert out[r] == (134.0, 6.25)          # every rank sees the job totals
    assert 134.0 / 6.25 == pytest.approx(21.44)


def test_single_rank_aggregate_is_its_own():
    assert bench.job_aggregate(70, 5.5, 1) == (70.0, 5.5)


def test_replicas_share_the_operator_and_draw_their_own_noise():
    P = pg.make_problem("ct256", size=32)
    b0, b1, b2 = (bench.replica_rhs(P, r) for r in range(3))
    assert np.array_equal(b0, P.b[:, 0])
    clean = P.A.to_scipy() @ P.x_true[:, 0]
    for b in (b1, b2):
        e = b - clean
        assert not np.allclose(b, b0)
        # the workload's noise level: ||e|| = level ||A x_true||
        assert np.linalg.norm(e) == pytest.approx(P.meta["noise"] * np.linalg.norm(clean), rel=1e-12)
    assert not np.allclose(b1, b2)


def test_reference_arm_runs_on_rank_zero_only():
    class A:
        steps, warmup = 1, 0
    assert bench.reference_arm(A(), 2, 1) is None   # rank 1: no work, no output
