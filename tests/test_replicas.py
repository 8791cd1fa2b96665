"""The multi-GPU form of bench.py is independent replicas (RHS sharding, no data-path
collective): every rank times its own solves, the job's time is the max over ranks and its rate
is all ranks' right-hand sides over that time; the reference arm runs on rank 0 only.  The
multi-rank host logic is exercised here with world_size-2 gloo process groups on the CPU."""

import os
import socket
import sys

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, q):
    os.environ.update({"MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port),
                       "RANK": str(rank), "WORLD_SIZE": str(world), "LOCAL_RANK": str(rank)})
    sys.path.insert(0, ROOT)
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        w, r, _ = bench._dist()
        bench._barrier(w)
        per_rank_seconds = 1.0 + rank          # rank 1 is the slow replica
        t = bench._reduce_max(per_rank_seconds, w)
        rate = bench.whole_job_rate(w, 16, 5, t)
        # the reference arm: every rank but 0 leaves at once, without work
        class A:
            pass
        args = A()
        args.workload, args.steps, args.warmup, args.tol = "const2d_128", 0, 0, 1e-6
        ref = bench.run_reference(args) if r != 0 else None
        q.put((r, w, t, rate, ref))
    finally:
        dist.destroy_process_group()


def test_replicas_take_the_slowest_rank_and_sum_the_work():
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=180)
        assert p.exitcode == 0
    out = sorted(q.get(timeout=10) for _ in range(world))
    for rank, w, t, rate, ref in out:
        assert w == world
        assert t == 2.0                          # max over ranks
        assert rate == pytest.approx(2 * 16 * 5 / 2.0)
    assert out[1][4] == 0                        # rank 1: reference arm exits 0 without work
