"""Host-side logic of the multi-GPU benchmark (replicas: each rank solves its
own slice, no data-path collective) on CPU with two gloo ranks: the job
time is the slowest rank's, the value counts every rank's units, and the
reference arm does no work on ranks other than 0."""
import os
import socket
import sys

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def worker(rank, world, port, out):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    t = bench.max_over_ranks(10.0 + 5.0 * rank)
    v = bench.job_value(30 * 4, world, t)

    class A:
        steps, warmup, gpus = 2, 0, world
    # the reference arm on a non-zero rank returns without running the oracle
    ref_rc = bench.run_reference(A) if rank != 0 else 0
    out.put((rank, t, v, ref_rc))
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_timing_and_value():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = free_port()
    procs = [ctx.Process(target=worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, t, v, ref_rc in res:
        assert t == 15.0                          # max over ranks
        assert v == pytest.approx(30 * 4 * 2 / 0.015)
        assert ref_rc == 0


def test_single_process_needs_no_process_group():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(7.5) == 7.5
    assert bench.job_value(60, 1, 1000.0) == 60.0
