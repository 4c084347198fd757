"""Multi-rank bookkeeping of bench.py on CPU (gloo, world_size 2).

The path shards as independent replicas (one system per rank, no data-path
collective); the only cross-rank operations are the barrier and the maximum
of the timed region, which define the whole-job throughput.  Here two gloo
ranks report different local times and both must agree on
units * steps * world / max(time).  The reference arm under torchrun runs on
rank 0 only; the other ranks exit immediately.
"""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    local_ms = 100.0 + 50.0 * rank
    value, total = bench.whole_job_rate(9000, 20, local_ms, dist, "cpu")
    dist.barrier()
    q.put((rank, value, total))
    dist.destroy_process_group()


def _ref_worker(rank, world, q):
    os.environ["RANK"] = str(rank)
    import bench

    class A:
        workload = "gas24"
        steps = 1
        warmup = 0
        gpus = world
    if rank != 0:
        q.put((rank, bench.run_reference(A)))
    else:
        q.put((rank, "skipped"))


def test_whole_job_rate_two_gloo_ranks():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    ps = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in ps:
        p.start()
    out = [q.get(timeout=120) for _ in ps]
    for p in ps:
        p.join(timeout=60)
        assert p.exitcode == 0
    expect = 9000 * 20 * 2 / 0.150
    for rank, value, total in out:
        assert total == pytest.approx(150.0)
        assert value == pytest.approx(expect)


def test_reference_arm_runs_on_rank_zero_only():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    p = ctx.Process(target=_ref_worker, args=(1, 2, q))
    p.start()
    rank, rc = q.get(timeout=120)
    p.join(timeout=60)
    assert rank == 1 and rc == 0 and p.exitcode == 0
