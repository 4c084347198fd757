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


def _shard_worker(rank, world, port, q):
    import numpy as np
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import oracle
    import synth
    from paper_2207_14276_gb300.router import serve_sharded
    reqs, sizes, orc = _requests()

    def evaluate(s):
        r = orc.energy_forces(s.coords, s.species, s.box, s.mask)
        return r["energy"], r["forces"]
    out = serve_sharded(reqs, sizes, evaluate, dist)
    if rank == 0:
        q.put([(e, f.tolist()) for e, f in out])
    dist.barrier()
    dist.destroy_process_group()


def _requests():
    import numpy as np
    import oracle
    import synth
    spec = synth.model_spec("ani4")
    orc = oracle.Model(spec, synth.make_weights(spec, 1))
    mols, _, _ = synth.workload("molecules64")
    reqs = list(mols[:9]) + [synth.water_box(60, 12.0, 4, seed=2)]
    sizes = [m.n_ml for m in reqs]
    return reqs, sizes, orc


def test_replicas_behind_a_router_gather_the_single_rank_results():
    """Two gloo ranks each evaluate the requests the router assigns them (the FP64
    oracle stands in for each replica's GPU evaluation); the results rank 0
    gathers, in request order, equal those of one rank evaluating everything."""
    import numpy as np
    from paper_2207_14276_gb300.router import serve_sharded, shard
    reqs, sizes, orc = _requests()
    owner = shard(sizes, 2)
    assert set(owner) == {0, 1}                        # both replicas get work
    load = [sum(n for n, o in zip(sizes, owner) if o == r) for r in (0, 1)]
    assert abs(load[0] - load[1]) <= max(sizes)        # balanced to one request
    single = serve_sharded(reqs, sizes,
                           lambda s: (lambda r: (r["energy"], r["forces"]))(
                               orc.energy_forces(s.coords, s.species, s.box, s.mask)))
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    ps = [ctx.Process(target=_shard_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in ps:
        p.start()
    got = q.get(timeout=300)
    for p in ps:
        p.join(timeout=120)
        assert p.exitcode == 0
    assert len(got) == len(single)
    for (e, f), (e0, f0) in zip(got, single):
        assert e == e0
        np.testing.assert_array_equal(np.asarray(f), f0)


def test_router_policy():
    """Resident boxes stay on the replica that holds them; other requests go to
    the least-loaded replica by outstanding ML atoms, lowest index on ties."""
    from paper_2207_14276_gb300.router import Router
    r = Router(3)
    assert [r.place_resident(b, 20000) for b in (0, 1, 2, 3)] == [0, 1, 2, 0]
    assert r.place_resident(1, 20000) == 1
    assert r.assign(40, box_id=3) == 0
    assert r.assign(100) == 1 and r.assign(50) == 2 and r.assign(10) == 0
    assert r.load == [50, 100, 50]
    r.complete(1, 100)
    assert r.assign(5) == 1
    with pytest.raises(KeyError):
        r.assign(10, box_id=9)
