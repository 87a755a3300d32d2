"""Multi-rank replica placement, run as world-size-2 gloo process groups on the CPU."""
import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

from paper_1204_2088_gb300 import inputs, replicas


def test_partition_covers_every_replica_once_and_balances():
    sites = [c["grid"][0] * c["grid"][1] * c["grid"][2] for c in inputs.batch48()]
    for world in (1, 2, 3, 4, 8, 64):
        parts = replicas.partition(sites, world)
        flat = sorted(i for p in parts for i in p)
        assert flat == list(range(len(sites)))
        loads = [sum(sites[i] for i in p) for p in parts]
        assert max(loads) <= sum(sites) / world + max(sites)


def test_aggregate_rate_uses_the_slowest_rank():
    assert replicas.aggregate_rate([100, 300], [1.0, 2.0]) == pytest.approx(400 / 2e-3)
    with pytest.raises(ValueError):
        replicas.aggregate_rate([1], [0.0])


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, q):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        cfgs = inputs.batch48()
        sites = [c["grid"][0] * c["grid"][1] * c["grid"][2] for c in cfgs]
        mine = replicas.partition(sites, world)[rank]
        # every rank derives the same placement independently: gather and compare
        got = [None] * world
        dist.all_gather_object(got, mine)
        # a rank's own single-system replica differs from every other rank's
        seeds = [None] * world
        dist.all_gather_object(seeds, replicas.rank_seed(11, rank))
        # the timed region: max over ranks of the elapsed time, sum of the sites
        t = torch.tensor([1.0 + rank], dtype=torch.float64)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        n = torch.tensor([float(sum(sites[i] for i in mine))], dtype=torch.float64)
        dist.all_reduce(n, op=dist.ReduceOp.SUM)
        if rank == 0:
            q.put((got, seeds, float(t.item()), float(n.item()), sum(sites)))
    finally:
        dist.destroy_process_group()


def test_two_rank_placement_and_timing_reduction_gloo():
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
    assert all(p.exitcode == 0 for p in procs)
    got, seeds, tmax, nsum, total = q.get(timeout=10)
    assert sorted(i for g in got for i in g) == list(range(48))
    assert not set(got[0]) & set(got[1])
    assert len(set(seeds)) == world
    assert tmax == 2.0 and nsum == total
