"""Multi-rank host logic of the batched workload, on CPU with gloo.

Two ranks shard the 64 uneven instances of the batched workload: the
shards are disjoint, cover every instance, balance the work within 10%,
and the ranks agree on them without exchanging anything but a check.
"""
import os

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

from paper_2111_11538_gb300 import inputs, sharding


def _costs(precond="mg"):
    desc = inputs.batch_instances(64, 4)
    return [sharding.instance_cost((d["n"], d["n"]), precond) for d in desc]


def _worker(rank, world, port, q):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    costs = _costs()
    mine = sharding.shard(costs, world)[rank]
    # every rank computes the same split: gather and compare
    flags = torch.zeros(len(costs), dtype=torch.int64)
    flags[mine] = 1
    dist.all_reduce(flags)
    work = torch.tensor([float(sum(costs[i] for i in mine))], dtype=torch.float64)
    works = [torch.zeros(1, dtype=torch.float64) for _ in range(world)]
    dist.all_gather(works, work)
    if rank == 0:
        q.put((flags.tolist(), [w.item() for w in works]))
    dist.destroy_process_group()


def test_two_ranks_shard_the_batch():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = 29500 + (os.getpid() % 1000)
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    flags, works = q.get(timeout=120)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert flags == [1] * 64                      # disjoint and complete
    assert max(works) <= 1.1 * (sum(works) / 2)   # balanced


@pytest.mark.parametrize("precond", ["mg", "jacobi"])
def test_shard_properties(precond):
    costs = _costs(precond)
    for world in (1, 3, 8):
        parts = sharding.shard(costs, world)
        assert sorted(i for p in parts for i in p) == list(range(64))
        loads = [sum(costs[i] for i in p) for p in parts]
        assert max(loads) <= max(costs) + sum(costs) / world
    with pytest.raises(ValueError):
        sharding.shard(costs, 0)
    with pytest.raises(ValueError):
        sharding.instance_cost((8, 8), "cg")
