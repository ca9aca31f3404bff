"""Host-side sharding of the sweep over ranks (CPU; world_size 2 over gloo):
shards are disjoint, complete and balanced, every rank derives the same
partition, and the step time is reduced as the maximum over ranks."""
import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

import inputs
from paper_2607_08447_b300.sweep import partition_sweep, shard_of


def test_partition_is_disjoint_complete_and_balanced():
    costs = [p.n_unknowns for p in inputs.config4()]
    for world in (1, 2, 3, 8):
        shards = partition_sweep(costs, world)
        flat = sorted(i for s in shards for i in s)
        assert flat == list(range(len(costs)))
        loads = [sum(costs[i] for i in s) for s in shards]
        # LPT bound: max load <= mean + largest item
        assert max(loads) <= sum(costs) / world + max(costs)


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, costs, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    mine = shard_of(costs, rank, world)
    gathered = [None] * world
    dist.all_gather_object(gathered, mine)
    # per-rank "time" reduced by MAX, as bench.py reduces its timed region
    t = torch.tensor([float(sum(costs[i] for i in mine))], dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    out[rank] = (gathered, float(t.item()))
    dist.barrier()
    dist.destroy_process_group()


def test_gloo_two_ranks_agree_on_the_partition():
    costs = [p.n_unknowns for p in inputs.config4(16)]
    world = 2
    port = _free_port()
    ctx = mp.get_context("spawn")
    manager = ctx.Manager()
    out = manager.dict()
    procs = [ctx.Process(target=_worker, args=(r, world, port, costs, out)) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    g0, t0 = out[0]
    g1, t1 = out[1]
    assert g0 == g1 == partition_sweep(costs, world)
    assert set(g0[0]).isdisjoint(g0[1])
    assert t0 == t1 == max(sum(costs[i] for i in s) for s in g0)
