"""Multi-rank placement of independent instances, exercised with world
size 2 on the gloo backend (CPU): every instance lands on exactly one rank,
loads are balanced, and the max-over-ranks timing reduction works."""
import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

from paper_1606_04809_gb300 import sharding


def test_lpt_assignment_properties():
    costs = [5, 3, 3, 2, 2, 2, 1, 9]
    shares = sharding.shard_instances(costs, 3)
    flat = sorted(i for s in shares for i in s)
    assert flat == list(range(len(costs)))
    loads = [sum(costs[i] for i in s) for s in shares]
    assert max(loads) - min(loads) <= max(costs)
    assert sharding.shard_instances([1.0], 4) == [[0], [], [], []]
    with pytest.raises(ValueError):
        sharding.shard_instances([1.0], 0)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, costs, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    mine = sharding.rank_instances(costs, world, rank)
    gathered = [None] * world
    dist.all_gather_object(gathered, mine)
    t = torch.tensor([float(rank + 1) * 0.25], dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.barrier()
    if rank == 0:
        out.put((gathered, float(t.item())))
    dist.destroy_process_group()


def test_two_ranks_cover_every_instance_once():
    costs = [float(c) for c in (40, 7, 7, 30, 1, 1, 1, 22, 13, 2)]
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, costs, q)) for r in range(2)]
    for p in procs:
        p.start()
    gathered, tmax = q.get(timeout=120)
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    assert sorted(gathered[0] + gathered[1]) == list(range(len(costs)))
    assert not set(gathered[0]) & set(gathered[1])
    loads = [sum(costs[i] for i in g) for g in gathered]
    assert abs(loads[0] - loads[1]) <= max(costs)
    assert tmax == 0.5
