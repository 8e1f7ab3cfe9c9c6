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


def _solve_worker(rank, world, port, out):
    """The batch flow of one rank with the float64 checker standing in for
    the GPU call: place the instances, solve this rank's share, then gather
    every rank's results and the max over ranks of the solve time."""
    import time

    import numpy as np

    from oracle import reference as R
    from paper_1606_04809_gb300 import synth

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    specs = synth.batch_params(count=7, seed=5, n_range=(300, 900), d_range=(50, 200), density_range=(0.02, 0.08),
                               lam_range=(1e-3, 1e-2), storage="f32")
    mine = sharding.rank_instances([s["n"] * s["k_mean"] for s in specs], world, rank)
    t0 = time.perf_counter()
    results = {}
    for i in mine:
        p = synth.batch_instance(specs[i], values="f64", threads=1)
        res = R.certified_fstar(p, lambda ep, p=p: synth.sample_indices(p.n, p.n, 30, ep), rel_tol=1e-10,
                                max_epochs=2000, check_every=5)
        results[i] = (res["fstar"], res["bound"])
    el = time.perf_counter() - t0
    gathered = [None] * world
    dist.all_gather_object(gathered, results)
    t = torch.tensor([el], dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    times = [None] * world
    dist.all_gather_object(times, el)
    dist.barrier()
    if rank == 0:
        out.put((gathered, float(t.item()), times))
    dist.destroy_process_group()


def test_two_ranks_solve_their_shares_and_gather_every_instance_once():
    import numpy as np

    from oracle import reference as R
    from paper_1606_04809_gb300 import synth

    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_solve_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    gathered, tmax, times = q.get(timeout=300)
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    keys = [set(g) for g in gathered]
    assert keys[0].isdisjoint(keys[1]) and sorted(keys[0] | keys[1]) == list(range(7))
    assert tmax == max(times)
    # every gathered optimum is the instance's own: a Newton solve on rank 0 agrees
    specs = synth.batch_params(count=7, seed=5, n_range=(300, 900), d_range=(50, 200), density_range=(0.02, 0.08),
                               lam_range=(1e-3, 1e-2), storage="f32")
    merged = {**gathered[0], **gathered[1]}
    for i, (fstar, bound) in merged.items():
        p = synth.batch_instance(specs[i], values="f64", threads=1)
        f_newton = R.objective(p, R.newton(p))
        assert f_newton <= fstar <= f_newton + bound + 1e-14
