"""The multi-rank path of bench.py on CPU: two gloo ranks, each with its own
independent problem (seed offset by rank); the job time is the slowest
rank's and the throughput aggregates all ranks' DOFs. No data-path
collective is involved (the problems are independent)."""

import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    sys.path.insert(0, root)
    import bench
    from fem_inputs import hex_lattice
    # independent problems: different seeds give different meshes
    c, h, kappa, xgen = bench.make_problem(2, 3, seed_offset=bench.rank_seed_offset(rank))
    per_rank_ms = 10.0 + 5.0 * rank
    slowest = bench.reduce_max(per_rank_ms)
    digest = torch.tensor([float(c.sum()), float(kappa.sum())], dtype=torch.float64)
    gathered = [torch.zeros(2, dtype=torch.float64) for _ in range(world)]
    dist.all_gather(gathered, digest)
    out[rank] = (slowest, [g.tolist() for g in gathered])
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_max_time_and_independent_problems():
    world = 2
    port = _free_port()
    ctx = mp.get_context("spawn")
    mgr = ctx.Manager()
    out = mgr.dict()
    procs = [ctx.Process(target=_worker, args=(r, world, port, out)) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    for r in range(world):
        slowest, digests = out[r]
        assert slowest == 15.0                      # max over ranks
        assert digests[0] != digests[1]             # rank-local problems differ
    # aggregate throughput: all ranks' DOFs over the slowest rank's time
    ndof = (2 * 3 + 1) ** 3
    value = world * ndof / (15.0e-3) / 1e9
    assert value == pytest.approx(2 * 343 / 0.015 / 1e9)


def test_reduce_max_without_process_group():
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import bench
    assert bench.reduce_max(3.5) == 3.5
