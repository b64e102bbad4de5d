"""Multi-process host logic of the replica benchmark (CPU, gloo, world size 2): the job's
rate takes the slowest rank's time, and the ranks' warm-start seeds are disjoint."""

import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

import bench


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        seconds = 1.0 + rank  # rank 1 is the slow one
        rate, t_max = bench.whole_job_rate(dist, world, 10, seconds, "cpu")
        seeds = torch.tensor(bench.step_seeds(rank, 23), dtype=torch.int64)
        gathered = [torch.zeros_like(seeds) for _ in range(world)]
        dist.all_gather(gathered, seeds)
        out[rank] = (rate, t_max, [g.tolist() for g in gathered])
    finally:
        dist.destroy_process_group()


def test_whole_job_rate_and_disjoint_seeds_two_ranks():
    world = 2
    port = _free_port()
    ctx = mp.get_context("spawn")
    with ctx.Manager() as mgr:
        out = mgr.dict()
        procs = [ctx.Process(target=_worker, args=(r, world, port, out)) for r in range(world)]
        for p in procs:
            p.start()
        for p in procs:
            p.join(timeout=120)
            assert p.exitcode == 0
        res = dict(out)
    for r in range(world):
        rate, t_max, seeds = res[r]
        assert t_max == pytest.approx(2.0)
        assert rate == pytest.approx(world * 10 / 2.0)
        assert not set(seeds[0]) & set(seeds[1])


def test_whole_job_rate_single_rank():
    rate, t_max = bench.whole_job_rate(None, 1, 7, 3.5, "cpu")
    assert t_max == 3.5 and rate == pytest.approx(2.0)
