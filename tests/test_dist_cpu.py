"""The multi-rank logic of the benchmark on CPU with two gloo ranks: disjoint phantom seeds
per rank (independent problems, no data-path collective) and the max over ranks of the
timings."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
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
    import bench
    seeds = bench.rank_seeds(rank, 16)
    times = bench.max_over_ranks([10.0 + rank, 5.0 - rank], world)
    gathered = [None] * world
    dist.all_gather_object(gathered, seeds)
    out[rank] = (seeds, times, gathered)
    dist.destroy_process_group()


def test_two_gloo_ranks():
    world = 2
    port = _free_port()
    mgr = mp.get_context("spawn").Manager()
    out = mgr.dict()
    mp.start_processes(_worker, args=(world, port, out), nprocs=world, start_method="spawn", join=True)
    s0, t0, g0 = out[0]
    s1, t1, g1 = out[1]
    assert s0 == list(range(0, 16)) and s1 == list(range(16, 32))
    assert not set(s0) & set(s1)
    assert t0 == t1 == [11.0, 5.0]
    assert g0 == g1 == [s0, s1]
