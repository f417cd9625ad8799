"""The multi-GPU path of bench.py is replicas only (independent solves, no
data-path collective); its host logic -- max-over-ranks timing and the
whole-job rate -- is checked here with two gloo ranks on the CPU."""

import os
import socket

import pytest


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, out):
    import torch.distributed as dist

    import bench

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    mine = [3.0, 7.5][rank]  # per-rank timed seconds
    m = bench.reduce_max(mine, dist, "cpu")
    out[rank] = (m, bench.aggregate_rate(100, world, m))
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_max_and_rate():
    import torch.multiprocessing as mp

    port = _free_port()
    manager = mp.Manager()
    out = manager.dict()
    mp.spawn(_worker, args=(2, port, out), nprocs=2, join=True)
    assert out[0] == out[1] == (7.5, 2 * 100 / 7.5)
