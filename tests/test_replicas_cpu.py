"""The replicas-only multi-process path of bench.py, on CPU with gloo (world size 2)."""

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


def _rank(rank, world, port, ms, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        agg = bench.replica_step_ms(ms[rank], dist, torch.device("cpu"))
        out[rank] = (agg, bench.replica_value(agg, world))
    finally:
        dist.barrier()
        dist.destroy_process_group()


def test_replica_timing_takes_the_slowest_rank():
    world = 2
    port = _free_port()
    ms = [0.125, 0.250]
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_rank, args=(world, port, ms, out), nprocs=world, join=True)
        res = dict(out)
    for r in range(world):
        agg, value = res[r]
        assert agg == pytest.approx(0.250)                 # max over ranks
        assert value == pytest.approx(world * 1000.0 / 0.250)  # all ranks' resultants
