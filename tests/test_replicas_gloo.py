"""The multi-GPU form of the benchmark runs independent replicas (one instance per rank, no
collective on the data path); the only cross-rank step is the max over ranks of the timed
region.  Checked here with two CPU processes on the gloo backend."""
import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

import bench


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    local = [12.5, 40.0][rank]
    got = bench.max_over_ranks(local, world, device="cpu")
    units = bench.replica_units(steps=5, world=world)
    q.put((rank, got, units))
    dist.destroy_process_group()


def test_two_rank_max_and_weak_scaling_units():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = [q.get(timeout=120) for _ in range(2)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, got, units in out:
        assert got == 40.0
        assert units == 10


def test_single_rank_needs_no_process_group():
    assert bench.max_over_ranks(3.0, 1) == 3.0
    assert bench.replica_units(steps=7, world=1) == 7
