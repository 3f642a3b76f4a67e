"""Multi-process host logic of the bench's replica mode on CPU (gloo,
world size 2): whole-job timing is the maximum over ranks, and every rank
builds an independent network from its own seed (no data-path collective)."""
from __future__ import annotations

import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    from workloads import configs as C
    t = bench.barrier_max(10.0 + 5.0 * rank, world)
    bench.barrier(world)
    W = C.million_sparse(n_rec=300, k_in=20, T=10, seed=bench.replica_seed(rank))
    out[rank] = (t, int(W["col"][:50].sum()), float(W["w"][:50].sum()))
    dist.destroy_process_group()


def test_two_replicas_take_the_max_time_and_build_independent_networks():
    world = 2
    mgr = mp.Manager()
    out = mgr.dict()
    mp.spawn(_worker, args=(world, _free_port(), out), nprocs=world, join=True)
    assert out[0][0] == out[1][0] == 15.0
    assert out[0][1:] != out[1][1:]
