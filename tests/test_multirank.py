"""The multi-GPU form is replicas: each rank simulates its own shots and the
benchmark reports all ranks' ops over the slowest rank's time.  Checked with
two gloo ranks on CPU (no GPU, no collective on the data path)."""
import os
import socket

import pytest
import torch.distributed as dist
import torch.multiprocessing as mp

import bench


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        t_local = 1.0 + rank                       # rank 1 is the slower one
        value, t = bench.aggregate(t_local, ops_per_step=1000, steps=5, world=world,
                                   dist=dist, device="cpu")
        shots = bench.shot_indices(rank, 5, 3)
        dist.barrier()
        out[rank] = (value, t, shots)
    finally:
        dist.destroy_process_group()


def test_two_rank_aggregation_and_disjoint_shots():
    world = 2
    port = _free_port()
    mgr = mp.Manager()
    out = mgr.dict()
    mp.spawn(_rank, args=(world, port, out), nprocs=world, join=True)
    v0, t0, s0 = out[0]
    v1, t1, s1 = out[1]
    assert t0 == t1 == pytest.approx(2.0)              # max over ranks
    assert v0 == v1 == pytest.approx(1000 * 5 * 2 / 2.0)
    assert not set(s0) & set(s1) and len(s0) == len(s1) == 8


def test_single_rank_aggregation_needs_no_process_group():
    v, t = bench.aggregate(0.5, 200, 4, 1)
    assert t == 0.5 and v == pytest.approx(1600.0)
