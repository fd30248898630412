"""The multi-GPU path of bench.py is request sharding with no data-path
collective: each rank serves its own batch (distinct seeds and object ids)
and only the timing is reduced (max over ranks). Checked with two gloo
ranks on CPU."""
import os
import socket

import pytest
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _rank(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    plan = bench.shard_plan(rank, 64)
    t = bench.reduce_max(10.0 * (rank + 1), dist, "cpu")
    dist.barrier()
    out[rank] = (plan["input_seed"], plan["level_seed"], plan["first_index"], t)
    dist.destroy_process_group()


def test_two_rank_sharding_and_max_timing():
    mgr = mp.Manager()
    out = mgr.dict()
    mp.spawn(_rank, args=(2, _free_port(), out), nprocs=2, join=True)
    a, b = out[0], out[1]
    assert a[0] != b[0] and a[1] != b[1]          # different inputs and levels per rank
    assert b[2] - a[2] == 64                       # disjoint object ids (encryption streams)
    assert a[3] == b[3] == 20.0                    # every rank reports the slowest rank's time


def test_single_rank_is_identity():
    import bench
    assert bench.reduce_max(3.5, None, "cpu") == 3.5
