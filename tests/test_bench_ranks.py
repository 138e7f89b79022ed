"""The multi-process replica path of bench.py on CPU (gloo, world size 2):
the job's time is the slowest rank's and its work the sum over the ranks,
every rank builds a different replica graph, and every rank returns the same
aggregate."""
import os
import socket
import sys

import numpy as np
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def worker(rank, world, port, out):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    ms = [120.0, 95.5][rank]
    upd = [1000, 2500][rank]
    res = bench.reduce_over_ranks(ms, upd, dist, "cpu")
    out[rank] = res
    dist.barrier()
    dist.destroy_process_group()


def test_reduce_over_ranks_gloo():
    world = 2
    with mp.Manager() as mgr:
        out = mgr.dict()
        mp.spawn(worker, args=(world, free_port(), out), nprocs=world, join=True)
        res = dict(out)
    assert res[0] == res[1] == (120.0, 3500.0)


def test_single_process_is_its_own_aggregate():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.reduce_over_ranks(7.5, 42, None, "cpu") == (7.5, 42.0)


def test_replicas_get_different_graphs(monkeypatch):
    sys.path.insert(0, ROOT)
    import bench
    monkeypatch.setitem(bench.WL, "scale", 8)
    a, b = bench.make_inputs(0).train, bench.make_inputs(1).train
    assert not (a.n == b.n and np.array_equal(a.col, b.col))
