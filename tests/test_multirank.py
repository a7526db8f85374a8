"""The multi-rank (torchrun) path of bench.py on CPU: world size 2 over gloo.

Each rank recovers its own batch; the job's time is the slowest rank's, taken
with an all-reduce(MAX) of the timing only (no collective on the data path)."""
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, out):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    dist.init_process_group("gloo", init_method="tcp://127.0.0.1:%d" % port, rank=rank, world_size=world)
    ms, value = bench.aggregate([12.5, 20.0][rank], per_rank_batch=4, steps=2, world=world, dist=dist)
    # the replicas' inputs differ by rank (seeded per rank)
    import argparse
    args = argparse.Namespace(size=8, ratio=0.25, batch=2)
    _, _, _, _, _, x = bench.workload(args, rank)
    out[rank] = (ms, value, float(x.sum()))
    dist.barrier()
    dist.destroy_process_group()


def test_bench_aggregation_world_size_2():
    import torch.multiprocessing as mp
    port = _free_port()
    mgr = mp.get_context("spawn").Manager()   # no fork of a threaded test process
    out = mgr.dict()
    mp.spawn(_worker, args=(2, port, out), nprocs=2, join=True)
    assert out[0][0] == out[1][0] == 20.0                       # max over ranks
    assert out[0][1] == out[1][1] == pytest.approx(2 * 4 * 2 / 0.020)
    assert out[0][2] != out[1][2]                               # different images per rank
