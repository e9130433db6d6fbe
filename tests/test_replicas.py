"""Replica reduction of bench.py on CPU with world_size 2 (gloo): every rank advances
an independent replica; the job value is all ranks' cells*steps over the slowest
rank's time, and V-cycles are summed."""
import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, q):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    import sys

    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import bench

    dist.init_process_group("gloo", rank=rank, world_size=world)
    t = [1.5, 2.5][rank]
    vc = [10, 14][rank]
    tmax, vtot = bench.reduce_replicas(dist, t, vc, "cpu")
    q.put((rank, bench.job_value(world, 1000, 20, tmax), vtot))
    dist.destroy_process_group()


def test_replica_reduction_gloo():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, value, vtot in out:
        assert value == pytest.approx(2 * 1000 * 20 / 2.5)
        assert vtot == 24.0


def test_launch_count_model():
    import bench

    fixed, per = bench._launches_per_step(7, 4, True)
    assert fixed == 2 * 2 + 4 + 3
    assert per == 5 + 1 + 6 * 4 + 2
    assert bench._launches_per_step(1, 4, False) == (2 + 4 + 3, 4)
