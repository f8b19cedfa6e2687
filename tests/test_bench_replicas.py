"""The multi-GPU form of the benchmark runs independent replicas (a single
factor does not shard): the whole-job value is every rank's bytes over the
slowest rank's time.  Checked here with two gloo ranks on the CPU."""
from __future__ import annotations

import os
import socket

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank(rank, world, port, q):
    import sys
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    ms_local = 2.0 + rank          # rank 1 is the slowest
    value, ms_max = bench.aggregate(ms_local, 1e9, world, "cpu")
    q.put((rank, value, ms_max))
    dist.barrier()
    dist.destroy_process_group()


def test_replica_throughput_is_total_bytes_over_slowest_rank():
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    got = sorted(q.get(timeout=10) for _ in range(world))
    for rank, value, ms_max in got:
        assert ms_max == pytest.approx(3.0)
        assert value == pytest.approx(world * 1e9 / 3e-3 / 1e9)


def test_single_rank_is_its_own_time():
    import sys
    sys.path.insert(0, ROOT)
    import bench
    value, ms = bench.aggregate(4.0, 2e9, 1)
    assert ms == 4.0 and value == pytest.approx(2e9 / 4e-3 / 1e9)
