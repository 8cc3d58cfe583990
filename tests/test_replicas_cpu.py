"""bench.py's multi-GPU path is "replicas only": every rank runs the whole
workload on its own GPU and rank 0 reports all ranks' work over the slowest
rank's time.  The aggregation runs here on CPU with two gloo ranks."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench

    local = [0.5, 2.0][rank]  # rank 1 is the slow one
    t, v = bench.aggregate_replicas(local, world, 1000, dist)
    out[rank] = (t, v)
    dist.destroy_process_group()


def test_two_replicas_report_slowest_time():
    world, port = 2, _free_port()
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_rank, args=(world, port, out), nprocs=world, join=True)
        res = dict(out)
    for r in range(world):
        t, v = res[r]
        assert t == 2.0
        assert v == pytest.approx(2 * 1000 / 2.0)


def test_single_process_needs_no_group():
    import bench

    assert bench.aggregate_replicas(0.25, 1, 100) == (0.25, 400.0)
