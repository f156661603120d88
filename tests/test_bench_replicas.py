"""The bench's multi-GPU path is replicas only (every rank solves the whole
workload, no collective in the data path): the whole-job value is the units
all ranks processed over the slowest rank's time.  Checked here with two
gloo ranks on the CPU."""
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


def _rank(rank, world, port, ms, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    value, ms_max = bench.replica_value(torch, ms[rank], world, 320, 5, torch.device("cpu"))
    out[rank] = (value, ms_max)
    dist.barrier()
    dist.destroy_process_group()


def test_two_replicas_report_the_slowest_rank():
    world, port = 2, _free_port()
    ms = [400.0, 500.0]                      # 5 steps of 320 solves on each rank
    with mp.Manager() as mgr:
        out = mgr.dict()
        mp.spawn(_rank, args=(world, port, ms, out), nprocs=world, join=True)
        res = dict(out)
    for r in range(world):
        value, ms_max = res[r]
        assert ms_max == 500.0
        assert value == pytest.approx(world * 320 * 5 / 0.5)


def test_single_rank_needs_no_process_group():
    import bench
    value, ms_max = bench.replica_value(torch, 250.0, 1, 320, 5, torch.device("cpu"))
    assert ms_max == 250.0 and value == pytest.approx(320 * 5 / 0.25)
