"""Multi-rank host logic of bench.py on CPU (gloo, world size 2): ranks run
independent replicas of the model, the job time is the slowest rank's and the
throughput counts every rank's work.  No GPU is used."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    local_seconds = [1.5, 2.25][rank]
    mx = bench.reduce_max(local_seconds, dist, "cpu")
    value = bench.replica_throughput(world, 1048576, 100, mx)
    out[rank] = (mx, value)
    dist.barrier()
    dist.destroy_process_group()


def test_replica_reduction_world2():
    port = _free_port()
    mgr = mp.get_context("spawn").Manager()
    out = mgr.dict()
    mp.start_processes(_worker, args=(2, port, out), nprocs=2, start_method="spawn")
    assert out[0][0] == out[1][0] == 2.25
    assert out[0][1] == pytest.approx(2 * 1048576 * 100 / 2.25)


def test_single_rank_identity():
    import bench
    assert bench.reduce_max(3.0, None, "cpu") == 3.0
    assert bench.replica_throughput(1, 10, 5, 2.0) == 25.0
