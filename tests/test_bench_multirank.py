"""The N > 1 path of bench.py (independent replicas, max-over-ranks timing)
with world_size 2 gloo ranks on CPU."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    t = bench.reduce_max(10.0 + 5.0 * rank)  # rank 1 is slower
    out[rank] = (t, bench.replica_throughput(1000, 4, world, t))
    dist.barrier()
    dist.destroy_process_group()


def test_replicas_take_the_slowest_rank():
    mgr = mp.get_context("spawn").Manager()
    out = mgr.dict()
    port = _free_port()
    mp.start_processes(_worker, args=(2, port, out), nprocs=2, start_method="spawn", join=True)
    assert out[0][0] == 15.0 and out[1][0] == 15.0
    # 2 replicas x 1000 rows x 4 steps in 15 ms
    assert abs(out[0][1] - 2 * 1000 * 4 / 0.015) < 1e-6


def test_single_rank_identity():
    import bench
    assert bench.reduce_max(3.5) == 3.5
    assert bench.replica_throughput(100, 2, 1, 1.0) == 200_000.0
