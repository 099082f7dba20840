"""The N > 1 path of bench.py on CPU: two gloo ranks, each timing its own
replica; the job time is the slowest rank's and the job rate counts every
rank's lattice updates (replicas only: no data-path collective)."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    my_ms = 10.0 + 5.0 * rank            # rank 1 is the slow one
    mx = bench.reduce_max(my_ms, dist, "cpu")
    out[rank] = (mx, bench.job_mlups(1000, 20, world, mx))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_take_the_slowest_time():
    world = 2
    port = _free_port()
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_worker, args=(world, port, out), nprocs=world, join=True)
        res = dict(out)
    assert res[0][0] == res[1][0] == 15.0
    # 2 replicas x 1000 nodes x 20 steps in 15 ms
    assert res[0][1] == pytest.approx(2 * 1000 * 20 / 15e-3 / 1e6)


def test_single_process_needs_no_group():
    import bench
    assert bench.reduce_max(3.5, None, "cpu") == 3.5
