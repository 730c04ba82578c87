"""The multi-rank host logic of bench.py on CPU (gloo, world size 2): every rank gets the slowest rank's
time and the whole-job rate, and each rank draws its own query batch of the same scene (weak scaling,
replicas only: no data-path collective)."""
import os
import socket
import sys

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench

    total, rate = bench.whole_job_rate(1.0 + rank, world, 1000, 5, torch.device("cpu"))

    class A:
        samples, queries = 2000, 512

    w = bench.make_workload(A, rank)
    out[rank] = (total, rate, w.xq.copy(), len(w.x))
    dist.barrier()
    dist.destroy_process_group()


def test_two_ranks_gloo():
    world = 2
    port = _free_port()
    with mp.Manager() as mgr:
        out = mgr.dict()
        mp.spawn(_worker, args=(world, port, out), nprocs=world, join=True)
        res = dict(out)
    for r in range(world):
        total, rate, xq, S = res[r]
        assert total == 2.0  # the slowest rank's seconds
        assert rate == world * 1000 * 5 / 2.0
        assert xq.shape == (512, 3) and S == 2000
    assert not np.array_equal(res[0][2], res[1][2])  # each rank its own query batch
