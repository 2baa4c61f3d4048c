"""The replicas path of bench.py on CPU: two gloo ranks, the job time is the
slower rank's and the work is the sum over ranks."""
import os
import sys

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _rank(rank, world, port, out):
    sys.path.insert(0, ROOT)
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench

    res = bench.reduce_over_ranks(dist, 1.0 + rank, 2.0 + 3 * rank, 100.0 * (rank + 1), 10.0, "cpu")
    out[rank] = res
    dist.destroy_process_group()


def test_reduce_over_ranks_gloo():
    port = 29500 + os.getpid() % 1000
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_rank, args=(2, port, out), nprocs=2, join=True)
        for r in (0, 1):
            assert out[r] == (2.0, 5.0, 300.0, 20.0)


def test_single_rank_is_identity():
    sys.path.insert(0, ROOT)
    import bench

    assert bench.reduce_over_ranks(None, 1.5, 2.5, 7.0, 8.0, "cpu") == (1.5, 2.5, 7.0, 8.0)
