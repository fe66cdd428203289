"""The benchmark's N > 1 path on CPU: under torchrun every rank runs an independent replica (the
step does not shard, no data-path collective); the only cross-rank operation is one element-wise
max of the timed totals, which every rank must join before rank 0 alone reports.  Two gloo ranks
on 127.0.0.1 check that reduction and the whole-job aggregate."""
import os
import socket
import sys

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
    import bench

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        # rank r timed totals: r + 1 ms for the first form, 10 - r for the second, 0 for an absent form
        got = bench.max_over_ranks([rank + 1.0, 10.0 - rank, 0.0], dist, "cpu")
        out[rank] = got
    finally:
        dist.destroy_process_group()


def test_max_over_ranks_with_two_gloo_ranks():
    world, port = 2, _free_port()
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_worker, args=(world, port, out), nprocs=world, join=True)
        res = dict(out)
    assert res[0] == res[1] == [2.0, 10.0, 0.0]


def test_aggregate_is_whole_job_over_the_slowest_rank():
    sys.path.insert(0, ROOT)
    import bench

    assert bench.max_over_ranks([1.5, 2.0]) == [1.5, 2.0]
    # 2 ranks x 524288 nodes x 100 steps in 5 ms (slowest rank) = 20971.52 MLUPS
    assert abs(bench.aggregate_mlups(2, 524288, 100, 5.0) - 20971.52) < 1e-9
    assert abs(bench.aggregate_mlups(1, 524288, 100, 5.0) - 10485.76) < 1e-9
