"""The multi-rank host logic of the benchmark on CPU (gloo, world size 2,
127.0.0.1): the whole-job rate takes the slowest rank's time and all ranks'
cells, and a cell range splits into disjoint contiguous blocks that cover it.
The step itself has no data-path collective (cells are independent)."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    import torch.distributed as dist
    import bench
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        ms_local = [2.0, 5.0][rank]
        ms, rate = bench.job_rate(dist, world, ms_local, 1000, "cpu")
        first, count = bench.cell_shard(10_001, rank, world)
        out[rank] = (ms, rate, first, count)
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_job_rate_and_shards_over_two_ranks():
    import torch.multiprocessing as mp
    world = 2
    port = _free_port()
    mgr = mp.Manager()
    out = mgr.dict()
    mp.spawn(_worker, args=(world, port, out), nprocs=world, join=True)
    for rank in range(world):
        ms, rate, first, count = out[rank]
        assert ms == 5.0                                   # the slowest rank
        assert abs(rate - 2 * 1000 / 5e-3) < 1e-6
    blocks = sorted((out[r][2], out[r][3]) for r in range(world))
    assert blocks[0][0] == 0 and blocks[0][0] + blocks[0][1] == blocks[1][0]
    assert blocks[1][0] + blocks[1][1] == 10_001


def test_single_rank_needs_no_collective():
    import bench
    ms, rate = bench.job_rate(None, 1, 4.0, 500, "cpu")
    assert ms == 4.0 and rate == 500 / 4e-3
    assert bench.cell_shard(7, 0, 1) == (0, 7)
