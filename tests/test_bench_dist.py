"""The multi-rank path of bench.py (one independent replica per rank, timing reduced
with a max over ranks) on CPU with the gloo backend, world size 2."""
import os
import sys

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _worker(rank, world, port, out):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    assert bench.dist_info() == (world, rank, rank)
    # each rank "times" a different duration; all must agree on the slowest
    ms = 100.0 + 50.0 * rank
    mx = bench.reduce_max(ms, world)
    rate = bench.aggregate_rate(1000 * 10, world, mx)
    out[rank] = (mx, rate)
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_timing_reduction_gloo():
    world = 2
    port = 29500 + (os.getpid() % 1000)
    mgr = mp.Manager()
    out = mgr.dict()
    mp.spawn(_worker, args=(world, port, out), nprocs=world, join=True)
    for r in range(world):
        mx, rate = out[r]
        assert mx == 150.0
        assert rate == pytest.approx(2 * 10000 / 0.150)
