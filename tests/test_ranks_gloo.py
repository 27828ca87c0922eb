"""The multi-GPU form is replicas only: each rank advances its own grid, the
job time is the slowest rank's and the throughput counts every rank's cells.
This runs that aggregation with two gloo ranks on the CPU (no GPU needed)."""
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
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import bench
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank,
                            world_size=world)
    # rank r took (10 + 5 r) ms for a grid of (1000 + r) cells, 100 steps
    ms, value = bench.aggregate_over_ranks(10.0 + 5 * rank, 1000 + rank, 100, dist, "cpu")
    out[rank] = (ms, value)
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_take_the_slowest_time_and_all_cells():
    world, port = 2, _free_port()
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_worker, args=(world, port, out), nprocs=world, join=True)
        res = dict(out)
    slowest = 15.0
    cells = 1000 + 1001
    for rank in range(world):
        ms, value = res[rank]
        assert ms == slowest
        assert value == pytest.approx(cells * 100 / (slowest * 1e-3) / 1e9)


def test_single_rank_needs_no_process_group():
    import bench
    ms, value = bench.aggregate_over_ranks(20.0, 4096, 10)
    assert ms == 20.0 and value == pytest.approx(4096 * 10 / 0.02 / 1e9)
