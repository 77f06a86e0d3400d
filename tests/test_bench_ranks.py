"""The benchmark's multi-rank path on CPU: two gloo ranks, each with its own
replica's time and edge count, agree on the whole-job throughput (all ranks' edges
over the slowest rank's time)."""
import os
import sys

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _rank(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    sys.path.insert(0, ROOT)
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    # rank r: 1 + r seconds for 100 (r + 1) edges; e2e and FP64 twice as slow
    t = 1.0 + rank
    vals = torch.tensor([t, 100.0 * (rank + 1), 2 * t, 100.0 * (rank + 1), 4 * t,
                         100.0 * (rank + 1)], dtype=torch.float64)
    out[rank] = bench.aggregate_ranks(vals, world, dist)
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_aggregate():
    world, port = 2, 29517
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_rank, args=(world, port, out), nprocs=world, join=True)
        res = dict(out)
    # edges 100 + 200 over the slowest time 2 s (4 s, 8 s)
    for r in range(world):
        assert res[r] == pytest.approx((150.0, 75.0, 37.5))
