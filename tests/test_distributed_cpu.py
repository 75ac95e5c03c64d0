"""The N > 1 bench path runs independent replicas (a single transform does not
shard): every rank times its own steps, the job time is the max over ranks
and the value sums the ranks' units.  Checked with world size 2 on gloo."""
import os
import sys

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _worker(rank, world, port, out):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    # rank r "measured" (r + 1) * 100 ms over 10 steps for 1000 nodes
    agg = bench.aggregate_replicas((rank + 1) * 100.0, 1000, 10)
    dist.barrier()
    out[rank] = (agg["world"], agg["ms_total_max"], agg["ms_per_step"], agg["value"])
    dist.destroy_process_group()


def test_replica_aggregation_world2_gloo():
    port = 29500 + (os.getpid() % 1000)
    mgr = mp.Manager()
    out = mgr.dict()
    mp.spawn(_worker, args=(2, port, out), nprocs=2, join=True)
    for r in range(2):
        world, tmax, mps, value = out[r]
        assert world == 2
        assert tmax == pytest.approx(200.0)            # the slowest rank
        assert mps == pytest.approx(20.0)
        assert value == pytest.approx(2 * 1000 / 0.020)  # all ranks' units over the slowest time


def test_replica_aggregation_single_process():
    sys.path.insert(0, ROOT)
    import bench
    agg = bench.aggregate_replicas(50.0, 2000, 5)
    assert agg["world"] == 1 and agg["ms_per_step"] == pytest.approx(10.0)
    assert agg["value"] == pytest.approx(2000 / 0.010)
