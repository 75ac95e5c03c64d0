"""The N > 1 bench paths, checked with world size 2 on gloo.

Single transforms run as independent replicas (a single transform does not
shard): every rank times its own steps, the job time is the max over ranks
and the value sums the ranks' units.  The batched workload is split: its
independent problems are divided over the ranks with no collective on the
data path; the split must cover every problem exactly once, and each
rank's results must be the one-rank run's results for its problems."""
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


def _split_worker(rank, world, port, out):
    import numpy as np
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    from oracle import nfft as onfft
    from paper_2208_00049_gb300 import inputs
    probs = inputs.batched_problems(n_problems=64, sizes=(8, 12, 16))
    mine = bench.split_problems(bench.batch_weights(probs), world, rank)
    # this rank's results: the oracle's forward transform of its problems
    res = {i: onfft.forward(probs[i]["k"][:50], probs[i]["f"]) for i in mine}
    gathered = [None] * world
    dist.all_gather_object(gathered, (mine, res))
    agg = bench.aggregate_split(100.0 * (rank + 1), sum(probs[i]["M"] for i in mine), 10)
    out[rank] = (gathered, agg["value"], agg["ms_per_step"], agg["units"])
    dist.destroy_process_group()


def test_batched_split_world2_gloo():
    import numpy as np
    sys.path.insert(0, ROOT)
    from oracle import nfft as onfft
    from paper_2208_00049_gb300 import inputs
    port = 29700 + (os.getpid() % 1000)
    mgr = mp.Manager()
    out = mgr.dict()
    mp.spawn(_split_worker, args=(2, port, out), nprocs=2, join=True)
    probs = inputs.batched_problems(n_problems=64, sizes=(8, 12, 16))
    gathered, value, mps, units = out[0]
    owners = {}
    for r, (mine, res) in enumerate(gathered):
        for i in mine:
            assert i not in owners          # each problem on exactly one rank
            owners[i] = r
            want = onfft.forward(probs[i]["k"][:50], probs[i]["f"])   # the one-rank run
            assert np.array_equal(res[i], want)
    assert sorted(owners) == list(range(64))
    total = sum(p["M"] for p in probs)
    assert units == total
    assert mps == pytest.approx(20.0)                          # the slowest rank
    assert value == pytest.approx(total / 0.020)
    assert out[1][1] == pytest.approx(value)
