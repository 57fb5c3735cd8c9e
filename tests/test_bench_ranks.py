"""Host logic of the multi-GPU bench path on CPU: two gloo ranks (127.0.0.1)
run the replica bookkeeping of bench.py -- distinct replica seeds, whole-job
throughput = all ranks' units over the slowest rank's time."""
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    local_ms = 10.0 * (rank + 1)                      # rank 1 is the slow one
    ms_max, value = bench.job_throughput(local_ms, 1000.0, world, "cpu")
    seeds = [None] * world
    dist.all_gather_object(seeds, bench.replica_seed(rank))
    out[rank] = (ms_max, value, seeds)
    dist.destroy_process_group()


def test_two_gloo_ranks_aggregate_like_the_bench():
    torch = pytest.importorskip("torch")
    import torch.multiprocessing as mp
    world = 2
    port = _free_port()
    with mp.Manager() as mgr:
        out = mgr.dict()
        mp.start_processes(_rank_main, args=(world, port, out), nprocs=world, join=True, start_method="spawn")
        res = dict(out)
    for rank in range(world):
        ms_max, value, seeds = res[rank]
        assert ms_max == 20.0                           # the slowest rank's time
        assert value == pytest.approx(2 * 1000.0 / 0.020)  # both ranks' units
        assert len(set(seeds)) == world                 # independent replicas


def test_single_process_is_the_identity():
    pytest.importorskip("torch")
    sys.path.insert(0, ROOT)
    import bench
    ms_max, value = bench.job_throughput(5.0, 100.0, 1, "cpu")
    assert ms_max == 5.0 and value == pytest.approx(100.0 / 0.005)
