"""The multi-replica aggregation of bench.py, on CPU with two gloo ranks.

The path does not shard: N GPUs run N independent replicas of the workload.
The job's throughput is every rank's units over the slowest rank's time, so
a rank that finishes early must not raise the figure.
"""
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

torch = pytest.importorskip("torch")


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out_dir):
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    import bench
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    # rank r "took" 1.5 + r seconds for the same 20 steps
    secs = bench.max_over_ranks(1.5 + rank)
    value = bench.replica_throughput(20, secs, world)
    with open(os.path.join(out_dir, f"r{rank}.txt"), "w") as f:
        f.write(f"{secs} {value}\n")
    dist.barrier()
    dist.destroy_process_group()


def test_max_over_ranks_and_throughput(tmp_path):
    world, port = 2, _free_port()
    torch.multiprocessing.spawn(_rank_main, args=(world, port, str(tmp_path)), nprocs=world, join=True)
    for r in range(world):
        secs, value = map(float, open(tmp_path / f"r{r}.txt").read().split())
        assert secs == 2.5              # every rank sees the slowest rank's time
        assert value == 2 * 20 / 2.5    # both replicas' steps over that time


def test_single_process_is_identity():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(3.25) == 3.25
    assert bench.replica_throughput(10, 2.0, 1) == 5.0
