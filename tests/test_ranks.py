"""The benchmark's multi-process reduction (one replica bed per rank, no
data-path collective): two gloo ranks on the CPU agree on the slowest rank's
time and on the whole-job rate."""
import json
import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank(rank, world, port, outdir):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    t = bench.rank_max(1.5 + rank, "cpu")          # rank 1 is the slow one
    rate = bench.job_throughput(1000, world, t)
    with open(os.path.join(outdir, f"rank{rank}.json"), "w") as f:
        json.dump([t, rate], f)
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_take_the_slowest_time(tmp_path):
    # ranks are spawned (never forked from this multi-threaded process) and
    # report through files
    world = 2
    mp.spawn(_rank, args=(world, _free_port(), str(tmp_path)), nprocs=world, join=True)
    got = [json.load(open(tmp_path / f"rank{r}.json")) for r in range(world)]
    assert got[0] == got[1] == [2.5, world * 1000 / 2.5]


def test_single_process_is_the_identity():
    import bench
    assert not dist.is_initialized()
    assert bench.rank_max(3.25) == 3.25
    assert bench.job_throughput(10, 1, 2.0) == 5.0
