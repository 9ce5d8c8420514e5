"""The multi-process path of bench.py on CPU: two gloo ranks (one process per
GPU in production, replicas of the same workload) meet at the barriers and
agree on the maximum per-step time and the job-wide throughput."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    r, w, _ = bench.dist_env()
    assert (r, w) == (rank, world)
    bench.rank_barrier(world)
    t = bench.max_over_ranks(0.1 * (rank + 1), world, device="cpu")
    out[rank] = (t, bench.replica_throughput(t, world))
    bench.rank_barrier(world)
    dist.destroy_process_group()


def test_two_gloo_ranks_agree_on_max_time():
    world = 2
    port = _free_port()
    mgr = mp.get_context("spawn").Manager()  # no fork of a process that holds OpenMP threads
    out = mgr.dict()
    mp.start_processes(_worker, args=(world, port, out), nprocs=world, join=True, start_method="spawn")
    for rank in range(world):
        t, thr = out[rank]
        assert t == pytest.approx(0.2)
        assert thr == pytest.approx(world * 2 / 0.2)
