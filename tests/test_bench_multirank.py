"""The benchmark's multi-rank bookkeeping on CPU: two gloo ranks (the same
code path the NCCL ranks take on GPUs, with the reduction on the host)."""
import os
import socket
import sys

import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, totals, steps, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    q.put((rank, bench.job_time(totals[rank], steps, world, "cpu")))
    dist.barrier()
    dist.destroy_process_group()


def test_job_time_is_the_slowest_rank_over_the_whole_job():
    """Every rank reports the longest timed region; the value is the time per
    frontal solve of the job (per-step time / number of ranks, each rank solving
    one front per step)."""
    world, steps = 2, 4
    q = mp.get_context("spawn").SimpleQueue()
    mp.spawn(_worker, args=(world, _free_port(), [10.0, 14.0], steps, q), nprocs=world, join=True)
    res = dict(q.get() for _ in range(world))
    for r in range(world):
        total, per_step, value = res[r]
        assert total == 14.0 and per_step == 3.5 and value == 1.75


def test_job_time_single_rank_needs_no_process_group():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.job_time(12.0, 3, 1, "cpu") == (12.0, 4.0, 4.0)
