"""World-size-2 gloo ranks on the CPU: disjoint work per rank, the slowest
rank's time as the job's time, and the whole-job per-volume figure."""
import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

from paper_2410_14900_gb300 import sharding


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        seed = sharding.rank_seed(6, rank)
        seeds = [None] * world
        dist.all_gather_object(seeds, seed)
        t = sharding.max_over_ranks(10.0 + 5.0 * rank, dist)
        lo, hi = sharding.rank_views(496, rank, world)
        spans = [None] * world
        dist.all_gather_object(spans, (lo, hi))
        dist.barrier()
        if rank == 0:
            out.put((seeds, t, spans, sharding.whole_job_ms_per_volume(t, 1, world)))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_partition_and_reduce():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    try:
        seeds, t, spans, per_vol = q.get(timeout=120)
    finally:
        for p in procs:
            p.join(timeout=60)
            if p.is_alive():
                p.kill()
    assert len(set(seeds)) == 2                     # independent problems
    assert t == 15.0                                # the slowest rank
    assert per_vol == 7.5                           # 2 volumes in 15 ms
    covered = sorted(v for lo, hi in spans for v in range(lo, hi))
    assert covered == list(range(496))              # views split without overlap


def test_single_process_defaults():
    assert sharding.max_over_ranks(3.0) == 3.0
    assert sharding.rank_views(10, 0, 1) == (0, 10)
    assert sharding.rank_seed(1, 0) == 1
