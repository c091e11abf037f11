"""World-size-2 gloo ranks on the CPU.

- Independent problems: disjoint work per rank, the slowest rank's time as
  the job's time, and the whole-job per-volume figure.
- One problem split over the ranks (the multi-GPU design of the path): each
  rank runs the FP64 oracle on its share (its views for the filter, its
  z-slab for the backprojection), the ranks exchange g^F (all-gather) or
  partial volumes (reduced slab by slab), and the gathered volume must equal
  the single-rank oracle reconstruction of Eq. 12 (the sum over views of
  Eq. 5 is what the exchange has to reproduce).
- Data-parallel training: dL/dW of each rank's batch items, summed over the
  ranks, equals the single-rank gradient of the whole batch.
"""
import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

from paper_2410_14900_gb300 import sharding

from cases import phantom_projections, ragged, random_weights


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


# ------------------------------------------------------- split reconstruction
def _split_worker(rank, world, port, out, mode):
    import numpy as np

    from oracle import oracle as orc

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        case = ragged(B=2)
        d = case.desc
        V, Z, Y, X = d["n_views"], d["vol_z"], d["vol_y"], d["vol_x"]
        g = phantom_projections(case, n=4)                  # same seeded data on every rank
        W = random_weights(case)
        og = orc.Geometry(d, case.P, case.vdl)
        lo, hi = sharding.rank_views(V, rank, world)

        def filter_views(g_local):
            return torch.from_numpy(orc.filter(og, g_local.numpy(), W, views=np.arange(lo, hi)))

        def backproject_slab(gF_all, z0, z1):
            idx = np.arange(z0 * Y * X, z1 * Y * X)
            return torch.from_numpy(np.stack([
                orc.backproject_points(og, gF_all[b].numpy(), idx).reshape(z1 - z0, Y, X)
                for b in range(gF_all.shape[0])]))

        def backproject_views(gF_local):
            sub = dict(d)
            sub["n_views"] = hi - lo
            og_sub = orc.Geometry(sub, case.P[lo:hi], case.vdl[lo:hi])
            return torch.from_numpy(orc.backproject(og_sub, gF_local.numpy()))

        g_local = torch.from_numpy(np.ascontiguousarray(g[:, lo:hi]))
        if mode == "gather":
            slab, (z0, z1) = sharding.split_reconstruct(dist, rank, world, V, Z, g_local,
                                                        filter_views, backproject_slab, align=8)
        else:
            slab, (z0, z1) = sharding.split_reconstruct_reduce(dist, rank, world, Z, g_local,
                                                               filter_views, backproject_views,
                                                               align=8)
        slabs = [None] * world
        dist.all_gather_object(slabs, (z0, z1, slab.numpy()))
        if rank == 0:
            vol = np.concatenate([s[2] for s in sorted(slabs, key=lambda t: t[0])], axis=1)
            ref = orc.reconstruct(og, g, W)
            out.put((vol, ref, [(a, b) for a, b, _ in slabs], [(lo, hi)]))
    finally:
        dist.destroy_process_group()


def _grad_worker(rank, world, port, out):
    import numpy as np

    from oracle import oracle as orc

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        case = ragged(B=2)
        d = case.desc
        g = phantom_projections(case, n=4)
        W = random_weights(case)
        G = np.random.default_rng(9).normal(size=g.shape)   # dL/dg^F of the batch
        og = orc.Geometry(d, case.P, case.vdl)
        b0, b1 = sharding.rank_views(g.shape[0], rank, world)   # this rank's batch items
        _, gW = orc.filter_adjoint(og, g[b0:b1], G[b0:b1], W, want_grad_g=False)
        total = sharding.allreduce_grad(dist, torch.from_numpy(gW))
        if rank == 0:
            _, ref = orc.filter_adjoint(og, g, G, W, want_grad_g=False)
            out.put((total.numpy(), ref))
    finally:
        dist.destroy_process_group()


def _run(target, *args):
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=target, args=(r, 2, port, q) + args) for r in range(2)]
    for p in procs:
        p.start()
    try:
        return q.get(timeout=300)
    finally:
        for p in procs:
            p.join(timeout=60)
            if p.is_alive():
                p.kill()


@pytest.mark.parametrize("mode", ["gather", "reduce"])
def test_split_reconstruction_equals_single_rank_oracle(mode):
    import numpy as np
    vol, ref, spans, _ = _run(_split_worker, mode)
    assert sorted(spans) == [(0, 16), (16, 21)]          # both ranks own planes
    assert vol.shape == ref.shape
    # same FP64 arithmetic per voxel; only the order of the sum over views
    # differs in the reduce form
    assert np.max(np.abs(vol - ref)) <= 1e-12 * np.max(np.abs(ref))


def test_data_parallel_grad_W_equals_single_rank():
    import numpy as np
    total, ref = _run(_grad_worker)
    assert np.max(np.abs(total - ref)) <= 1e-12 * np.max(np.abs(ref))


def test_partitions_cover_everything_once():
    for V in (1, 7, 23, 496):
        for world in (1, 2, 3, 8):
            spans = [sharding.rank_views(V, r, world) for r in range(world)]
            assert [v for lo, hi in spans for v in range(lo, hi)] == list(range(V))
            sizes = [hi - lo for lo, hi in spans]
            assert max(sizes) - min(sizes) <= 1
    for Z in (1, 21, 64, 512, 513):
        for world in (1, 2, 3, 8):
            spans = [sharding.rank_slab(Z, r, world) for r in range(world)]
            assert [z for a, b in spans for z in range(a, b)] == list(range(Z))
            assert all(a % 32 == 0 for a, b in spans if b > a)
