"""Work partition of the reconstruction across ranks (one GPU each).

Two ways to use N ranks:

- independent problems (the benchmark's default): every rank reconstructs
  its own volume; nothing is exchanged on the data path, only the
  benchmark's barrier and its max-over-ranks timing talk to each other;
- one problem split over the ranks (`split_reconstruct`): Eq. 12 filters
  every view on its own (a1-a4 are per view), and the backprojection of
  Eq. 5 sums over all views.  Rank r filters its contiguous view range, the
  filtered projections g^F are all-gathered (FP32, or BF16 to halve the
  bytes), and rank r backprojects every view into its own z-slab of the
  volume.  The alternative exchange (`split_reconstruct_reduce`) backprojects
  each rank's views into the whole volume and sums the partial volumes
  slab by slab (a reduce-scatter); it moves the FP32 volume instead of g^F.
- training, data-parallel over the batch (`allreduce_grad`): each rank runs
  the forward and reverse mode on its batch items, and dL/dW is summed over
  the ranks.

The orchestration here is independent of the compute backend: the filter,
the backprojection of a slab and the collectives are passed in, so that the
same code drives the CUDA library (with NCCL) and CPU stand-ins (with gloo).
"""
from __future__ import annotations

from typing import Callable, Tuple


def rank_seed(base_seed: int, rank: int) -> int:
    """Seed of the phantom that rank `rank` reconstructs (disjoint per rank)."""
    return int(base_seed) + 1000 * int(rank)


def rank_views(n_views: int, rank: int, world: int) -> Tuple[int, int]:
    """Contiguous view range [lo, hi) of a rank when one problem's filter is
    split by views (each view is independent in the filter).  Ranges are as
    even as possible (sizes differ by at most one) and cover every view."""
    n_views, rank, world = int(n_views), int(rank), int(world)
    base, extra = divmod(n_views, world)
    lo = rank * base + min(rank, extra)
    return lo, lo + base + (1 if rank < extra else 0)


def rank_slab(n_z: int, rank: int, world: int, align: int = 32) -> Tuple[int, int]:
    """z-planes [z0, z1) of a rank's slab: slabs are whole multiples of
    `align` planes (the backprojector's box depth) where the volume allows,
    as even as possible, covering every plane; a rank may get an empty slab
    when there are fewer blocks of planes than ranks."""
    n_z, rank, world = int(n_z), int(rank), int(world)
    blocks = (n_z + align - 1) // align
    base, extra = divmod(blocks, world)
    b0 = rank * base + min(rank, extra)
    b1 = b0 + base + (1 if rank < extra else 0)
    return min(n_z, b0 * align), min(n_z, b1 * align)


def max_over_ranks(value: float, dist=None, device=None) -> float:
    """The slowest rank's time (the whole job finishes with it)."""
    if dist is None or not dist.is_available() or not dist.is_initialized():
        return float(value)
    import torch
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_ms_per_volume(ms_step_max: float, volumes_per_rank: int, world: int) -> float:
    """ms per volume of the whole job: all ranks' volumes in the slowest step."""
    return float(ms_step_max) / (int(volumes_per_rank) * int(world))


# ----------------------------------------------------------------- exchanges
def all_gather_views(dist, local, n_views: int, world: int, group=None):
    """Concatenate every rank's view range of g^F ([B][V_r][H][W] tensors)
    along the view axis into [B][V][H][W] on every rank.  Ranges may differ
    by one view, so each rank's block is padded to the largest range for the
    collective and trimmed afterwards."""
    import torch
    B, _, H, W = local.shape
    spans = [rank_views(n_views, r, world) for r in range(world)]
    vmax = max(hi - lo for lo, hi in spans)
    pad = torch.zeros((B, vmax, H, W), dtype=local.dtype, device=local.device)
    pad[:, :local.shape[1]] = local
    parts = [torch.empty_like(pad) for _ in range(world)]
    dist.all_gather(parts, pad.contiguous(), group=group)
    return torch.cat([p[:, :hi - lo] for p, (lo, hi) in zip(parts, spans)], dim=1)


def reduce_slabs(dist, partial, n_z: int, rank: int, world: int, group=None, align: int = 32):
    """Sum the ranks' partial volumes ([B][Z][Y][X]) and keep this rank's
    z-slab.  NCCL does this as one reduce-scatter; backends without one (the
    CPU's gloo) sum everything and slice."""
    import torch
    z0, z1 = rank_slab(n_z, rank, world, align)
    backend = dist.get_backend(group) if group is not None else dist.get_backend()
    if backend == "nccl":
        spans = [rank_slab(n_z, r, world, align) for r in range(world)]
        zmax = max(b - a for a, b in spans)
        B, _, Y, X = partial.shape
        chunks = []
        for a, b in spans:
            c = torch.zeros((B, zmax, Y, X), dtype=partial.dtype, device=partial.device)
            c[:, :b - a] = partial[:, a:b]
            chunks.append(c)
        out = torch.empty_like(chunks[0])
        dist.reduce_scatter(out, chunks, group=group)
        return out[:, :z1 - z0]
    total = partial.clone()
    dist.all_reduce(total, group=group)
    return total[:, z0:z1].contiguous()


def allreduce_grad(dist, grad, group=None):
    """dL/dW summed over the ranks' batch items (data-parallel training)."""
    dist.all_reduce(grad, group=group)
    return grad


# ------------------------------------------------------------ orchestration
def split_reconstruct(dist, rank: int, world: int, n_views: int, n_z: int,
                      g_local, filter_views: Callable, backproject_slab: Callable,
                      gather_dtype=None, group=None, align: int = 32):
    """Eq. 12 for one problem on `world` ranks, exchanging g^F.

    g_local          : [B][V_r][H][W], this rank's views (rank_views).
    filter_views     : g_local -> g^F of those views, [B][V_r][H][W].
    backproject_slab : (g^F of all views, z0, z1) -> [B][z1-z0][Y][X], Eq. 5
                       over every view for the planes [z0, z1).
    gather_dtype     : dtype of g^F on the wire (None keeps the filter's).
    Returns this rank's slab and its plane range.
    """
    gF_local = filter_views(g_local)
    if gather_dtype is not None and gF_local.dtype != gather_dtype:
        gF_local = gF_local.to(gather_dtype)
    gF_all = all_gather_views(dist, gF_local, n_views, world, group)
    z0, z1 = rank_slab(n_z, rank, world, align)
    return backproject_slab(gF_all, z0, z1), (z0, z1)


def split_reconstruct_reduce(dist, rank: int, world: int, n_z: int, g_local,
                             filter_views: Callable, backproject_views: Callable, group=None,
                             align: int = 32):
    """Eq. 12 for one problem on `world` ranks, exchanging partial volumes:
    each rank backprojects its own views into the whole volume
    (backproject_views: g^F of this rank's views -> [B][Z][Y][X]) and the
    partial sums are reduced slab by slab."""
    partial = backproject_views(filter_views(g_local))
    z0, z1 = rank_slab(n_z, rank, world, align)
    return reduce_slabs(dist, partial, n_z, rank, world, group, align), (z0, z1)


# --------------------------------------------------------------- CUDA backend
def view_subset_geometry(desc: dict, P, vdl, lo: int, hi: int):
    """Geometry handle of views [lo, hi) of an orbit.  The tangents a'(λ)Δλ
    must be those of the whole orbit: pass them (vdl [V][3]); central
    differences inside the subset would be one-sided at its ends."""
    import numpy as np

    from . import api
    if vdl is None:
        raise ValueError("view_subset_geometry needs the orbit's tangents (vdl)")
    sub = dict(desc)
    sub["n_views"] = hi - lo
    return api.Geometry(sub, np.ascontiguousarray(P[lo:hi]), np.ascontiguousarray(vdl[lo:hi]))


def slab_geometry(desc: dict, P, vdl, z0: int, z1: int):
    """Geometry handle whose volume is the planes [z0, z1) of desc's volume
    (same voxel centres, every view)."""
    from . import api
    sub = dict(desc)
    nz = int(desc["vol_z"])
    dz = float(desc["voxel"][2])
    c = list(desc.get("vol_center", (0.0, 0.0, 0.0)))
    c[2] = c[2] + (0.5 * (z0 + z1 - 1) - 0.5 * (nz - 1)) * dz
    sub["vol_z"] = z1 - z0
    sub["vol_center"] = tuple(c)
    return api.Geometry(sub, P, vdl)


def cuda_backend(desc: dict, P, vdl, rank: int, world: int, W=None, storage: str = "f32"):
    """filter_views / backproject_slab callables of `split_reconstruct` for
    the CUDA library on this rank's device: the filter runs on a handle of
    the rank's views (W rows of those views), the backprojection on a
    handle of every view whose volume is the rank's slab.  The third value
    holds the two handles (the view handle's volume is the whole volume, so
    it also backprojects the rank's views for `split_reconstruct_reduce`)."""
    from . import api
    if vdl is None:
        # tangents a'(λ)Δλ of the whole orbit (finite differences across the
        # rank's range ends), as the full geometry computes them
        full = api.Geometry(desc, P, None)
        vdl = api.dc_get_view_geometry(full)[:, 15:18].copy()
        full.close()
    lo, hi = rank_views(desc["n_views"], rank, world)
    z0, z1 = rank_slab(desc["vol_z"], rank, world)
    gv = view_subset_geometry(desc, P, vdl, lo, hi)
    gs = slab_geometry(desc, P, vdl, z0, z1) if z1 > z0 else None
    W_local = None if W is None else W[lo:hi].contiguous()

    def filter_views(g_local):
        gF, _ = api.dc_filter(gv, g_local, W_local, storage)
        return gF

    def backproject_slab(gF_all, a, b):
        import torch
        if gs is None:
            return torch.empty((gF_all.shape[0], 0, desc["vol_y"], desc["vol_x"]),
                               device=gF_all.device)
        return api.dc_backproject(gs, gF_all, None, kahan=(gF_all.dtype != torch.float32))

    return filter_views, backproject_slab, (gv, gs)
