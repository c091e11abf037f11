"""The multi-GPU split of one problem with the CUDA backend, on one GPU: the
ranks run one after another in this process and the exchange is emulated
(the all-gather of g^F is a concatenation over the ranks' view ranges, the
slab reduction a sum of the ranks' partial volumes), so no kernel waits on
another.  What is checked is the CUDA side of the split: geometry handles
of a rank's views (with the whole orbit's tangents, Eq. 10's K) and of a
rank's z-slab (shifted volume centre), and that Eq. 5's sum over views
reassembles to the single-GPU reconstruction and to the FP64 oracle.
"""
import numpy as np
import pytest
import torch

from oracle import oracle as orc
from paper_2410_14900_gb300 import api, sharding

from cases import arc_open, circle64, phantom_projections, ragged, random_weights, rel_l2

pytestmark = pytest.mark.gpu

CASES = {"circle64": circle64, "ragged": ragged, "arc_open": arc_open}


def _dev(a):
    return torch.as_tensor(np.ascontiguousarray(a, dtype=np.float32), device="cuda")


@pytest.mark.parametrize("name", list(CASES))
@pytest.mark.parametrize("world", [2, 3])
@pytest.mark.parametrize("storage", ["f32", "f32x2"])
def test_split_by_views_and_slabs_reassembles(name, world, storage):
    case = CASES[name]()
    d = case.desc
    g = phantom_projections(case).astype(np.float32)
    W = random_weights(case).astype(np.float32)
    gt, Wt = _dev(g), _dev(W)
    full = api.Geometry(d, case.P, case.vdl)
    ref_gpu = api.reconstruct(full, gt, Wt, dtype=storage)

    backends = [sharding.cuda_backend(d, case.P, case.vdl, r, world, Wt, storage)
                for r in range(world)]
    # each rank filters its own views
    parts = []
    for r, (filter_views, _, _) in enumerate(backends):
        lo, hi = sharding.rank_views(d["n_views"], r, world)
        parts.append(filter_views(gt[:, lo:hi].contiguous()))
    gF_all = torch.cat(parts, dim=1).contiguous()       # the all-gather
    # each rank backprojects every view into its slab
    slabs = []
    for r, (_, backproject_slab, _) in enumerate(backends):
        z0, z1 = sharding.rank_slab(d["vol_z"], r, world)
        slabs.append(backproject_slab(gF_all, z0, z1))
    vol = torch.cat(slabs, dim=1)
    torch.cuda.synchronize()
    assert vol.shape == ref_gpu.shape
    # the same kernels; voxel coordinates taken from the slab's centre round
    # differently in FP32 (~1e-7 of a position), views summed in another
    # order: agreement to FP32 rounding, well inside the oracle's 1e-4
    assert rel_l2(vol.double().cpu().numpy(), ref_gpu.double().cpu().numpy()) < 1e-5
    og = orc.Geometry(d, case.P, case.vdl)
    assert rel_l2(vol.double().cpu().numpy(), orc.reconstruct(og, g, W)) < 1e-4

    # the other exchange: each rank's views into the whole volume, summed
    partial = torch.zeros_like(ref_gpu)
    for (filter_views, _, (gv, _)), r in zip(backends, range(world)):
        lo, hi = sharding.rank_views(d["n_views"], r, world)
        gF_r = filter_views(gt[:, lo:hi].contiguous())
        partial += api.dc_backproject(gv, gF_r)
    torch.cuda.synchronize()
    assert rel_l2(partial.double().cpu().numpy(), ref_gpu.double().cpu().numpy()) < 1e-5
    for _, _, (gv, gs) in backends:
        api.dc_sync_status(gv)
        gv.close()
        if gs is not None:
            gs.close()
    full.close()
