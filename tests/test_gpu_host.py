"""Eq. 12 from host buffers with overlapped transfers (dc_reconstruct_host)
against the device-resident path and the FP64 oracle."""
import numpy as np
import pytest
import torch

from oracle import oracle as orc
from paper_2410_14900_gb300 import api

from cases import arc_open, circle64, phantom_projections, ragged, rel_l2

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("name", ["circle64", "ragged", "arc_open"])
@pytest.mark.parametrize("n_slabs", [0, 1, 2, 3])
def test_host_pipeline_equals_device_path(name, n_slabs):
    case = {"circle64": circle64, "ragged": ragged, "arc_open": arc_open}[name]()
    geom = api.Geometry(case.desc, case.P, case.vdl)
    g = phantom_projections(case).astype(np.float32)
    g_host = torch.from_numpy(g).pin_memory()
    vol_host = torch.empty((case.B,) + geom.vol_shape).pin_memory()
    api.dc_reconstruct_host(geom, g_host, vol_host, n_slabs=n_slabs, relu=(n_slabs == 2))
    torch.cuda.synchronize()
    ref = api.reconstruct(geom, torch.as_tensor(g, device="cuda"), relu=(n_slabs == 2))
    torch.cuda.synchronize()
    assert rel_l2(vol_host.double().numpy(), ref.double().cpu().numpy()) < 1e-6
    if n_slabs == 0:
        og = orc.Geometry(case.desc, case.P, case.vdl)
        assert rel_l2(vol_host.double().numpy(), orc.reconstruct(og, g, None)) < 1e-4
    api.dc_sync_status(geom)


def test_host_pipeline_storage_forms_and_pageable_memory():
    case = circle64()
    geom = api.Geometry(case.desc, case.P, case.vdl)
    g = phantom_projections(case).astype(np.float32)
    gd = torch.as_tensor(g, device="cuda")
    for dt in ("bf16", "f16", "f32x2"):
        vol_host = torch.empty((1,) + geom.vol_shape)          # pageable on purpose
        api.dc_reconstruct_host(geom, torch.from_numpy(g), vol_host, dtype=dt, kahan=True)
        torch.cuda.synchronize()
        ref = api.reconstruct(geom, gd, dtype=dt, kahan=True)
        torch.cuda.synchronize()
        assert rel_l2(vol_host.double().numpy(), ref.double().cpu().numpy()) < 1e-6


def test_host_pipeline_back_to_back_calls_reuse_buffers():
    """Two calls in a row on the same device buffers: the second may not
    overwrite g_dev before the first call's filter has read it."""
    case = ragged(B=2)
    geom = api.Geometry(case.desc, case.P, case.vdl)
    g1 = phantom_projections(case, seed=1).astype(np.float32)
    g2 = phantom_projections(case, seed=7).astype(np.float32)
    shp = (case.B, geom.V, geom.H, geom.W)
    bufs = dict(g_dev=torch.empty(shp, device="cuda"), gF=torch.empty(shp, device="cuda"),
                vol_dev=torch.empty((case.B,) + geom.vol_shape, device="cuda"))
    outs, ins = [], []   # host buffers stay alive until the stream has run
    for g in (g1, g2):
        vh = torch.empty((case.B,) + geom.vol_shape).pin_memory()
        gh = torch.from_numpy(g).pin_memory()
        api.dc_reconstruct_host(geom, gh, vh, **bufs)
        outs.append(vh)
        ins.append(gh)
    torch.cuda.synchronize()
    for g, vh in zip((g1, g2), outs):
        ref = api.reconstruct(geom, torch.as_tensor(g, device="cuda"))
        torch.cuda.synchronize()
        assert rel_l2(vh.double().numpy(), ref.double().cpu().numpy()) < 1e-6


def test_host_pipeline_argument_errors():
    from paper_2410_14900_gb300 import _lib as L
    case = circle64()
    geom = api.Geometry(case.desc, case.P, case.vdl)
    Lh = L.load()
    shp = (1, geom.V, geom.H, geom.W)
    gd = torch.empty(shp, device="cuda")
    gF = torch.empty(shp, device="cuda")
    vd = torch.empty((1,) + geom.vol_shape, device="cuda")
    gh = torch.empty(shp).pin_memory()
    vh = torch.empty((1,) + geom.vol_shape).pin_memory()
    args = [geom.handle, 1, gh.data_ptr(), None, gd.data_ptr(), gF.data_ptr(), L.DC_F32, None,
            vd.data_ptr(), vh.data_ptr(), 0, 0, None]
    for i, bad in ((2, None), (9, None), (4, None), (8, None), (11, -1), (1, 0), (10, 64),
                   (6, 7)):
        a = list(args)
        a[i] = bad
        assert Lh.dc_reconstruct_host(*a) == L.DC_ERR_ARG, (i, bad)
    assert Lh.dc_reconstruct_host(*args) == L.DC_OK
    torch.cuda.synchronize()
    api.dc_sync_status(geom)
