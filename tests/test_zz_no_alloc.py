"""The allocation-free line-sum entry point (dc_radon2d_noalloc).

It serves callers that cannot allocate device memory when they run (a
fixed-budget real-time loop, or a host embedding the library in another
runtime's memory pool).  Through the C ABI it must give the same line sums
as dc_radon2d of a geometry handle, on two calls in a row (the fixed work
area keeps the previous call's contents, which must not leak), and reject
sizes beyond its fixed maximum.  This file is collected last on purpose.
"""
import ctypes

import numpy as np
import pytest
import torch

from oracle import oracle as orc
from paper_2410_14900_gb300 import _lib as L
from paper_2410_14900_gb300 import api, synth

from cases import rel_l2

pytestmark = pytest.mark.gpu


def _geometry(V, H, W, p, n_mu, n_s, ds):
    o = synth.sinusoid_orbit(V)
    desc = dict(n_views=V, det_rows=H, det_cols=W, n_mu=n_mu, n_s=n_s, pitch=p, ds=ds,
                vol_x=8, vol_y=8, vol_z=8, voxel=(1.0, 1.0, 1.0), closed_orbit=1)
    return api.Geometry(desc, synth.projection_matrices(o, H, W, p), o.vdl)


@pytest.mark.parametrize("V,H,W,p,n_mu,n_s,ds", [(6, 64, 64, 2.0, 180, 64, 2.0),
                                                 (5, 37, 50, 1.5, 33, 45, 1.7)])
def test_noalloc_matches_handle_entry_point_twice(V, H, W, p, n_mu, n_s, ds):
    Lh = L.load()
    geom = _geometry(V, H, W, p, n_mu, n_s, ds)
    cu, cv = (W - 1) / 2.0, (H - 1) / 2.0   # principal point of every view
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    for seed in (1, 2):                      # two calls in a row, new data each
        gen = torch.Generator(device="cuda")
        gen.manual_seed(seed)
        img = torch.randn((1, V, H, W), device="cuda", generator=gen)
        ref = api.dc_radon2d(geom, img)
        out = torch.full((V, n_mu, n_s), float("nan"), device="cuda")
        rc = Lh.dc_radon2d_noalloc(V, H, W, n_mu, n_s, p, ds, cu, cv,
                                   ctypes.c_void_p(img.data_ptr()),
                                   ctypes.c_void_p(out.data_ptr()), stream)
        assert rc == L.DC_OK, Lh.dc_last_error()
        torch.cuda.synchronize()
        got = out.double().cpu().numpy()
        want = ref[0].double().cpu().numpy()
        assert np.isfinite(got).all()
        assert rel_l2(got, want) < 2e-6
        # and directly against the FP64 oracle's Joseph line sums (Eq. 7)
        img_h = img[0].double().cpu().numpy()
        for i in range(V):
            ref_o = orc.radon(img_h[i], p, n_mu, n_s, ds, cu, cv)
            assert rel_l2(got[i], ref_o) < 2e-6


def test_noalloc_rejects_sizes_beyond_its_maximum():
    Lh = L.load()
    x = torch.zeros(4, device="cuda")
    ptr = ctypes.c_void_p(x.data_ptr())
    # one 4096 x 4096 image needs 64 MiB of work area: more than the fixed 32 MiB
    rc = Lh.dc_radon2d_noalloc(1, 4096, 4096, 90, 4096, 1.0, 1.0, 2047.5, 2047.5, ptr, ptr, None)
    assert rc == L.DC_ERR_ARG
    assert b"fixed" in Lh.dc_last_error()
    # the limit is H * round4(W) * 4 bytes <= 32 MiB - 256 KiB: 2040 rows of
    # 4096 floats are beyond it (2032 rows fill it exactly)
    rc = Lh.dc_radon2d_noalloc(1, 2040, 4096, 90, 64, 1.0, 1.0, 2047.5, 1019.5, ptr, ptr, None)
    assert rc == L.DC_ERR_ARG
    assert b"fixed" in Lh.dc_last_error()
    cap = (32 << 20) - (256 << 10)
    assert 2032 * 4096 * 4 == cap < 2040 * 4096 * 4
    rc = Lh.dc_radon2d_noalloc(1, 64, 64, 4096, 64, 1.0, 1.0, 31.5, 31.5, ptr, ptr, None)
    assert rc == L.DC_ERR_ARG
    rc = Lh.dc_radon2d_noalloc(1, 64, 64, 90, 64, 1.0, 1.0, 31.5, 31.5, None, ptr, None)
    assert rc == L.DC_ERR_ARG
