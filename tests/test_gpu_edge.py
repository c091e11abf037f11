"""Edge cases of the CUDA path against the FP64 oracle, through the C ABI.

- Voxels behind the source (depth <= 0) for some views, Eq. 5: those views
  give such voxels nothing.  The volume reaches beyond the source's circle,
  so the boxes holding those voxels take the backprojector's bounds-checked
  global-load path instead of a staged detector tile.
- Footprints larger than the staged detector tile (coarse voxels, fine
  pixels): every box takes the global-load path.
- A NaN / infinite redundancy weight: dc_sync_status reports
  DC_ERR_NONFINITE, only the outputs that depend on that weight are NaN, the
  flag clears, and a later call is unaffected.
"""
import numpy as np
import pytest
import torch

from oracle import oracle as orc
from paper_2410_14900_gb300 import _lib as L
from paper_2410_14900_gb300 import api, synth

from cases import phantom_projections, random_weights, rel_l2, Case

pytestmark = pytest.mark.gpu


def _dev(a):
    return torch.as_tensor(np.ascontiguousarray(a, dtype=np.float32), device="cuda")


def _host(t):
    torch.cuda.synchronize()
    return t.double().cpu().numpy()


def _case(orbit, H, W, p, n_mu, n_s, vol, voxel, B=1, name="edge"):
    desc = dict(n_views=orbit.n_views, det_rows=H, det_cols=W, n_mu=n_mu, n_s=n_s, pitch=p,
                ds=p, vol_x=vol[2], vol_y=vol[1], vol_z=vol[0], voxel=voxel,
                vol_center=(0.0, 0.0, 0.0), closed_orbit=1)
    return Case(name, desc, synth.projection_matrices(orbit, H, W, p), orbit.vdl, orbit, B)


def behind_source_case():
    # source circle of radius 40 mm; volume 100 x 100 x 60 mm: its corners lie
    # behind the source of the nearby views.  Nearest voxel centre to any
    # source is 1.4 mm away, and voxels within 2 mm of depth 0 project far off
    # the 64-pixel detector, so the FP32 / FP64 depth tests cannot disagree on
    # a voxel that contributes.
    o = synth.circle_orbit(24, sid=40.0, sdd=64.0)
    return _case(o, 48, 64, 1.0, 48, 64, (24, 40, 40), (2.5, 2.5, 2.5), B=2, name="behind")


def wide_footprint_case():
    # 2 mm voxels, 0.25 mm pixels: a 16-voxel box spans ~200 pixels, more than
    # the 64 x 48 staged tile
    o = synth.sinusoid_orbit(20)
    return _case(o, 96, 128, 0.25, 40, 128, (32, 24, 24), (2.0, 2.0, 2.0), name="wide")


# FP32 floor of the detector position with white-noise data (neighbouring
# pixels uncorrelated, so a position error of e pixels is a relative value
# error of about e): voxels 1.4 mm from the source are magnified ~45x, and
# 0.25 mm pixels put 4800 pixels per unit of lateral slope, so FP32 rounding
# of the coordinates moves projections by 1e-5 to 1e-4 pixel
@pytest.mark.parametrize("make,tol", [(behind_source_case, 5e-5), (wide_footprint_case, 5e-5)])
def test_backprojection_global_paths_match_oracle(make, tol):
    case = make()
    d = case.desc
    gg = api.Geometry(d, case.P, case.vdl)
    og = orc.Geometry(d, case.P, case.vdl)
    rng = np.random.default_rng(11)
    gF = rng.normal(size=(case.B, d["n_views"], d["det_rows"], d["det_cols"])).astype(np.float32)
    ref = orc.backproject(og, gF)
    assert np.abs(ref).max() > 0
    for kahan in (False, True):
        vol = _host(api.dc_backproject(gg, _dev(gF), kahan=kahan))
        assert rel_l2(vol, ref) < tol
    # the transpose through the same paths
    gv = rng.normal(size=(case.B, d["vol_z"], d["vol_y"], d["vol_x"])).astype(np.float32)
    adj = _host(api.dc_backproject_adjoint(gg, _dev(gv)))
    ref_adj = orc.backproject_adjoint(og, gv)
    assert rel_l2(adj, ref_adj) < tol
    api.dc_sync_status(gg)


def test_behind_source_voxels_get_nothing_from_those_views():
    case = behind_source_case()
    d = case.desc
    gg = api.Geometry(d, case.P, case.vdl)
    og = orc.Geometry(d, case.P, case.vdl)
    # one view only: every voxel with depth <= 0 in it must stay exactly 0
    gF = np.zeros((1, d["n_views"], d["det_rows"], d["det_cols"]), np.float32)
    gF[0, 0] = 1.0
    vol = _host(api.dc_backproject(gg, _dev(gF)))[0]
    ref = orc.backproject(og, gF)[0]
    a = og.source(0)
    lz = og.frame(0)[2]
    xs, ys, zs = synth.voxel_centers((d["vol_z"], d["vol_y"], d["vol_x"]), d["voxel"])
    Z, Y, Xg = np.meshgrid(zs, ys, xs, indexing="ij")
    depth = (a[0] - Xg) * lz[0] + (a[1] - Y) * lz[1] + (a[2] - Z) * lz[2]
    behind = depth <= 0
    assert behind.any() and (~behind).any()
    assert np.all(vol[behind] == 0.0) and np.all(ref[behind] == 0.0)
    assert rel_l2(vol, ref) < 5e-5


def test_full_reconstruction_behind_source_matches_oracle():
    case = behind_source_case()
    d = case.desc
    gg = api.Geometry(d, case.P, case.vdl)
    og = orc.Geometry(d, case.P, case.vdl)
    g = phantom_projections(case, n=4).astype(np.float32)
    vol = _host(api.reconstruct(gg, _dev(g)))
    ref = orc.reconstruct(og, g)
    assert rel_l2(vol, ref) < 1e-4


@pytest.mark.parametrize("bad", [float("nan"), float("inf")])
def test_nonfinite_weight_is_reported_and_contained(bad):
    o = synth.sinusoid_orbit(12)
    case = _case(o, 32, 40, 2.0, 24, 40, (16, 24, 24), (1.25, 1.25, 1.25))
    d = case.desc
    gg = api.Geometry(d, case.P, case.vdl)
    g = _dev(phantom_projections(case, n=3))
    W = random_weights(case).astype(np.float32)
    clean, _ = api.dc_filter(gg, g, _dev(W))
    clean = _host(clean)
    api.dc_sync_status(gg)
    Wb = W.copy()
    Wb[5, 7, 11] = bad
    gF, _ = api.dc_filter(gg, g, _dev(Wb))
    with pytest.raises(L.DCError) as err:
        api.dc_sync_status(gg)
    assert err.value.code == L.DC_ERR_NONFINITE
    out = _host(gF)
    # only view 5 depends on that weight
    others = [v for v in range(d["n_views"]) if v != 5]
    assert np.array_equal(out[:, others], clean[:, others])
    assert not np.isfinite(out[0, 5]).all()
    # the reverse mode reads W too
    ggF = torch.ones_like(g)
    api.dc_filter_adjoint(gg, ggF, g, _dev(Wb))
    with pytest.raises(L.DCError) as err:
        api.dc_sync_status(gg)
    assert err.value.code == L.DC_ERR_NONFINITE
    # flags clear once reported; a clean call reports nothing
    again, _ = api.dc_filter(gg, g, _dev(W))
    api.dc_sync_status(gg)
    assert np.array_equal(_host(again), clean)
