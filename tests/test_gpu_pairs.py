"""The FP32 pair storage form of g^F (DC_F32X2: per pixel the value and the
difference to its right neighbour, zero beyond the last column) through the
C ABI: the filter's pairs equal the FP32 filter's values and their
differences bit for bit, and the backprojection from pairs matches the FP64
oracle (Eq. 5) on every test orbit, including odd detector widths (no TMA
tiles: the global-load kernel reads the pairs' values), boxes behind the
source and footprints wider than the staged tile.
"""
import numpy as np
import pytest
import torch

from oracle import oracle as orc
from paper_2410_14900_gb300 import api, synth

from cases import arc_open, circle64, phantom_projections, ragged, random_nn, rel_l2, Case

pytestmark = pytest.mark.gpu


def _dev(a):
    return torch.as_tensor(np.ascontiguousarray(a, dtype=np.float32), device="cuda")


def _host(t):
    torch.cuda.synchronize()
    return t.double().cpu().numpy()


def to_pairs(gF: torch.Tensor) -> torch.Tensor:
    """(g, g_right - g) with zero beyond the last column, in FP32."""
    right = torch.cat([gF[..., 1:], torch.zeros_like(gF[..., :1])], dim=-1)
    return torch.stack([gF, right - gF], dim=-1).contiguous()


def odd_width_case():
    o = synth.sinusoid_orbit(18)
    H, W, p = 36, 45, 1.5
    desc = dict(n_views=o.n_views, det_rows=H, det_cols=W, n_mu=36, n_s=44, pitch=p, ds=p,
                vol_x=28, vol_y=26, vol_z=20, voxel=(1.4, 1.4, 1.4),
                vol_center=(0.0, 0.0, 0.0), closed_orbit=1)
    return Case("odd_width", desc, synth.projection_matrices(o, H, W, p), o.vdl, o, 1)


CASES = {"circle64": circle64, "ragged": ragged, "arc_open": arc_open, "random_nn": random_nn,
         "odd_width": odd_width_case}


@pytest.fixture(scope="module", params=list(CASES))
def prob(request):
    case = CASES[request.param]()
    return dict(case=case, gpu=api.Geometry(case.desc, case.P, case.vdl),
                orc=orc.Geometry(case.desc, case.P, case.vdl),
                g=phantom_projections(case).astype(np.float32))


def test_filter_pairs_are_the_fp32_values_and_differences(prob):
    g = _dev(prob["g"])
    gF, _ = api.dc_filter(prob["gpu"], g, None, "f32")
    gP, sc = api.dc_filter(prob["gpu"], g, None, "f32x2")
    torch.cuda.synchronize()
    assert sc is None and gP.shape == gF.shape + (2,)
    assert torch.equal(gP[..., 0], gF)
    assert torch.equal(gP[..., 1], to_pairs(gF)[..., 1])
    api.dc_sync_status(prob["gpu"])


def test_backprojection_from_pairs_matches_oracle(prob):
    case = prob["case"]
    d = case.desc
    rng = np.random.default_rng(5)
    gF = rng.normal(size=(case.B, d["n_views"], d["det_rows"], d["det_cols"])).astype(np.float32)
    ref = orc.backproject(prob["orc"], gF)
    pairs = to_pairs(_dev(gF))
    plain = _host(api.dc_backproject(prob["gpu"], _dev(gF)))
    for kahan in (False, True):
        vol = _host(api.dc_backproject(prob["gpu"], pairs, kahan=kahan))
        assert rel_l2(vol, ref) < 1e-5
        # the same interpolation arithmetic as the FP32 form, except where one
        # form stages a view and the other reads it from global memory
        # (footprints that only fit the wider pair tiles; detectors whose FP32
        # rows are not a multiple of 16 bytes, like this ragged one): there
        # the reciprocals round differently, ~1e-6 of the position
        assert rel_l2(vol, plain) < 5e-6
    relu = _host(api.dc_backproject(prob["gpu"], pairs, relu=True))
    assert rel_l2(relu, np.maximum(ref, 0)) < 1e-5
    acc = _host(api.dc_backproject(prob["gpu"], pairs, out=_dev(ref), accum=True))
    assert rel_l2(acc, 2 * ref) < 1e-5
    api.dc_sync_status(prob["gpu"])


def test_reconstruction_through_pairs_matches_oracle(prob):
    vol = api.reconstruct(prob["gpu"], _dev(prob["g"]), None, dtype="f32x2")
    ref = orc.reconstruct(prob["orc"], prob["g"], None)
    assert rel_l2(_host(vol), ref) < 1e-4
    api.dc_sync_status(prob["gpu"])


@pytest.mark.parametrize("which", ["behind", "wide"])
def test_pairs_on_the_global_load_paths(which):
    from test_gpu_edge import behind_source_case, wide_footprint_case
    case = behind_source_case() if which == "behind" else wide_footprint_case()
    d = case.desc
    gg = api.Geometry(d, case.P, case.vdl)
    og = orc.Geometry(d, case.P, case.vdl)
    rng = np.random.default_rng(12)
    gF = rng.normal(size=(case.B, d["n_views"], d["det_rows"], d["det_cols"])).astype(np.float32)
    ref = orc.backproject(og, gF)
    vol = _host(api.dc_backproject(gg, to_pairs(_dev(gF))))
    assert rel_l2(vol, ref) < 5e-5
    api.dc_sync_status(gg)


def test_pair_storage_argument_checks():
    case = circle64()
    gg = api.Geometry(case.desc, case.P, case.vdl)
    g = _dev(phantom_projections(case))
    # an output of the FP32 shape is refused for the pair form
    with pytest.raises(ValueError):
        api.dc_filter(gg, g, None, "f32x2", out=torch.empty((1, gg.V, gg.H, gg.W), device="cuda"))
    # a misaligned pair buffer is refused by the library (16-byte stores)
    buf = torch.empty(2 * gg.V * gg.H * gg.W + 2, device="cuda")
    from paper_2410_14900_gb300 import _lib as L
    rc = L.load().dc_filter(gg.handle, 1, api._ptr(g), None,
                            api.ctypes.c_void_p(buf.data_ptr() + 8), L.DC_F32X2, None,
                            api._stream())
    assert rc == L.DC_ERR_ARG
