"""CUDA path versus the FP64 oracle, element by element, through the C ABI.

Tolerance: 1e-4 relative L2 for FP32 results (the target the method is
built to); tighter where no derivative amplifies rounding (line sums,
backprojection).  Inputs are identical FP32-rounded arrays on both sides.
"""
import numpy as np
import pytest
import torch

from oracle import oracle as orc
from paper_2410_14900_gb300 import api
from paper_2410_14900_gb300 import _lib as L

from cases import (arc_open, circle64, phantom_projections, ragged, random_nn, random_weights,
                   rel_l2)

pytestmark = pytest.mark.gpu

CASES = {"circle64": circle64, "ragged": ragged, "arc_open": arc_open, "random_nn": random_nn}


def _setup(case):
    return api.Geometry(case.desc, case.P, case.vdl), orc.Geometry(case.desc, case.P, case.vdl)


def _dev(a):
    return torch.as_tensor(np.ascontiguousarray(a, dtype=np.float32), device="cuda")


def _host(t):
    torch.cuda.synchronize()
    return t.double().cpu().numpy()


@pytest.fixture(scope="module", params=list(CASES))
def prob(request):
    case = CASES[request.param]()
    gg, og = _setup(case)
    g32 = phantom_projections(case).astype(np.float32)
    W32 = random_weights(case).astype(np.float32)
    return dict(case=case, gpu=gg, orc=og, g=g32, W=W32)


def test_geometry_matches_oracle(prob):
    v = api.dc_get_view_geometry(prob["gpu"])
    og = prob["orc"]
    for i in range(prob["case"].desc["n_views"]):
        np.testing.assert_allclose(v[i, 0:3], og.source(i), rtol=0, atol=1e-9)
        lx, ly, lz = og.frame(i)
        np.testing.assert_allclose(v[i, 3:6], lx, atol=1e-13)
        np.testing.assert_allclose(v[i, 6:9], ly, atol=1e-13)
        np.testing.assert_allclose(v[i, 9:12], lz, atol=1e-13)
        assert abs(v[i, 12] - og.D(i)) < 1e-9
        np.testing.assert_allclose(v[i, 13:15], og.principal_point(i), atol=1e-9)
        np.testing.assert_allclose(v[i, 15:18], og.tangent(i), rtol=1e-12, atol=1e-9)


def test_radon2d_matches_oracle(prob):
    case, og = prob["case"], prob["orc"]
    d = case.desc
    rng = np.random.default_rng(1)
    img = rng.normal(size=(case.B, d["n_views"], d["det_rows"], d["det_cols"])).astype(np.float32)
    R = _host(api.dc_radon2d(prob["gpu"], _dev(img)))
    for b in range(case.B):
        for i in range(0, d["n_views"], max(1, d["n_views"] // 5)):
            cu, cv = og.principal_point(i)
            ref = orc.radon(img[b, i], d["pitch"], d["n_mu"], d["n_s"], d["ds"], cu, cv)
            assert rel_l2(R[b, i], ref) < 2e-6


def test_radon2d_adjoint_matches_oracle(prob):
    case, og = prob["case"], prob["orc"]
    d = case.desc
    rng = np.random.default_rng(2)
    R = rng.normal(size=(case.B, d["n_views"], d["n_mu"], d["n_s"])).astype(np.float32)
    img = _host(api.dc_radon2d_adjoint(prob["gpu"], _dev(R)))
    for b in range(case.B):
        for i in range(0, d["n_views"], max(1, d["n_views"] // 5)):
            cu, cv = og.principal_point(i)
            ref = orc.radon_T(R[b, i], d["det_rows"], d["det_cols"], d["pitch"], d["ds"], cu, cv)
            assert rel_l2(img[b, i], ref) < 1e-5


def test_grangeat_matches_oracle(prob):
    case, og = prob["case"], prob["orc"]
    S = _host(api.dc_grangeat(prob["gpu"], _dev(prob["g"])))
    errs = []
    for b in range(case.B):
        for i in range(case.desc["n_views"]):
            errs.append(rel_l2(S[b, i], orc.grangeat(og, i, prob["g"][b, i])))
    assert max(errs) < 1e-4, max(errs)


def test_filter_matches_oracle(prob):
    case = prob["case"]
    W = prob["W"] if case.name != "circle64" else None
    gF, _ = api.dc_filter(prob["gpu"], _dev(prob["g"]), None if W is None else _dev(W))
    ref = orc.filter(prob["orc"], prob["g"], W)
    err = rel_l2(_host(gF), ref)
    assert err < 1e-4, err


def test_backproject_matches_oracle(prob):
    case = prob["case"]
    d = case.desc
    rng = np.random.default_rng(3)
    gF = rng.normal(size=(case.B, d["n_views"], d["det_rows"], d["det_cols"])).astype(np.float32)
    ref = orc.backproject(prob["orc"], gF)
    for kahan in (False, True):
        vol = _host(api.dc_backproject(prob["gpu"], _dev(gF), kahan=kahan))
        assert rel_l2(vol, ref) < 1e-5
    relu = _host(api.dc_backproject(prob["gpu"], _dev(gF), relu=True))
    assert rel_l2(relu, np.maximum(ref, 0)) < 1e-5
    base = _dev(ref)
    acc = _host(api.dc_backproject(prob["gpu"], _dev(gF), out=base, accum=True))
    assert rel_l2(acc, 2 * ref) < 1e-5


def test_reconstruction_matches_oracle(prob):
    case = prob["case"]
    W = prob["W"] if case.name != "circle64" else None
    vol = api.reconstruct(prob["gpu"], _dev(prob["g"]), None if W is None else _dev(W))
    ref = orc.reconstruct(prob["orc"], prob["g"], W)
    err = rel_l2(_host(vol), ref)
    assert err < 1e-4, err


def test_backproject_adjoint_matches_oracle(prob):
    case = prob["case"]
    d = case.desc
    rng = np.random.default_rng(4)
    gv = rng.normal(size=(case.B, d["vol_z"], d["vol_y"], d["vol_x"])).astype(np.float32)
    out = _host(api.dc_backproject_adjoint(prob["gpu"], _dev(gv)))
    ref = orc.backproject_adjoint(prob["orc"], gv)
    assert rel_l2(out, ref) < 1e-5
    # ReLU mask: zero gradient where the forward output was clamped
    mask = rng.normal(size=gv.shape).astype(np.float32)
    out2 = _host(api.dc_backproject_adjoint(prob["gpu"], _dev(gv), relu_vol=_dev(mask)))
    ref2 = orc.backproject_adjoint(prob["orc"], gv * (mask > 0))
    assert rel_l2(out2, ref2) < 1e-5


def test_filter_adjoint_matches_oracle(prob):
    case = prob["case"]
    d = case.desc
    rng = np.random.default_rng(6)
    G = rng.normal(size=(case.B, d["n_views"], d["det_rows"], d["det_cols"])).astype(np.float32)
    W = prob["W"]
    gg, gW = api.dc_filter_adjoint(prob["gpu"], _dev(G), _dev(prob["g"]), _dev(W))
    rg, rW = orc.filter_adjoint(prob["orc"], prob["g"], G, W)
    assert rel_l2(_host(gg), rg) < 1e-4
    assert rel_l2(_host(gW), rW) < 1e-4
    # view chunking does not change the result
    gg2, gW2 = api.dc_filter_adjoint(prob["gpu"], _dev(G), _dev(prob["g"]), _dev(W),
                                     view_chunk=3)
    assert rel_l2(_host(gg2), _host(gg)) < 1e-6
    assert rel_l2(_host(gW2), _host(gW)) < 1e-6


def test_low_precision_storage_error_is_bounded(prob):
    """BF16 / FP16 storage of g^F with FP32 interpolation (error vs FP64 stated)."""
    case = prob["case"]
    ref = orc.reconstruct(prob["orc"], prob["g"], None)
    g = _dev(prob["g"])
    errs = {}
    for dt in ("bf16", "f16"):
        gF, sc = api.dc_filter(prob["gpu"], g, None, dtype=dt)
        for kahan in (False, True):
            vol = api.dc_backproject(prob["gpu"], gF, sc, kahan=kahan)
            errs[(dt, kahan)] = rel_l2(_host(vol), ref)
    print(case.name, errs)
    assert errs[("bf16", True)] < 1e-2
    assert errs[("f16", True)] < 2e-3
    api.dc_sync_status(prob["gpu"])


def test_argument_errors_on_gpu():
    case = circle64()
    gg = api.Geometry(case.desc, case.P, case.vdl)
    Lh = L.load()
    x = torch.zeros(1, device="cuda")
    p = x.data_ptr()
    assert Lh.dc_filter(gg.handle, 0, p, None, p, 0, None, None) == L.DC_ERR_ARG
    assert Lh.dc_filter(gg.handle, 1, p, None, p, 7, None, None) == L.DC_ERR_ARG
    assert Lh.dc_filter(gg.handle, 1, p, None, p, L.DC_F16, None, None) == L.DC_ERR_ARG
    assert Lh.dc_backproject(gg.handle, 1, p, 0, None, p, 64, None) == L.DC_ERR_ARG
    bad = dict(case.desc, ds=case.desc["pitch"] * 0.3)
    g2 = api.Geometry(bad, case.P, case.vdl)
    assert Lh.dc_filter(g2.handle, 1, p, None, p, 0, None, None) == L.DC_ERR_UNSUPPORTED
    with pytest.raises(L.DCError):
        api.Geometry(case.desc, case.P * np.array([1, 1.5, 1, 1])[None, None, :], case.vdl)
    api.dc_sync_status(gg)


def test_allocation_failure_is_reported():
    case = circle64()
    Lh = L.load()
    for n in range(0, 64):
        Lh.dc_debug_fail_alloc_after(n)
        try:
            g = api.Geometry(case.desc, case.P, case.vdl)
        except L.DCError as e:
            assert e.code == L.DC_ERR_OOM
            continue
        finally:
            Lh.dc_debug_fail_alloc_after(-1)
        g.close()
        break
    else:
        pytest.fail("setup never succeeded")


@pytest.mark.parametrize("frac", [0.5, 0.8])
def test_fine_s_grid_matches_oracle(frac):
    """ds below the pitch: a pixel meets up to six lines of an angle (the
    multi-tap 2-D backprojection); filter, its adjoint and A2d^T."""
    base = ragged(B=1)
    desc = dict(base.desc, ds=base.desc["pitch"] * frac, n_s=int(base.desc["n_s"] / frac) + 1)
    gg = api.Geometry(desc, base.P, base.vdl)
    og = orc.Geometry(desc, base.P, base.vdl)
    g = phantom_projections(base).astype(np.float32)
    rng = np.random.default_rng(31)
    W = rng.uniform(0.2, 0.8, size=(desc["n_views"], desc["n_mu"], desc["n_s"])).astype(np.float32)
    gF, _ = api.dc_filter(gg, _dev(g), _dev(W))
    assert rel_l2(_host(gF), orc.filter(og, g, W)) < 1e-4
    R = rng.normal(size=(1, desc["n_views"], desc["n_mu"], desc["n_s"])).astype(np.float32)
    img = _host(api.dc_radon2d_adjoint(gg, _dev(R)))
    for i in range(0, desc["n_views"], 7):
        cu, cv = og.principal_point(i)
        ref = orc.radon_T(R[0, i], desc["det_rows"], desc["det_cols"], desc["pitch"], desc["ds"],
                          cu, cv)
        assert rel_l2(img[0, i], ref) < 1e-5
    G = rng.normal(size=g.shape).astype(np.float32)
    gg_g, gg_W = api.dc_filter_adjoint(gg, _dev(G), _dev(g), _dev(W))
    rg, rW = orc.filter_adjoint(og, g, G, W)
    assert rel_l2(_host(gg_g), rg) < 1e-4
    assert rel_l2(_host(gg_W), rW) < 1e-4
    api.dc_sync_status(gg)


@pytest.mark.parametrize("kind,fn", [("f", "deriv_f"), ("fT", "deriv_f_T"), ("b", "deriv_b"),
                                     ("bT", "deriv_b_T")])
def test_deriv_matches_oracle(prob, kind, fn):
    case, d = prob["case"], prob["case"].desc
    rng = np.random.default_rng(41)
    x = rng.normal(size=(case.B, d["n_views"], d["n_mu"], d["n_s"])).astype(np.float32)
    got = _host(api.dc_deriv(prob["gpu"], _dev(x), kind))
    for b in range(case.B):
        for i in range(d["n_views"]):
            ref = getattr(orc, fn)(x[b, i], d["ds"])
            assert rel_l2(got[b, i], ref) < 1e-6


def test_kept_grangeat_function_gives_the_same_filter_and_gradients(prob):
    """dc_filter_with_s keeps S (equal to dc_grangeat's) and leaves g^F
    unchanged; dc_filter_adjoint_from_s gives dc_filter_adjoint's gradients."""
    case, d = prob["case"], prob["case"].desc
    g, W = _dev(prob["g"]), _dev(prob["W"])
    S = torch.empty((case.B, d["n_views"], d["n_mu"], d["n_s"]), device="cuda")
    gF1, _ = api.dc_filter(prob["gpu"], g, W)
    gF2, _ = api.dc_filter(prob["gpu"], g, W, S_out=S)
    assert torch.equal(gF1, gF2)
    S_ref = api.dc_grangeat(prob["gpu"], g)
    assert torch.equal(S, S_ref)
    G = _dev(np.random.default_rng(51).normal(size=prob["g"].shape))
    gg1, gW1 = api.dc_filter_adjoint(prob["gpu"], G, g, W)
    gg2, gW2 = api.dc_filter_adjoint(prob["gpu"], G, None, W, S=S)
    torch.cuda.synchronize()
    assert torch.equal(gg1, gg2) and torch.equal(gW1, gW2)


def test_kept_grangeat_function_across_chunks():
    """The kept S is indexed by (item, view) in every chunk: with chunks of
    4 images and a batch of 2 the forward runs 2 items x 2 views per chunk
    (23 views: a ragged last chunk), the reverse mode 2 x 1 (view_chunk 1)
    or 2 x 2; the reverse mode from S still equals the recomputing one and
    the oracle's."""
    case = ragged(B=2)
    d = case.desc
    gg = api.Geometry(d, case.P, case.vdl)
    og = orc.Geometry(d, case.P, case.vdl)
    api.dc_geometry_set_tuning(gg, 4, 0)
    g32 = phantom_projections(case).astype(np.float32)
    W32 = random_weights(case).astype(np.float32)
    g, W = _dev(g32), _dev(W32)
    S = torch.empty((case.B, d["n_views"], d["n_mu"], d["n_s"]), device="cuda")
    gF, _ = api.dc_filter(gg, g, W, S_out=S)
    assert torch.equal(S, api.dc_grangeat(gg, g))
    Gn = np.random.default_rng(52).normal(size=g32.shape).astype(np.float32)
    G = _dev(Gn)
    ref_g, ref_W = orc.filter_adjoint(og, g32, Gn, W32)
    for chunk in (1, 0):
        gg1, gW1 = api.dc_filter_adjoint(gg, G, g, W, view_chunk=chunk)
        gg2, gW2 = api.dc_filter_adjoint(gg, G, None, W, view_chunk=chunk, S=S)
        torch.cuda.synchronize()
        assert torch.equal(gg1, gg2) and torch.equal(gW1, gW2)
        assert rel_l2(_host(gg2), ref_g) < 1e-4
        assert rel_l2(_host(gW2), ref_W) < 1e-4
    api.dc_sync_status(gg)
