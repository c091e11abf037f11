"""Parity at the benchmark's full sizes, in the launch configuration the
benchmark times: every GPU call runs on the whole problem, and the oracle
checks sampled outputs it can compute one by one (selected views of the
filter, selected voxels of the backprojection)."""
import numpy as np
import pytest
import torch

from oracle import oracle as orc
from paper_2410_14900_gb300 import api, synth

from cases import rel_l2

pytestmark = pytest.mark.gpu


def _geoms(w):
    return (api.Geometry(w.desc_dict(), w.matrices(), w.orbit.vdl),
            orc.Geometry(w.desc_dict(), w.matrices(), w.orbit.vdl))


def _projections(w, device="cuda"):
    blobs = w.phantoms()[0]
    g = synth.project_phantom(blobs, w.orbit, w.det_rows, w.det_cols, w.pitch, device=device,
                              dtype=torch.float32)
    if w.photons:
        g = synth.add_poisson_noise(g, w.photons, 0.02, seed=w.seed)
    return g[None].contiguous()


@pytest.mark.parametrize("name", ["circle_arc512", "paper400"])
@pytest.mark.parametrize("storage", ["f32", "f32x2", "bf16"])
def test_backprojection_full_size_sampled_voxels(name, storage):
    w = synth.workload(name)
    gg, og = _geoms(w)
    V, H, W = w.n_views, w.det_rows, w.det_cols
    gen = torch.Generator(device="cuda")
    gen.manual_seed(11)
    gF = torch.randn((1, V, H, W), device="cuda", generator=gen)
    if storage == "bf16":
        gF = gF.to(torch.bfloat16)
    stored = gF
    if storage == "f32x2":   # (value, right difference) pairs of the same values
        right = torch.cat([gF[..., 1:], torch.zeros_like(gF[..., :1])], dim=-1)
        stored = torch.stack([gF, right - gF], dim=-1).contiguous()
    vol = api.dc_backproject(gg, stored, kahan=(storage == "bf16"))
    nvox = w.vol_shape[0] * w.vol_shape[1] * w.vol_shape[2]
    flat = np.random.default_rng(3).choice(nvox, size=4096, replace=False)
    # the oracle sees exactly the stored values.  White-noise data turn any
    # detector-position error into relative error one to one; FP32 positions
    # up to 512 pixels carry ~2e-5 pixel rounding, so this worst case lands
    # near 2e-5 (smooth filtered projections stay far below).
    ref = orc.backproject_points(og, gF[0].double().cpu().numpy(), flat)
    got = vol.reshape(-1)[torch.as_tensor(flat, device="cuda")].double().cpu().numpy()
    assert rel_l2(got, ref) < 1e-4


@pytest.mark.parametrize("name,views", [("circle_arc512", [0, 97, 359, 360, 430, 495]),
                                        ("paper400", [0, 133, 399])])
def test_filter_full_size_sampled_views(name, views):
    w = synth.workload(name)
    gg, og = _geoms(w)
    g = _projections(w)
    gF, _ = api.dc_filter(gg, g)
    torch.cuda.synchronize()
    g_np = g[0, views].double().cpu().numpy()
    ref = orc.filter(og, g_np[None], None, views=views)[0]
    for t, i in enumerate(views):
        err = rel_l2(gF[0, i].double().cpu().numpy(), ref[t])
        assert err < 1e-4, (i, err)


def test_pair_filter_full_size_equals_fp32_filter():
    """The benchmark's storage form at its size: the filter's pairs are the
    FP32 filter's values (checked against the oracle above) and their
    right differences, bit for bit."""
    w = synth.workload("circle_arc512")
    gg, _ = _geoms(w)
    g = _projections(w)
    gF, _ = api.dc_filter(gg, g, None, "f32")
    gP, _ = api.dc_filter(gg, g, None, "f32x2")
    torch.cuda.synchronize()
    assert torch.equal(gP[..., 0], gF)
    right = torch.cat([gF[..., 1:], torch.zeros_like(gF[..., :1])], dim=-1)
    assert torch.equal(gP[..., 1], right - gF)


def test_sinusoid_full_chain_sampled_voxels():
    """256^3 sinusoidal orbit with Poisson noise: whole reconstruction on the
    GPU; the oracle filters every view and backprojects sampled voxels."""
    w = synth.workload("sinusoid256")
    gg, og = _geoms(w)
    g = _projections(w)
    vol = api.reconstruct(gg, g)
    g_np = g[0].double().cpu().numpy()
    gF = orc.filter(og, g_np[None])[0]
    nvox = 256 ** 3
    flat = np.random.default_rng(4).choice(nvox, size=4096, replace=False)
    ref = orc.backproject_points(og, gF, flat)
    got = vol.reshape(-1)[torch.as_tensor(flat, device="cuda")].double().cpu().numpy()
    assert rel_l2(got, ref) < 1e-4
