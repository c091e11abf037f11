"""Randomised shapes against the FP64 oracle: detector sizes that are not
multiples of 4 (the untiled backprojection fallback), tiny and odd angle and
s-bin counts, s spacings from just above pitch/3 (multi-tap 2-D
backprojection) to twice the pitch, small odd volumes, several orbits and
batch sizes.  Every entry point of the reconstruction and its reverse mode
(odd seeds backproject with Kahan summation)."""
import numpy as np
import pytest
import torch

from oracle import oracle as orc
from paper_2410_14900_gb300 import api, synth

from cases import rel_l2

pytestmark = pytest.mark.gpu


def _random_case(seed):
    rng = np.random.default_rng(1000 + seed)
    V = int(rng.integers(1, 7))
    kind = ["circle", "sinusoid", "random_nn"][seed % 3]
    o = {"circle": lambda: synth.circle_orbit(max(V, 2)),
         "sinusoid": lambda: synth.sinusoid_orbit(max(V, 2)),
         "random_nn": lambda: synth.random_nn_orbit(max(V, 2), seed=seed)}[kind]()
    V = o.n_views
    H, W = int(rng.integers(5, 71)), int(rng.integers(5, 91))
    p = float(rng.uniform(0.8, 2.5))
    n_s = int(rng.integers(3, 81))
    ds = float(rng.uniform(0.35, 2.0)) * p
    n_mu = int(rng.integers(3, 51))
    r_det = 0.5 * np.hypot(H, W) * p * synth.SID_MM / o.sdd
    vox = float(rng.uniform(0.6, 1.6)) * r_det / 12.0
    desc = dict(n_views=V, det_rows=H, det_cols=W, n_mu=n_mu, n_s=n_s, pitch=p, ds=ds,
                vol_x=int(rng.integers(3, 21)), vol_y=int(rng.integers(3, 21)),
                vol_z=int(rng.integers(3, 21)), voxel=(vox, vox * 0.9, vox * 1.1),
                vol_center=tuple(float(c) for c in rng.uniform(-2.0, 2.0, 3)),
                closed_orbit=int(o.closed))
    P = synth.projection_matrices(o, H, W, p)
    B = int(rng.integers(1, 4))
    return desc, P, o.vdl, B, rng


@pytest.mark.parametrize("seed", range(30))
def test_random_shapes_match_oracle(seed):
    desc, P, vdl, B, rng = _random_case(seed)
    gg = api.Geometry(desc, P, vdl)
    og = orc.Geometry(desc, P, vdl)
    V, H, W = desc["n_views"], desc["det_rows"], desc["det_cols"]
    g = rng.normal(size=(B, V, H, W)).astype(np.float32)
    Wred = rng.uniform(0.2, 0.8, size=(V, desc["n_mu"], desc["n_s"])).astype(np.float32)
    dev = lambda a: torch.as_tensor(np.ascontiguousarray(a), device="cuda")
    host = lambda t: (torch.cuda.synchronize(), t.double().cpu().numpy())[1]

    R = host(api.dc_radon2d(gg, dev(g)))
    for i in range(V):
        cu, cv = og.principal_point(i)
        ref = orc.radon(g[0, i], desc["pitch"], desc["n_mu"], desc["n_s"], desc["ds"], cu, cv)
        assert rel_l2(R[0, i], ref) < 2e-6, ("radon", i)
    gF, _ = api.dc_filter(gg, dev(g), dev(Wred))
    gF_ref = orc.filter(og, g, Wred)
    assert rel_l2(host(gF), gF_ref) < 1e-4, "filter"
    gF32 = gF_ref.astype(np.float32)
    vol = host(api.dc_backproject(gg, dev(gF32), kahan=bool(seed % 2)))
    assert rel_l2(vol, orc.backproject(og, gF32)) < 1e-4, "backproject"
    Gv = rng.normal(size=vol.shape).astype(np.float32)
    gadj = host(api.dc_backproject_adjoint(gg, dev(Gv)))
    assert rel_l2(gadj, orc.backproject_adjoint(og, Gv)) < 1e-4, "backproject adjoint"
    G = rng.normal(size=g.shape).astype(np.float32)
    gg_g, gg_W = api.dc_filter_adjoint(gg, dev(G), dev(g), dev(Wred))
    rg, rW = orc.filter_adjoint(og, g, G, Wred)
    assert rel_l2(host(gg_g), rg) < 1e-4, "filter adjoint (g)"
    assert rel_l2(host(gg_W), rW) < 1e-4, "filter adjoint (W)"
    api.dc_sync_status(gg)
