"""Long detector rows: the line-sum kernel stages shorter bands (16 or 8
detector rows instead of 32) when a 32-row band of such rows would not fit in
shared memory.  Line sums and the whole filter against the FP64 oracle."""
import numpy as np
import pytest
import torch

from oracle import oracle as orc
from paper_2410_14900_gb300 import api, synth

from cases import rel_l2

pytestmark = pytest.mark.gpu


def _wide_case(H, W, n_views=5, n_mu=24, n_s=96):
    o = synth.sinusoid_orbit(n_views)
    p = 0.8
    desc = dict(n_views=n_views, det_rows=H, det_cols=W, n_mu=n_mu, n_s=n_s, pitch=p,
                ds=1.25 * max(H, W) * p / n_s, vol_x=8, vol_y=8, vol_z=8, voxel=(1.0, 1.0, 1.0),
                closed_orbit=1)
    P = synth.projection_matrices(o, H, W, p)
    return desc, P, o.vdl


# 1536 columns take 8-row bands, 900 columns 16-row bands
@pytest.mark.parametrize("H,W", [(24, 1536), (40, 900), (900, 40)])
def test_long_rows_match_oracle(H, W):
    desc, P, vdl = _wide_case(H, W)
    gg = api.Geometry(desc, P, vdl)
    og = orc.Geometry(desc, P, vdl)
    rng = np.random.default_rng(H + W)
    img = rng.normal(size=(1, desc["n_views"], H, W)).astype(np.float32)
    R = api.dc_radon2d(gg, torch.as_tensor(img, device="cuda"))
    torch.cuda.synchronize()
    R = R.double().cpu().numpy()
    for i in range(desc["n_views"]):
        cu, cv = og.principal_point(i)
        ref = orc.radon(img[0, i], desc["pitch"], desc["n_mu"], desc["n_s"], desc["ds"], cu, cv)
        assert rel_l2(R[0, i], ref) < 2e-6
    gF, _ = api.dc_filter(gg, torch.as_tensor(img, device="cuda"))
    torch.cuda.synchronize()
    err = rel_l2(gF.double().cpu().numpy(), orc.filter(og, img.astype(np.float64), None))
    assert err < 1e-4, err
    api.dc_sync_status(gg)
