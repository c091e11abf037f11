"""The Eq. 9 weight generator on the GPU against the FP64 oracle, and a
reconstruction that uses it."""
import numpy as np
import pytest
import torch

from oracle import oracle as orc
from paper_2410_14900_gb300 import api, synth

from cases import arc_open, circle64, phantom_projections, ragged, random_nn, rel_l2

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("name", ["circle64", "ragged", "arc_open", "random_nn"])
@pytest.mark.parametrize("m,taper", [(2, 3), (1, 0), (0, 0)])
def test_crofton_weights_match_oracle(name, m, taper):
    case = {"circle64": circle64, "ragged": ragged, "arc_open": arc_open,
            "random_nn": random_nn}[name]()
    segs = {"arc_open": [(0, True), (20, False)], "random_nn": [(0, False)]}.get(name)
    gg = api.Geometry(case.desc, case.P, case.vdl)
    og = orc.Geometry(case.desc, case.P, case.vdl)
    W = api.dc_crofton_weights(gg, segs, m=m, taper=taper).double().cpu().numpy()
    ref = orc.crofton_weights(og, segs, m=m, taper=taper)
    K = np.stack([orc.redundancy_K(og, i) for i in range(case.desc["n_views"])])
    # compare the effective weight W*K: where K ~ 0 (plane tangent to the orbit
    # at the source) M is a ratio of vanishing terms and carries no weight
    err = rel_l2(W * np.abs(K), ref * np.abs(K))
    assert err < (1e-4 if m > 0 else 2e-3), err


def test_reconstruction_with_crofton_weights_matches_oracle():
    case = arc_open()
    segs = [(0, True), (20, False)]
    gg = api.Geometry(case.desc, case.P, case.vdl)
    og = orc.Geometry(case.desc, case.P, case.vdl)
    g = phantom_projections(case).astype(np.float32)
    W = api.dc_crofton_weights(gg, segs)
    vol = api.reconstruct(gg, torch.as_tensor(g, device="cuda"), W)
    ref = orc.reconstruct(og, g, orc.crofton_weights(og, segs))
    assert rel_l2(vol.double().cpu().numpy(), ref) < 1e-3
