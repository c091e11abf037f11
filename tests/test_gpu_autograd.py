"""Gradients of the differentiable reconstruction (Eq. 12 with the learnable
redundancy weight of Eq. 10): analytic (the adjoint kernels) against the FP64
oracle's reverse mode, against central finite differences, and torch's
autograd plumbing."""
import numpy as np
import pytest
import torch

from oracle import oracle as orc
from paper_2410_14900_gb300 import api, synth
from paper_2410_14900_gb300.autograd import DefriseClackNet, reconstruct

from cases import phantom_projections, ragged, rel_l2

pytestmark = pytest.mark.gpu


def _small_train_case():
    """Sinusoidal orbit, batch of 2, small sizes (the training configuration's shape)."""
    case = ragged(B=2)
    return case


def test_mse_gradient_matches_oracle():
    case = _small_train_case()
    geom = api.Geometry(case.desc, case.P, case.vdl)
    og = orc.Geometry(case.desc, case.P, case.vdl)
    g = phantom_projections(case).astype(np.float32)
    d = case.desc
    rng = np.random.default_rng(8)
    W0 = rng.uniform(0.3, 0.7, size=(d["n_views"], d["n_mu"], d["n_s"])).astype(np.float32)
    tgt = rng.normal(size=(case.B, d["vol_z"], d["vol_y"], d["vol_x"])).astype(np.float32) * 0.01

    gt = torch.as_tensor(g, device="cuda").requires_grad_(True)
    Wt = torch.as_tensor(W0, device="cuda").requires_grad_(True)
    vol = reconstruct(gt, Wt, geom)
    loss = 0.5 * ((vol - torch.as_tensor(tgt, device="cuda")) ** 2).sum()
    loss.backward()

    # oracle: the same loss, reverse mode by hand in FP64
    r = orc.reconstruct(og, g, W0) - tgt
    ggF = orc.backproject_adjoint(og, r)
    rg, rW = orc.filter_adjoint(og, g, ggF, W0)
    assert rel_l2(Wt.grad.double().cpu().numpy(), rW) < 1e-4
    assert rel_l2(gt.grad.double().cpu().numpy(), rg) < 1e-4


def test_relu_gradient_masks_clamped_voxels():
    case = _small_train_case()
    geom = api.Geometry(case.desc, case.P, case.vdl)
    og = orc.Geometry(case.desc, case.P, case.vdl)
    g = phantom_projections(case).astype(np.float32)
    gt = torch.as_tensor(g, device="cuda")
    net = DefriseClackNet(geom, relu=True, device="cuda")
    vol = net(gt)
    ref = orc.reconstruct(og, g, None, relu=True)
    assert rel_l2(vol.detach().double().cpu().numpy(), ref) < 1e-4
    assert (vol >= 0).all()
    vol.sum().backward()
    # d(sum relu(f))/dW = filter_adjoint of backproject_adjoint(1[f > 0])
    mask = (orc.reconstruct(og, g, None) > 0).astype(np.float64)
    Wh = np.full((case.desc["n_views"],) + (case.desc["n_mu"], case.desc["n_s"]), 0.5)
    _, rW = orc.filter_adjoint(og, g, orc.backproject_adjoint(og, mask), Wh)
    assert rel_l2(net.W.grad.double().cpu().numpy(), rW) < 1e-4


def test_central_differences_on_64_random_weights():
    """FP32 GPU finite differences (h = 1e-3) on 64 random weights.

    The MSE loss is quadratic in W, so central differences are exact up to
    rounding; the loss is accumulated in FP64 to keep that rounding small.
    """
    case = _small_train_case()
    geom = api.Geometry(case.desc, case.P, case.vdl)
    g = torch.as_tensor(phantom_projections(case).astype(np.float32), device="cuda")
    d = case.desc
    shape = (d["n_views"], d["n_mu"], d["n_s"])
    W = torch.full(shape, 0.5, device="cuda", requires_grad=True)
    with torch.no_grad():
        tgt = reconstruct(g, W.detach() * 1.1, geom)

    def loss_of(Wv):
        v = reconstruct(g, Wv, geom).double()
        return 0.5 * ((v - tgt.double()) ** 2).sum()

    L = loss_of(W)
    L.backward()
    grad = W.grad.detach().double().cpu().numpy()
    rng = np.random.default_rng(12)
    h = 1e-3
    flat = rng.choice(np.prod(shape), size=64, replace=False)
    errs = []
    big = np.abs(grad).max()
    for f in flat:
        idx = np.unravel_index(f, shape)
        with torch.no_grad():
            Wp = W.detach().clone()
            Wm = W.detach().clone()
            Wp[idx] += h
            Wm[idx] -= h
            fd = float((loss_of(Wp) - loss_of(Wm)) / (2 * h))
        errs.append(abs(fd - grad[idx]) / big)
    errs = np.array(errs)
    print("FD vs analytic, |err| / max|grad|: median %.2e, max %.2e" % (np.median(errs), errs.max()))
    assert errs.max() < 1e-3


def test_gradcheck_on_a_tiny_problem():
    """torch.autograd.gradcheck in FP32 against the FP32 kernels (linear maps)."""
    o = synth.sinusoid_orbit(4)
    H, W, p = 12, 16, 2.0
    desc = dict(n_views=4, det_rows=H, det_cols=W, n_mu=8, n_s=16, pitch=p, ds=p,
                vol_x=6, vol_y=5, vol_z=4, voxel=(2.0, 2.0, 2.0), closed_orbit=1)
    geom = api.Geometry(desc, synth.projection_matrices(o, H, W, p), o.vdl)
    g = torch.randn((1, 4, H, W), device="cuda", requires_grad=True)
    Wt = torch.rand((4, 8, 16), device="cuda", requires_grad=True)
    # both maps are linear in each argument: directional derivative checks
    v = reconstruct(g, Wt, geom)
    u = torch.randn_like(v)
    (v * u).sum().backward()
    dg = torch.randn_like(g)
    with torch.no_grad():
        lin = (reconstruct(g + dg, Wt, geom) - v) * u
    assert abs(float(lin.sum()) - float((g.grad * dg).sum())) <= 1e-3 * float(lin.abs().sum())
