"""Training the redundancy weight of the Defrise-Clack network (Sec. 3.1).

The trainable layer is W (Eq. 10) followed by the Gaussian filter layer
(sigma 20, kernel 121); the optimiser is AdamW with the one-cycle learning
rate policy (the rate rises from a tenth of its peak to the peak and anneals
back over the run).  The loss is the mean squared error between the
normalised reconstruction and the normalised reference; the paper leaves the
normalisation unstated, and both volumes are divided here by the
reference's RMS, so the loss is the relative MSE and W's overall scale stays
learnable.  The SSIM term of Eq. 13 is not used.

Data are seeded synthetic phantoms (ellipsoids with exact line integrals and
their voxelised volumes); `compare` reports the relative error of learned
weights against the analytic ones (1/2 and Eq. 9) on held-out phantoms.

    python -m paper_2410_14900_gb300.train --workload sinusoid256_train --epochs 40
"""
from __future__ import annotations

import argparse
import json
import time
from typing import List, Optional, Sequence

import numpy as np
import torch

from . import api, synth
from .autograd import DefriseClackNet, reconstruct


def relative_mse(vol: torch.Tensor, ref: torch.Tensor) -> torch.Tensor:
    """mean((vol - ref)^2) / mean(ref^2): MSE after dividing both by ref's RMS."""
    return torch.mean((vol - ref) ** 2) / torch.mean(ref ** 2)


def make_data(w: synth.Workload, seeds: Sequence[int], device, n_objects: Optional[int] = None):
    """Projections [1, V, H, W] and voxelised volumes [1, Z, Y, X] of seeded phantoms."""
    gs, vols = [], []
    n = n_objects or w.n_objects
    for s in seeds:
        blobs = synth.random_ellipsoids(np.random.default_rng(s), n, w.r_fov())
        gs.append(synth.project_phantom(blobs, w.orbit, w.det_rows, w.det_cols, w.pitch,
                                        device=device, dtype=torch.float32)[None].contiguous())
        vols.append(synth.phantom_volume(blobs, w.vol_shape, w.voxel, device=device)[None]
                    .to(torch.float32).contiguous())
    return gs, vols


def train(net: DefriseClackNet, gs: List[torch.Tensor], refs: List[torch.Tensor],
          epochs: int, lr_max: float = 1e-2, weight_decay: float = 0.0,
          pct_start: float = 0.3, log=None) -> List[float]:
    """AdamW + one-cycle over `epochs` passes of the (g, ref) pairs; returns
    the mean loss of every epoch."""
    opt = torch.optim.AdamW(net.parameters(), lr=lr_max, weight_decay=weight_decay)
    sched = torch.optim.lr_scheduler.OneCycleLR(
        opt, max_lr=lr_max, epochs=epochs, steps_per_epoch=len(gs), pct_start=pct_start,
        div_factor=10.0, final_div_factor=1.0, cycle_momentum=False)
    hist = []
    for ep in range(epochs):
        tot = 0.0
        for g, ref in zip(gs, refs):
            opt.zero_grad(set_to_none=True)
            loss = relative_mse(net(g), ref)
            loss.backward()
            opt.step()
            sched.step()
            tot += float(loss.detach())
        hist.append(tot / len(gs))
        if log:
            log(f"epoch {ep + 1}/{epochs}: loss {hist[-1]:.5f}")
    return hist


@torch.no_grad()
def evaluate(geom: api.Geometry, W: Optional[torch.Tensor], gs, refs, relu: bool = True) -> float:
    """Mean relative MSE of the reconstructions with weight W over the pairs."""
    errs = [float(relative_mse(reconstruct(g, W, geom, relu), ref)) for g, ref in zip(gs, refs)]
    return float(np.mean(errs))


def compare(workload="sinusoid256_train", epochs: int = 40, n_train: int = 4,
            n_test: int = 2, lr_max: float = 1e-2, smooth=(20.0, 60), init="uniform",
            device="cuda", log=print) -> dict:
    """Train W on seeded phantoms, then compare learned and analytic weights
    on held-out phantoms.  `workload` is a preset name or a synth.Workload."""
    w = synth.workload(workload) if isinstance(workload, str) else workload
    geom = api.Geometry(w.desc_dict(), w.matrices(), w.orbit.vdl)
    gs, refs = make_data(w, range(1000, 1000 + n_train), device)
    gt, rt = make_data(w, range(2000, 2000 + n_test), device)
    net = DefriseClackNet(geom, init=init, relu=True, device=device, smooth=smooth)
    t0 = time.time()
    hist = train(net, gs, refs, epochs, lr_max, log=log)
    torch.cuda.synchronize()
    secs = time.time() - t0
    with torch.no_grad():
        W_learned = net.weights().detach()
    segs = None if w.orbit.closed else [(0, False)]
    res = {"workload": w.name, "epochs": epochs, "train_phantoms": n_train,
           "test_phantoms": n_test, "smooth": list(smooth) if smooth else None, "init": init,
           "loss_first_epoch": hist[0], "loss_last_epoch": hist[-1],
           "train_seconds": secs,
           "test_rel_mse": {"learned": evaluate(geom, W_learned, gt, rt),
                            "half": evaluate(geom, None, gt, rt),
                            "eq9": evaluate(geom, api.dc_crofton_weights(geom, segs), gt, rt)}}
    api.dc_sync_status(geom)
    geom.close()
    return res


def main():
    ap = argparse.ArgumentParser(description=__doc__.splitlines()[0])
    ap.add_argument("--workload", default="sinusoid256_train")
    ap.add_argument("--epochs", type=int, default=40)
    ap.add_argument("--train", type=int, default=4)
    ap.add_argument("--test", type=int, default=2)
    ap.add_argument("--lr", type=float, default=1e-2)
    ap.add_argument("--no-smooth", action="store_true")
    ap.add_argument("--init", default="uniform")
    a = ap.parse_args()
    init = a.init if a.init == "uniform" else float(a.init)
    print(json.dumps(compare(a.workload, a.epochs, a.train, a.test, a.lr,
                             None if a.no_smooth else (20.0, 60), init)))


if __name__ == "__main__":
    main()
