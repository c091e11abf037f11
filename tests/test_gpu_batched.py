"""Batched reconstruction (one persistent backprojection over uneven
problems, their filters either chunked or in one persistent launch) and its
CUDA-graph capture: every volume against the FP64 oracle's reconstruction of
its own problem (Eq. 12), and against the per-problem calls."""
import numpy as np
import pytest
import torch

from oracle import oracle as orc
from paper_2410_14900_gb300 import api, synth, tune

from cases import rel_l2

pytestmark = pytest.mark.gpu


def _problems():
    ws = synth.batch_workloads(n=4, seed=300, max_views=48, max_det=(96, 128),
                               sizes=(32, 48, 64), min_views=16, min_det=64)
    out = []
    for w in ws:
        geom = api.Geometry(w.desc_dict(), w.matrices(), w.orbit.vdl)
        g = synth.project_phantom(w.phantoms()[0], w.orbit, w.det_rows, w.det_cols, w.pitch,
                                  device="cuda", dtype=torch.float32).contiguous()
        out.append((w, geom, g))
    return out


# FP32 and FP32 pairs: the method's 1e-4 target; BF16 / FP16 storage of g^F:
# the stated storage error of those forms (measured ~7e-4 and ~1e-4 on these
# problems).  A pair batch keeps the chunked filters even when the
# persistent one is asked for.
@pytest.mark.parametrize("persistent", [False, True])
@pytest.mark.parametrize("dtype,tol", [("f32", 1e-4), ("f32x2", 1e-4), ("bf16", 3e-3),
                                       ("f16", 5e-4)])
def test_batched_matches_oracle(dtype, tol, persistent):
    probs = _problems()
    geoms = [p[1] for p in probs]
    g_list = [p[2] for p in probs]
    rng = np.random.default_rng(17)
    W_np = [rng.uniform(0.2, 0.8, size=(gm.V,) + gm.sino_shape).astype(np.float32)
            for gm in geoms]
    W_list = [torch.as_tensor(Wn, device="cuda") for Wn in W_np]
    # one problem keeps the default weight 1/2
    W_list[1] = None
    batch = api.Batch(geoms, dtype=dtype, kahan=(dtype in ("bf16", "f16")),
                      persistent_filter=persistent)
    vols = [torch.full(geom.vol_shape, float("nan"), device="cuda") for geom in geoms]
    batch.run(g_list, vols, W_list)
    torch.cuda.synchronize()
    errs = []
    for i, ((w, geom, g), v) in enumerate(zip(probs, vols)):
        og = orc.Geometry(w.desc_dict(), w.matrices(), w.orbit.vdl)
        g_np = g.double().cpu().numpy()[None]
        ref = orc.reconstruct(og, g_np, None if W_list[i] is None else W_np[i])[0]
        errs.append(rel_l2(v.double().cpu().numpy(), ref))
    assert max(errs) < tol, errs
    for geom in geoms:
        api.dc_sync_status(geom)
    batch.close()


# The batched filter computes the 2-D backprojection in taller pixel tiles
# than the per-problem calls, so the s-bin positions are taken from other
# tile origins and g^F agrees to FP32 rounding (FP32: ~1e-7 after the
# backprojection); stored in 16 bits, a few values then round the other way
# (one BF16 / FP16 step is 2^-8 / 2^-11 of the value), ~1e-5 in the volume.
@pytest.mark.parametrize("dtype,tol", [("f32", 1e-6), ("bf16", 1e-4), ("f16", 2e-5)])
def test_batched_equals_per_problem_calls(dtype, tol):
    probs = _problems()
    geoms = [p[1] for p in probs]
    g_list = [p[2] for p in probs]
    batch = api.Batch(geoms, dtype=dtype, kahan=(dtype != "f32"), persistent_filter=True)
    vols = [torch.full(geom.vol_shape, float("nan"), device="cuda") for geom in geoms]
    batch.run(g_list, vols)
    for (w, geom, g), v in zip(probs, vols):
        gF, sc = api.dc_filter(geom, g[None], None, dtype)
        ref = api.dc_backproject(geom, gF, sc, kahan=(dtype != "f32"))[0]
        torch.cuda.synchronize()
        assert torch.isfinite(v).all()
        assert rel_l2(v.double().cpu().numpy(), ref.double().cpu().numpy()) < tol
    for geom in geoms:
        api.dc_sync_status(geom)
    batch.close()


def test_batched_graph_replay_and_weights():
    probs = _problems()
    geoms = [p[1] for p in probs]
    g_list = [p[2] for p in probs]
    W_list = [torch.rand((geom.V,) + geom.sino_shape, device="cuda") for geom in geoms]
    batch = api.Batch(geoms, persistent_filter=True)
    tuned = tune.autotune_batch(batch, g_list, [torch.empty(gm.vol_shape, device="cuda")
                                                for gm in geoms])
    assert tuned["bp_nz"] in (0, 16, 32)   # 0: each problem's own depth
    vols = [torch.zeros(geom.vol_shape, device="cuda") for geom in geoms]
    batch.capture(g_list, vols, W_list)
    for v in vols:
        v.fill_(float("nan"))
    batch.replay()
    torch.cuda.synchronize()
    for (w, geom, g), v, Wt in zip(probs, vols, W_list):
        ref = api.reconstruct(geom, g[None], Wt)[0]
        torch.cuda.synchronize()
        # the tuned box depth may differ from the handle's: summation order only
        assert rel_l2(v.double().cpu().numpy(), ref.double().cpu().numpy()) < 1e-5
    batch.close()


def test_autotune_caches_and_applies(tmp_path, monkeypatch):
    monkeypatch.setenv("DC_TUNE_CACHE", str(tmp_path / "tune.json"))
    w, geom, g = _problems()[0]
    r1 = tune.autotune(geom, chunks=(4, 8), nzs=(16, 32))
    assert not r1["cached"]
    r2 = tune.autotune(geom, chunks=(4, 8), nzs=(16, 32))
    assert r2["cached"] and r2["bp_nz"] == r1["bp_nz"]
    t = api.dc_geometry_get_tuning(geom)
    assert t["bp_nz"] == r1["bp_nz"] and t["chunk_images"] == r1["chunk_images"]
    # results do not depend on the tuning
    outs = []
    for nz in (16, 32):
        api.dc_geometry_set_tuning(geom, 4, nz)
        outs.append(api.reconstruct(geom, g[None]).double().cpu().numpy())
    assert rel_l2(outs[0], outs[1]) < 1e-6
