"""Autotuner for the tile and chunk sizes of the CUDA library.

For a geometry it times the filter with several chunk sizes (images per
work-area chunk) and the backprojection with 16 or 32 voxels per thread
along z, on synthetic data of the problem's shape, with CUDA events, and
keeps the fastest.  Results are cached in a JSON file keyed by the problem
shape (DC_TUNE_CACHE, default ~/.cache/dracogb/tune.json).
"""
from __future__ import annotations

import json
import os
import threading

import torch

from . import api

_lock = threading.Lock()


def cache_path() -> str:
    return os.environ.get("DC_TUNE_CACHE",
                          os.path.join(os.path.expanduser("~"), ".cache", "dracogb", "tune.json"))


def shape_key(geom: api.Geometry, dtype: str = "f32") -> str:
    d = geom.desc
    return "V{n_views}_H{det_rows}_W{det_cols}_mu{n_mu}_s{n_s}_vol{vol_z}x{vol_y}x{vol_x}".format(
        **d) + f"_{dtype}"


def _load():
    try:
        with open(cache_path()) as f:
            return json.load(f)
    except Exception:
        return {}


def _store(db):
    p = cache_path()
    os.makedirs(os.path.dirname(p), exist_ok=True)
    tmp = p + f".tmp{os.getpid()}"
    with open(tmp, "w") as f:
        json.dump(db, f, indent=1, sort_keys=True)
    os.replace(tmp, p)


def _time(fn, reps=2):
    fn()
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(reps):
        fn()
    e1.record()
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / reps


def autotune(geom: api.Geometry, dtype: str = "f32", use_cache: bool = True,
             chunks=(8, 16, 32), nzs=(16, 32), kahan: bool = False) -> dict:
    """Pick chunk_images and bp_nz for `geom`, apply them and return them
    (the backprojection timed with Kahan summation when `kahan`)."""
    key = shape_key(geom, dtype) + ("|kahan" if kahan else "")
    with _lock:
        db = _load() if use_cache else {}
    if key in db:
        best = db[key]
        api.dc_geometry_set_tuning(geom, best["chunk_images"], best["bp_nz"])
        return dict(best, cached=True)
    cap = api.dc_geometry_get_tuning(geom)["chunk_capacity"]
    dev = torch.device("cuda", torch.cuda.current_device())
    g = torch.rand((1, geom.V, geom.H, geom.W), device=dev)
    gF = torch.empty(api.gF_shape(geom, 1, dtype), device=dev, dtype=api._DTYPES[dtype][1])
    sc = torch.empty((1, geom.V), device=dev) if dtype == "f16" else None
    vol = torch.empty((1,) + geom.vol_shape, device=dev)
    res = {"filter_ms": {}, "bp_ms": {}}
    for c in sorted({min(c, cap) for c in chunks}):
        api.dc_geometry_set_tuning(geom, c, 0)
        res["filter_ms"][c] = _time(lambda: api.dc_filter(geom, g, None, dtype, out=gF, scale=sc))
    best_c = min(res["filter_ms"], key=res["filter_ms"].get)
    for nz in nzs:
        api.dc_geometry_set_tuning(geom, 0, nz)
        res["bp_ms"][nz] = _time(lambda: api.dc_backproject(geom, gF, sc, out=vol, kahan=kahan))
    best_nz = min(res["bp_ms"], key=res["bp_ms"].get)
    api.dc_geometry_set_tuning(geom, best_c, best_nz)
    best = {"chunk_images": int(best_c), "bp_nz": int(best_nz),
            "filter_ms": {str(k): v for k, v in res["filter_ms"].items()},
            "bp_ms": {str(k): v for k, v in res["bp_ms"].items()}}
    if use_cache:
        with _lock:
            db = _load()
            db[key] = best
            _store(db)
    return dict(best, cached=False)


def autotune_batch(batch: "api.Batch", g_list, vol_list, nzs=(16, 32), dtype: str = "f32",
                   kahan: bool = False) -> dict:
    """Pick the batch backprojection's voxels per thread along z: one depth
    for every problem, or each problem's own (0: the depth `autotune` picks
    for that geometry alone), whichever runs the batch fastest."""
    per = {}
    for gm in batch.geoms:
        t = api.dc_geometry_get_tuning(gm)
        r = autotune(gm, dtype, chunks=(t["chunk_images"],), nzs=nzs, kahan=kahan)
        per[shape_key(gm, dtype)] = r["bp_nz"]
    times = {}
    for nz in (0,) + tuple(nzs):
        batch.set_bp_nz(nz)
        times[nz] = _time(lambda: batch.run(g_list, vol_list))
    best = min(times, key=times.get)
    batch.set_bp_nz(best)
    return {"bp_nz": int(best), "per_problem_nz": per,
            "run_ms": {str(k): v for k, v in times.items()}}
