#!/usr/bin/env python
"""Benchmark of the Defrise-Clack reconstruction on GB300.

One step reconstructs one volume per GPU (Eq. 12): dc_filter over every view,
then dc_backproject.  Default workload: circle (360 views) plus a
perpendicular 60-degree arc (136 views), 384x512 detector at 0.6 mm,
720 x 512 planes per view, 512^3 volume, FP32 (the circle-plus-arc
configuration of the paper's workload class), seeded 20-ellipsoid phantom
with exact line integrals.  g^F is stored as FP32 (value, right difference)
pairs by default (--storage f32x2: the FP32 values and their FP32
differences, which the backprojection reads as its interpolation tiles);
--storage f32 / bf16 / f16 time the other forms.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

N > 1 is launched by torchrun: every rank reconstructs its own phantom (weak
scaling, no collective on the data path); rank 0 prints one JSON line.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "512³ DC-FBP recon ms/volume"
# bounded sample of the oracle at the 512^3 workload: 32 views of the filter
# and 20000 voxels of the backprojection over all views
ORACLE_SAMPLE_VIEWS = 32
ORACLE_SAMPLE_VOXELS = 20000
UNIT = "ms/volume"
PEAKS_FILE = os.path.join(ROOT, "MEASURED_PEAKS.json")

# FP32 operations the algorithm needs per unit of work (FMA = 2, a floor or
# a reciprocal = 1), used for the ALU roofline of the gather kernels:
#   k_bp3d    per voxel-view update, with the projected row differences
#             (g[r][j+1] - g[r][j]) stored beside the values:
#             a view whose u and depth are constant along a z column (a
#             circle about z): v FMA (2), floor + fraction (2), two row
#             lerps (FMA each, 4), lerp across rows (sub + FMA, 3), distance
#             weight (2 FMA, reciprocal, multiply: 6), accumulate (1) -> 18;
#             any other view adds depth FMA + reciprocal (3), u (2 FMA, 4),
#             v's perspective FMA (2), floor + fraction of u (2)      -> 29;
#             the unit count is weighted by the workload's mix of views
#   k_linesum per Joseph step: position FMA, fraction, lerp (sub+FMA),
#             accumulate                                                -> 7
#   k_bp2d    per pixel-angle pair: position FMA, fraction, two hat
#             weights (FMA+max each), two taps (FMA each)               -> 13
FLOPS_PER_UNIT = {"k_bp3d": None, "k_linesum": 7.0, "k_bp2d": 13.0}
BP_FLOPS_COLUMN_VIEW, BP_FLOPS_GENERAL_VIEW = 18.0, 29.0


def bp_flops_per_update(geom) -> tuple:
    """FP32 operations per voxel-view update of the backprojection for this
    geometry's mix of views (see FLOPS_PER_UNIT), and the fraction of views
    whose u and depth are constant along a z column (the backprojector's own
    test: the FP32 z-components of the l_x and l_z rows are zero)."""
    from paper_2410_14900_gb300 import api
    v = api.dc_get_view_geometry(geom)
    col = (np.float32(v[:, 5]) == 0) & (np.float32(v[:, 11]) == 0)
    frac = float(np.mean(col))
    return BP_FLOPS_COLUMN_VIEW * frac + BP_FLOPS_GENERAL_VIEW * (1.0 - frac), frac
SM_COUNT = 152
FP32_LANES_PER_SM = 128


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="circle_arc512")
    ap.add_argument("--storage", default="f32x2", choices=["f32", "f32x2", "bf16", "f16"])
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-forms", action="store_true")
    ap.add_argument("--no-train", action="store_true")
    ap.add_argument("--no-batched", action="store_true")
    ap.add_argument("--no-paper-shape", action="store_true")
    ap.add_argument("--no-interp-peak", action="store_true")
    ap.add_argument("--batched-only", action="store_true",
                    help="only the batched-orbits measurement (for profiling)")
    ap.add_argument("--train-only", action="store_true",
                    help="only the training-step measurement (for profiling)")
    ap.add_argument("--profile-case", choices=["filter_bp", "adj"], default=None,
                    help="run one small case twice for an ncu capture and exit: filter_bp = "
                         "the headline orbit, detector and planes with a 256^3 volume at the "
                         "headline voxel size (19 images per filter chunk); adj = the "
                         "backprojection transpose on the 256^3 sinusoid training geometry "
                         "with 90 views, batch 1")
    return ap.parse_args()


def profile_case(case: str, dev, storage: str = "f32"):
    """Small cases whose kernels are those of the full workloads, for ncu
    captures that end quickly (inputs still larger than L2)."""
    import torch
    from paper_2410_14900_gb300 import api, synth
    if case == "filter_bp":
        w = synth.workload("circle_arc512")
        desc = w.desc_dict()
        desc.update(vol_x=256, vol_y=256, vol_z=256)
        geom = api.Geometry(desc, w.matrices(), w.orbit.vdl)
        api.dc_geometry_set_tuning(geom, 19, 32)
        g = torch.randn((1, w.n_views, w.det_rows, w.det_cols), device=dev)
        for _ in range(2):
            gF, _ = api.dc_filter(geom, g, None, storage)
            api.dc_backproject(geom, gF)
    else:
        w = synth.scaled_workload("sinusoid256_train", views=90)
        geom = api.Geometry(w.desc_dict(), w.matrices(), w.orbit.vdl)
        gv = torch.randn((1,) + geom.vol_shape, device=dev)
        for _ in range(2):
            api.dc_backproject_adjoint(geom, gv)
    torch.cuda.synchronize()
    api.dc_sync_status(geom)
    geom.close()
    print(json.dumps({"profile_case": case, "ok": True}), flush=True)


# --------------------------------------------------------------- utilities
class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.thread.join(timeout=2)
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx = float(parts[2])
            except ValueError:
                continue
            for nm, val in zip(names, parts[5:9]):
                if val.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


def load_peaks():
    try:
        return json.load(open(PEAKS_FILE)), "measured"
    except Exception:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "sm_max_mhz": 2070.0}, "fallback"


KERNEL_SOURCES = {"k_bp3d": "paper_2410_14900_gb300/csrc/dc_backproject.cu",
                  "k_linesum": "paper_2410_14900_gb300/csrc/dc_filter.cu",
                  "k_bp2d": "paper_2410_14900_gb300/csrc/dc_filter.cu"}


def recorded_traffic(kernel: str, per_launch_units: float):
    """DRAM bytes per launch from the ncu capture recorded in
    profiles/traffic.json, scaled to this launch's work units; None when no
    capture exists or the kernel's source changed since it was taken."""
    import hashlib
    try:
        rec = json.load(open(os.path.join(ROOT, "profiles", "traffic.json")))[kernel]
        src = open(os.path.join(ROOT, KERNEL_SOURCES[kernel]), "rb").read()
    except Exception:
        return None
    if hashlib.sha256(src).hexdigest() != rec.get("source_sha256"):
        return None
    return rec["dram_bytes_per_launch"] * per_launch_units / rec["units_per_launch"]


def work_units(desc, B):
    """Algorithmic units per step: Joseph steps, pixel-angle pairs, updates."""
    V, H, W = desc["n_views"], desc["det_rows"], desc["det_cols"]
    n_mu, n_s = desc["n_mu"], desc["n_s"]
    # steps per line: detector rows for the row-stepping angles (the same
    # integer test as the library: 4m < n_mu or 4m >= 3 n_mu), columns else
    rows = sum(H if (4 * m < n_mu or 4 * m >= 3 * n_mu) else W for m in range(n_mu))
    return {"k_linesum": float(B) * V * rows * n_s,
            "k_bp2d": float(B) * V * n_mu * H * W,
            "k_bp3d": float(B) * V * desc["vol_x"] * desc["vol_y"] * desc["vol_z"]}


def interp_peaks(L, dev) -> dict:
    """Practical peaks of the three gather cores on this GPU (dc_microbench:
    the bare inner step on a resident shared-memory tile), steps per second."""
    import torch
    nb, iters = 152 * 4, 4000
    sink = torch.empty(nb * 512, device=dev)
    stream = torch.cuda.current_stream()
    out = {}
    for kind, name in enumerate(("joseph_step", "hat_pair", "bilinear_sample",
                                 "weighted_sample", "quad_weighted_sample")):
        for _ in range(2):
            L.dc_microbench(kind, nb, 100, sink.data_ptr(), stream.cuda_stream)
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        rc = L.dc_microbench(kind, nb, iters, sink.data_ptr(), stream.cuda_stream)
        e1.record(stream)
        torch.cuda.synchronize()
        if rc != 0:
            raise RuntimeError(L.dc_last_error().decode())
        out[name + "_peak_per_s"] = nb * 512.0 * iters * 32 / (e0.elapsed_time(e1) * 1e-3)
    return out


# --------------------------------------------------------------- CPU oracle
def oracle_sample(w, g_np, n_views_sample: int, n_vox_sample: int, seed: int = 0):
    """Time the FP64 oracle on a bounded sample and scale to one volume (ms)."""
    from oracle import oracle as orc
    desc = w.desc_dict()
    geom = orc.Geometry(desc, w.matrices(), w.orbit.vdl)
    V = desc["n_views"]
    rng = np.random.default_rng(seed)
    views = np.sort(rng.choice(V, size=min(n_views_sample, V), replace=False))
    t0 = time.perf_counter()
    orc.filter(geom, g_np[views][None], None, views=views)
    t_f = time.perf_counter() - t0
    nvox = desc["vol_x"] * desc["vol_y"] * desc["vol_z"]
    flat = rng.choice(nvox, size=min(n_vox_sample, nvox), replace=False)
    gF = rng.standard_normal((V, desc["det_rows"], desc["det_cols"]))
    t0 = time.perf_counter()
    orc.backproject_points(geom, gF, flat)
    t_b = time.perf_counter() - t0
    ms = 1e3 * (t_f * V / len(views) + t_b * nvox / len(flat))
    sample = (f"FP64 oracle filter on {len(views)} of {V} views and backprojection of "
              f"{len(flat)} of {nvox} voxels over all views, scaled linearly to one volume")
    return ms, sample, orc.num_threads(), t_f + t_b, len(views), len(flat)


def oracle_full(names=("circle64", "sinusoid256"), device=None) -> dict:
    """The FP64 oracle's complete reconstruction (Eq. 12, no sampling) of the
    two smaller configurations: 64-view circle 64^2 -> 64^3 and 360-view
    sinusoid 256^2 -> 256^3 with Poisson noise, timed on the host cores (the
    input projections are generated beforehand, on `device` if given,
    outside the timing).  With a device, the CUDA reconstruction of the same
    FP32-rounded input is timed beside it (CUDA events, 5 runs after 2
    warm-up runs) and compared with the oracle's volume (relative L2)."""
    import torch
    from oracle import oracle as orc
    from paper_2410_14900_gb300 import api, synth
    out = {}
    for name in names:
        w = synth.workload(name)
        og = orc.Geometry(w.desc_dict(), w.matrices(), w.orbit.vdl)
        g = synth.project_phantom(w.phantoms()[0], w.orbit, w.det_rows, w.det_cols, w.pitch,
                                  device=device, dtype=torch.float64)
        if w.photons:
            g = synth.add_poisson_noise(g, w.photons, 0.02, seed=w.seed)
        if device is not None:
            g = g.cpu().numpy()
        g32 = g.astype(np.float32).astype(np.float64)
        t0 = time.perf_counter()
        ref = orc.reconstruct(og, g32[None])
        rec = {"ms_per_volume": 1e3 * (time.perf_counter() - t0), "views": w.n_views,
               "detector": [w.det_rows, w.det_cols], "volume": list(w.vol_shape),
               "extrapolated": False}
        if device is not None:
            geom = api.Geometry(w.desc_dict(), w.matrices(), w.orbit.vdl)
            gt = torch.as_tensor(g32, device=device, dtype=torch.float32)[None].contiguous()
            for _ in range(2):
                vol = api.reconstruct(geom, gt)
            torch.cuda.synchronize()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record()
            for _ in range(5):
                vol = api.reconstruct(geom, gt)
            e1.record()
            torch.cuda.synchronize()
            v = vol.double().cpu().numpy()
            rec["gpu_ms_per_volume"] = e0.elapsed_time(e1) / 5
            rec["gpu_rel_l2_vs_oracle"] = float(np.linalg.norm(v - ref) / np.linalg.norm(ref))
            api.dc_sync_status(geom)
            geom.close()
        out[name] = rec
    return out


def workload_config(w, storage: str, B: int, world: int) -> dict:
    """The `config` both arms report for a workload."""
    return {"workload": w.name, "orbit": w.orbit.kind, "views": w.n_views,
            "detector": [w.det_rows, w.det_cols], "pitch_mm": w.pitch,
            "planes": [w.n_mu, w.n_s], "volume": list(w.vol_shape),
            "voxel_mm": list(w.voxel), "storage": storage,
            "batch_per_gpu": B, "parallelism": f"replicas x{world}"}


# --------------------------------------------------------------- reference arm
def run_reference(args, rank, world):
    """The oracle (this tier's reference) on the host cores, rank 0 only."""
    from paper_2410_14900_gb300 import synth
    if rank != 0:
        return
    w = synth.workload(args.workload)
    # a small stand-in projection set is enough: the oracle's cost does not
    # depend on the values
    g = np.random.default_rng(0).standard_normal((w.n_views, w.det_rows, w.det_cols))
    nv = min(ORACLE_SAMPLE_VIEWS, w.n_views)
    nvox = ORACLE_SAMPLE_VOXELS
    for _ in range(args.warmup):
        oracle_sample(w, g, 1, 1000)
    times = []
    sample = ""
    cores = 0
    for k in range(args.steps):
        ms, sample, cores, _, nvs, nxs = oracle_sample(w, g, nv, nvox, seed=k)
        times.append(ms)
    val = statistics.mean(times)
    line = {"impl": "reference", "metric": METRIC, "value": val, "unit": UNIT,
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": val,
            "higher_is_better": False, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": workload_config(w, args.storage, 1, world),
            "extrapolated": True,
            "cpu_baseline": {"value": val, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "extrapolated": True, "sample_views": nvs,
                             "sample_voxels": nxs, "sample": sample},
            "e2e": {"value": val, "unit": UNIT, "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# --------------------------------------------------------------- training
def train_step_measure(args, dev, L, world):
    """Forward + backward + AdamW step of the learnable redundancy weights:
    sinusoidal orbit, 360 views, 256^2 detector, 256^3 volume, batch of 4
    seeded phantoms, the Gaussian filter layer on W (sigma 20, kernel 121),
    MSE against the phantom volumes, ReLU output."""
    import torch
    from paper_2410_14900_gb300 import api, synth
    from paper_2410_14900_gb300.autograd import DefriseClackNet

    w = synth.workload("sinusoid256_train")
    geom = api.Geometry(w.desc_dict(), w.matrices(), w.orbit.vdl)
    phs = w.phantoms()
    g = torch.stack([synth.project_phantom(b, w.orbit, w.det_rows, w.det_cols, w.pitch,
                                           device=dev, dtype=torch.float32) for b in phs])
    tgt = torch.stack([synth.phantom_volume(b, w.vol_shape, w.voxel, device=dev) for b in phs])
    net = DefriseClackNet(geom, init=0.5, relu=True, device=dev, smooth=(20.0, 60))
    opt = torch.optim.AdamW(net.parameters(), lr=1e-3)

    def step():
        opt.zero_grad(set_to_none=True)
        loss = torch.nn.functional.mse_loss(net(g), tgt)
        loss.backward()
        opt.step()
        return loss

    for _ in range(max(1, args.warmup)):
        step()
    torch.cuda.synchronize()
    L.dc_profile_enable(1)
    L.dc_profile_collect(None, None, 0)
    stream = torch.cuda.current_stream()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        loss = step()
    e1.record(stream)
    torch.cuda.synchronize()
    ms_k = np.zeros(16)
    cnt_k = np.zeros(16, dtype=np.uint64)
    nk = L.dc_profile_collect(ms_k.ctypes.data, cnt_k.ctypes.data, 16)
    L.dc_profile_enable(0)
    kernels = {L.dc_profile_kernel_name(i).decode(): round(float(ms_k[i]) / args.steps, 3)
               for i in range(nk) if cnt_k[i]}
    ms = e0.elapsed_time(e1) / args.steps
    api.dc_sync_status(geom)
    geom.close()
    return {"workload": w.name, "ms_per_step": ms, "batch": w.batch,
            "views": w.n_views, "volume": list(w.vol_shape), "weights": [w.n_views, w.n_mu, w.n_s],
            "loss": float(loss.item()), "kernel_ms_per_step": kernels,
            "optimizer": "AdamW (lr 1e-3)", "smooth": [20.0, 60],
            "note": "forward + backward + optimizer step"}


def train_step_512_measure(args, dev, L):
    """Forward + backward + AdamW step at the 512^3 circle-plus-arc geometry
    (496 views, 384x512 detector, W of 496 x 720 x 512), batch 1, Gaussian
    filter layer on W, MSE against the phantom volume, ReLU output; once
    with Grangeat's S kept between the passes and once with S recomputed
    per chunk of 32 views (only g kept).  Reports each step's time and the
    peak of torch's allocator (every tensor of the step: projections,
    volumes, W with its gradient and AdamW moments, the kept S) plus the
    library's own work area."""
    import torch
    from paper_2410_14900_gb300 import api, synth
    from paper_2410_14900_gb300.autograd import DefriseClackNet

    w = synth.workload("circle_arc512")
    geom = api.Geometry(w.desc_dict(), w.matrices(), w.orbit.vdl)
    blobs = w.phantoms()[0]
    g = synth.project_phantom(blobs, w.orbit, w.det_rows, w.det_cols, w.pitch,
                              device=dev, dtype=torch.float32)[None].contiguous()
    tgt = synth.phantom_volume(blobs, w.vol_shape, w.voxel, device=dev)[None]
    t = api.dc_geometry_get_tuning(geom)
    per_img = 4 * (w.det_rows * ((w.det_cols + 3) // 4 * 4)
                   + 2 * w.n_mu * ((w.n_s + 3) // 4 * 4))
    work_bytes = int(t["chunk_capacity"]) * per_img
    stream = torch.cuda.current_stream()
    out = {"workload": w.name, "batch": 1, "views": w.n_views, "volume": list(w.vol_shape),
           "weights": [w.n_views, w.n_mu, w.n_s], "optimizer": "AdamW (lr 1e-3)",
           "smooth": [20.0, 60], "library_work_area_bytes": work_bytes,
           "note": "forward + backward + optimizer step"}
    steps = max(1, min(args.steps, 3))

    def measure(cache_s, chunk):
        # everything of one setting (the net, AdamW's moments, the autograd
        # graph of the last loss) dies when this returns
        net = DefriseClackNet(geom, init=0.5, relu=True, device=dev, smooth=(20.0, 60),
                              cache_s=cache_s, view_chunk=chunk)
        opt = torch.optim.AdamW(net.parameters(), lr=1e-3)

        def step():
            opt.zero_grad(set_to_none=True)
            loss = torch.nn.functional.mse_loss(net(g), tgt)
            loss.backward()
            opt.step()
            return loss.detach()

        step()
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(steps):
            loss = step()
        e1.record(stream)
        torch.cuda.synchronize()
        return {"ms_per_step": e0.elapsed_time(e1) / steps, "steps": steps,
                "torch_peak_bytes": int(torch.cuda.max_memory_allocated(dev)),
                "view_chunk": chunk, "loss": float(loss)}

    import gc
    for name, cache_s, chunk in (("kept_s", True, 0), ("recompute_s_chunk32", False, 32)):
        gc.collect()
        torch.cuda.synchronize()
        torch.cuda.empty_cache()
        torch.cuda.reset_peak_memory_stats(dev)
        out[name] = measure(cache_s, chunk)
    api.dc_sync_status(geom)
    geom.close()
    return out


# --------------------------------------------------------------- batched
def batched_measure(args, dev, L):
    """12 uneven orbits (4 circular, 4 sinusoidal, 4 circle plus arc; 200-720
    views; detectors 256^2 .. 616x480; volumes 128^3 .. 512^3) reconstructed by
    one graph-captured batch run (per-problem filters, one persistent
    backprojection), next to the same problems run one by one."""
    import torch
    from paper_2410_14900_gb300 import api, synth, tune

    ws = synth.batch_workloads()
    geoms = [api.Geometry(w.desc_dict(), w.matrices(), w.orbit.vdl) for w in ws]
    g_list = [synth.project_phantom(w.phantoms()[0], w.orbit, w.det_rows, w.det_cols, w.pitch,
                                    device=dev, dtype=torch.float32).contiguous() for w in ws]
    vols = [torch.empty(gm.vol_shape, device=dev) for gm in geoms]
    updates = float(sum(w.n_views * np.prod(w.vol_shape) for w in ws))
    stream = torch.cuda.current_stream()

    def timed(fn, reps):
        for _ in range(max(1, args.warmup)):
            fn()
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(reps):
            fn()
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / reps

    out = {"problems": len(ws), "views": [w.n_views for w in ws],
           "detectors": [[w.det_rows, w.det_cols] for w in ws],
           "volumes": [w.vol_shape[0] for w in ws], "voxel_view_updates": updates}
    for dtype, persistent in (("f32", False), ("bf16", False), ("f32", True), ("f32x2", False)):
        kh = dtype in ("bf16", "f16")
        batch = api.Batch(geoms, dtype=dtype, kahan=kh, persistent_filter=persistent)
        tuned = tune.autotune_batch(batch, g_list, vols, dtype=dtype, kahan=kh)
        batch.capture(g_list, vols)
        ms = timed(batch.replay, args.steps)
        tag = dtype + ("_persistent_filter" if persistent else "")
        out[f"{tag}_graph_ms_per_batch"] = ms
        out[f"{tag}_bp_nz"] = tuned["bp_nz"]
        batch.close()
        del batch
    # one by one, each problem with its own tuned box depth (set above by the
    # pair-storage tuning), in FP32 pair storage as the last batch
    def seq():
        for gm, g, v in zip(geoms, g_list, vols):
            gF, _ = api.dc_filter(gm, g[None], None, "f32x2")
            api.dc_backproject(gm, gF, out=v[None])
    out["f32x2_sequential_ms_per_batch"] = timed(seq, args.steps)
    out["f32_graph_ms_per_volume"] = out["f32_graph_ms_per_batch"] / len(ws)
    out["f32x2_graph_ms_per_volume"] = out["f32x2_graph_ms_per_batch"] / len(ws)
    for gm in geoms:
        api.dc_sync_status(gm)
        gm.close()
    return out


def paper_shape_measure(args, dev, L):
    """The paper's own workload shape (Tables 1-2: 400 views of a tilted
    sinusoid, 620x480 detector at 0.616 mm, 360 x 785 planes, 128x512x512
    volume at 0.25 mm), FP32, timed like the headline workload."""
    import torch
    from paper_2410_14900_gb300 import api, synth, tune

    w = synth.workload("paper400")
    geom = api.Geometry(w.desc_dict(), w.matrices(), w.orbit.vdl)
    st = args.storage if args.storage in ("f32", "f32x2") else "f32"
    tuned = tune.autotune(geom, st, chunks=(8, 12, 16, 20, 25), nzs=(16, 32))
    g = synth.project_phantom(w.phantoms()[0], w.orbit, w.det_rows, w.det_cols, w.pitch,
                              device=dev, dtype=torch.float32)[None].contiguous()
    gF = torch.empty(api.gF_shape(geom, 1, st), device=dev)
    vol = torch.empty((1,) + geom.vol_shape, device=dev)

    def step():
        api.dc_filter(geom, g, None, st, out=gF)
        api.dc_backproject(geom, gF, None, out=vol)

    stream = torch.cuda.current_stream()
    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    L.dc_profile_enable(1)
    L.dc_profile_collect(None, None, 0)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        step()
    e1.record(stream)
    torch.cuda.synchronize()
    ms_k = np.zeros(16, dtype=np.float64)
    cnt_k = np.zeros(16, dtype=np.uint64)
    nk = L.dc_profile_collect(ms_k.ctypes.data, cnt_k.ctypes.data, 16)
    L.dc_profile_enable(0)
    kern = {L.dc_profile_kernel_name(i).decode(): float(ms_k[i]) / args.steps
            for i in range(nk) if cnt_k[i]}
    api.dc_sync_status(geom)
    geom.close()
    bp = kern.get("k_bp3d", 0.0)
    return {"workload": w.name, "orbit": w.orbit.kind, "views": w.n_views,
            "detector": [w.det_rows, w.det_cols], "planes": [w.n_mu, w.n_s],
            "volume": list(w.vol_shape), "ms_per_volume": e0.elapsed_time(e1) / args.steps,
            "storage": st,
            "filter_ms": sum(kern.get(k, 0.0) for k in ("k_prep", "k_linesum", "k_bp2d",
                                                          "k_to_pairs")),
            "backproject_ms": bp,
            "bp_gups": w.n_views * float(np.prod(w.vol_shape)) / (bp * 1e-3) / 1e9 if bp else None,
            "tuning": {k: tuned[k] for k in ("chunk_images", "bp_nz")}}


# --------------------------------------------------------------- our arm
def run_ours(args, rank, world, local_rank):
    import torch
    import torch.distributed as dist

    from paper_2410_14900_gb300 import _lib, api, synth

    dev = torch.device("cuda", local_rank)
    torch.cuda.set_device(dev)
    L = _lib.load()
    w = synth.workload(args.workload)
    desc = w.desc_dict()
    geom = api.Geometry(desc, w.matrices(), w.orbit.vdl)
    # tile and chunk sizes picked by the autotuner (cached per problem shape)
    from paper_2410_14900_gb300 import tune
    tuned = tune.autotune(geom, args.storage, chunks=(8, 12, 16, 19, 24), nzs=(16, 32))
    # every rank reconstructs its own seeded phantom (independent problems)
    from paper_2410_14900_gb300 import sharding
    blobs = synth.random_ellipsoids(np.random.default_rng(sharding.rank_seed(w.seed, rank)),
                                    w.n_objects, w.r_fov())
    g = synth.project_phantom(blobs, w.orbit, w.det_rows, w.det_cols, w.pitch,
                              device=dev, dtype=torch.float32)[None].contiguous()
    B = 1
    V, H, Wd = w.n_views, w.det_rows, w.det_cols
    gF = torch.empty(api.gF_shape(geom, B, args.storage), device=dev,
                     dtype=api._DTYPES[args.storage][1])
    scale = torch.empty((B, V), device=dev) if args.storage == "f16" else None
    vol = torch.empty((B,) + geom.vol_shape, device=dev)
    kahan = args.storage in ("bf16", "f16")

    def step():
        api.dc_filter(geom, g, None, args.storage, out=gF, scale=scale)
        api.dc_backproject(geom, gF, scale, out=vol, kahan=kahan)

    def barrier():
        if world > 1:
            dist.barrier()

    stream = torch.cuda.current_stream()
    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    api.dc_sync_status(geom)
    barrier()
    torch.cuda.synchronize()

    sampler = ClockSampler(local_rank)
    sampler.start()
    L.dc_profile_enable(1)
    L.dc_profile_collect(None, None, 0)
    n0 = L.dc_launch_count()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        step()
    e1.record(stream)
    torch.cuda.synchronize()
    n_launch = L.dc_launch_count() - n0
    kid_n = 16
    ms_k = (np.zeros(kid_n, dtype=np.float64))
    cnt_k = (np.zeros(kid_n, dtype=np.uint64))
    nk = L.dc_profile_collect(ms_k.ctypes.data, cnt_k.ctypes.data, kid_n)
    L.dc_profile_enable(0)
    clocks = sampler.stop()
    barrier()
    torch.cuda.synchronize()
    ms_step = e0.elapsed_time(e1) / args.steps
    ms_step = sharding.max_over_ranks(ms_step, dist if world > 1 else None, dev)
    api.dc_sync_status(geom)

    kernels = {}
    for i in range(nk):
        name = L.dc_profile_kernel_name(i).decode()
        if cnt_k[i]:
            kernels[name] = {"ms_total": float(ms_k[i]), "launches": int(cnt_k[i]),
                             "ms_per_launch": float(ms_k[i] / cnt_k[i])}
    units = work_units(desc, B)
    interp = interp_peaks(L, dev) if not args.no_interp_peak else None
    peaks, peak_kind = load_peaks()
    sm_max = float(peaks.get("sm_max_mhz", 2070.0))
    fp32_peak_tflops = SM_COUNT * FP32_LANES_PER_SM * 2 * sm_max * 1e6 / 1e12
    dom = max(kernels, key=lambda k: kernels[k]["ms_total"])
    roof = None
    flops_unit = dict(FLOPS_PER_UNIT)
    flops_unit["k_bp3d"], column_view_frac = bp_flops_per_update(geom)
    if dom in flops_unit:
        per_launch_units = units[dom] * args.steps / kernels[dom]["launches"]
        ach = per_launch_units * flops_unit[dom] / (kernels[dom]["ms_per_launch"] * 1e-3) / 1e12
        roof = {"kernel": dom, "bound": "alu", "achieved": ach, "peak": fp32_peak_tflops,
                "unit": "TFLOP/s", "frac": ach / fp32_peak_tflops,
                "traffic": recorded_traffic(dom, per_launch_units),
                "peak_source": f"FP32 issue rate: {SM_COUNT} SMs x {FP32_LANES_PER_SM} lanes x "
                               f"2 x {sm_max:.0f} MHz (max clock of {peak_kind} peaks)",
                "units_per_launch": per_launch_units,
                "flops_per_unit": flops_unit[dom],
                "column_view_fraction": column_view_frac if dom == "k_bp3d" else None}
    filter_ms = sum(kernels.get(k, {}).get("ms_total", 0.0)
                    for k in ("k_prep", "k_linesum", "k_bp2d", "k_to_f16", "k_to_pairs")) / args.steps
    bp_ms = kernels.get("k_bp3d", {}).get("ms_total", 0.0) / args.steps
    hbm_bytes = (B * V * H * Wd * 4  # read g
                 + 2 * gF.numel() * gF.element_size()  # write + read g^F
                 + vol.numel() * 4)  # write f
    if interp:
        # each kernel's own rate (work units per second of its launches) as
        # a fraction of the bare inner step's rate on this GPU
        for kname, kind in (("k_linesum", "joseph_step"), ("k_bp2d", "hat_pair"),
                            ("k_bp3d", "bilinear_sample"), ("k_bp3d", "weighted_sample")):
            if kname in kernels:
                rate = units[kname] * args.steps / (kernels[kname]["ms_total"] * 1e-3)
                interp[kind + "_kernel_per_s"] = rate
                interp[kind + "_frac"] = rate / interp[kind + "_peak_per_s"]
    breakdown = {"filter_ms": filter_ms, "backproject_ms": bp_ms,
                 "bp_gups": units["k_bp3d"] / (bp_ms * 1e-3) / 1e9 if bp_ms else None,
                 "algorithmic_hbm_bytes": hbm_bytes,
                 "hbm_frac_of_step": hbm_bytes / (ms_step * 1e-3) / 1e9 / peaks.get("hbm_gbs", 6772.2),
                 "interp_peak": interp,
                 "kernels": kernels}

    # end to end through the public API with host buffers: dc_reconstruct_host
    # overlaps the uploads and downloads with the kernels; the serial form
    # (copy in, filter, backproject, copy out) is timed beside it
    e2e = None
    if not args.no_e2e:
        g_host = g.cpu().pin_memory()
        vol_host = torch.empty(vol.shape, dtype=torch.float32).pin_memory()
        g_dev = torch.empty_like(g)

        def e2e_step():
            api.dc_reconstruct_host(geom, g_host, vol_host, dtype=args.storage, kahan=kahan,
                                    g_dev=g_dev, gF=gF, scale=scale, vol_dev=vol)

        def serial_step():
            g_dev.copy_(g_host, non_blocking=True)
            gF2, sc2 = api.dc_filter(geom, g_dev, None, args.storage, out=gF, scale=scale)
            api.dc_backproject(geom, gF2, sc2, out=vol, kahan=kahan)
            vol_host.copy_(vol, non_blocking=True)

        def timed_e2e(fn):
            for _ in range(2):
                fn()
            torch.cuda.synchronize()
            barrier()
            a0 = torch.cuda.Event(enable_timing=True)
            a1 = torch.cuda.Event(enable_timing=True)
            a0.record(stream)
            for _ in range(args.steps):
                fn()
            a1.record(stream)
            torch.cuda.synchronize()
            t = a0.elapsed_time(a1) / args.steps
            return sharding.max_over_ranks(t, dist if world > 1 else None, dev)

        t_e2e = timed_e2e(e2e_step)
        breakdown["e2e_serial_ms"] = timed_e2e(serial_step) / B
        e2e = {"value": t_e2e / (B * world), "unit": UNIT,
               "h2d_bytes_per_step": int(g.numel() * 4), "d2h_bytes_per_step": int(vol.numel() * 4),
               "api": "dc_reconstruct_host (transfers overlapped with the kernels)"}

    # the other storage forms of g^F next to the timed one: FP32, FP32 pairs
    # (the same values; the backprojection reads its tiles in place), BF16 /
    # FP16 with Kahan summation
    forms = None
    if not args.no_forms and args.storage in ("f32", "f32x2"):
        forms = {f"{args.storage}_gF_bytes_per_volume": int(gF.numel() * gF.element_size())}
        for st in ("f32", "f32x2", "bf16", "f16"):
            if st == args.storage:
                continue
            kh = st in ("bf16", "f16")
            # voxels per thread along z tuned for this storage form
            ft = tune.autotune(geom, st, chunks=(tuned["chunk_images"],), nzs=(16, 32), kahan=kh)
            forms[f"{st}_bp_nz"] = ft["bp_nz"]
            gF2 = torch.empty(api.gF_shape(geom, B, st), device=dev, dtype=api._DTYPES[st][1])
            sc2 = torch.empty((B, V), device=dev) if st == "f16" else None
            for _ in range(2):
                api.dc_filter(geom, g, None, st, out=gF2, scale=sc2)
                api.dc_backproject(geom, gF2, sc2, out=vol, kahan=kh)
            torch.cuda.synchronize()
            f0 = torch.cuda.Event(enable_timing=True)
            f1 = torch.cuda.Event(enable_timing=True)
            f0.record(stream)
            for _ in range(args.steps):
                api.dc_filter(geom, g, None, st, out=gF2, scale=sc2)
                api.dc_backproject(geom, gF2, sc2, out=vol, kahan=kh)
            f1.record(stream)
            torch.cuda.synchronize()
            key = f"{st}_storage_kahan_ms_per_volume" if kh else f"{st}_storage_ms_per_volume"
            forms[key] = f0.elapsed_time(f1) / args.steps
            forms[f"{st}_gF_bytes_per_volume"] = int(gF2.numel() * gF2.element_size()
                                                     + (sc2.numel() * 4 if sc2 is not None else 0))
            del gF2
        api.dc_geometry_set_tuning(geom, tuned["chunk_images"], tuned["bp_nz"])

    batched = None
    if not args.no_batched:
        batched = batched_measure(args, dev, L)

    paper_shape = None
    if not args.no_paper_shape:
        paper_shape = paper_shape_measure(args, dev, L)

    train = None
    train512 = None
    if not args.no_train:
        del gF, vol
        torch.cuda.empty_cache()
        train = train_step_measure(args, dev, L, world)
        train512 = train_step_512_measure(args, dev, L)

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        g_np = g[0].double().cpu().numpy()
        nv = min(ORACLE_SAMPLE_VIEWS, V)
        ms, sample, cores, _, nvs, nxs = oracle_sample(w, g_np, nv, ORACLE_SAMPLE_VOXELS)
        cpu = {"value": ms, "unit": UNIT, "cores": cores, "kind": "oracle",
               "extrapolated": True, "sample_views": nvs, "sample_voxels": nxs,
               "sample": sample, "full_runs": oracle_full(device=dev)}

    if rank == 0:
        line = {"metric": METRIC, "value": sharding.whole_job_ms_per_volume(ms_step, B, world),
                "unit": UNIT, "n_gpus": world,
                "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_step,
                "higher_is_better": False, "scaling": "weak", "vs_baseline": None,
                "dtype": "f32", "data": "synthetic: seeded 20-ellipsoid phantom, exact line integrals",
                "config": workload_config(w, args.storage, B, world),
                "tuning": {k: tuned[k] for k in ("chunk_images", "bp_nz")},
                "l2": "inputs larger than L2 (g 390 MB, f 537 MB), no flush",
                "roofline": roof, "breakdown": breakdown, "forms": forms, "train_step": train,
                "train_step_512": train512,
                "batched": batched, "paper_shape": paper_shape,
                "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": int(n_launch),
                "clocks": clocks}
        print(json.dumps(line), flush=True)
    geom.close()


def main():
    args = parse()
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        run_reference(args, rank, world)
        return
    if args.profile_case:
        import torch
        torch.cuda.set_device(local_rank)
        profile_case(args.profile_case, torch.device("cuda", local_rank), args.storage)
        return
    if args.batched_only:
        import torch
        from paper_2410_14900_gb300 import _lib
        torch.cuda.set_device(local_rank)
        print(json.dumps({"batched": batched_measure(args, torch.device("cuda", local_rank),
                                                     _lib.load())}), flush=True)
        return
    if args.train_only:
        import torch
        from paper_2410_14900_gb300 import _lib
        torch.cuda.set_device(local_rank)
        dev = torch.device("cuda", local_rank)
        print(json.dumps({"train_step": train_step_measure(args, dev, _lib.load(), world),
                          "train_step_512": train_step_512_measure(args, dev, _lib.load())}),
              flush=True)
        return
    if world > 1:
        import torch
        import torch.distributed as dist
        torch.cuda.set_device(local_rank)
        dist.init_process_group("nccl")
    try:
        run_ours(args, rank, world, local_rank)
    finally:
        if world > 1:
            import torch.distributed as dist
            dist.destroy_process_group()


if __name__ == "__main__":
    main()
