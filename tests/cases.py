"""Shared problem builders for the parity tests (inputs only, no arithmetic
of the method): geometry descriptors, projection matrices and seeded data."""
from __future__ import annotations

import dataclasses

import numpy as np

from paper_2410_14900_gb300 import synth


@dataclasses.dataclass
class Case:
    name: str
    desc: dict
    P: np.ndarray
    vdl: object
    orbit: synth.Orbit
    B: int


def from_workload(w: synth.Workload, B: int = 1, use_vdl: bool = True) -> Case:
    return Case(w.name, w.desc_dict(), w.matrices(), w.orbit.vdl if use_vdl else None,
                w.orbit, B)


def circle64() -> Case:
    """The small circular configuration (64 views, 64x64 detector, 64^3)."""
    return from_workload(synth.workload("circle64"))


def ragged(B: int = 2) -> Case:
    """Odd sizes everywhere: padding, partial tiles, off-centre volume."""
    o = synth.sinusoid_orbit(23)
    H, W, p = 37, 50, 1.5
    desc = dict(n_views=23, det_rows=H, det_cols=W, n_mu=33, n_s=45, pitch=p, ds=1.7,
                vol_x=37, vol_y=29, vol_z=21, voxel=(1.1, 0.9, 1.3),
                vol_center=(1.5, -2.0, 3.0), closed_orbit=1)
    return Case("ragged", desc, synth.projection_matrices(o, H, W, p), o.vdl, o, B)


def arc_open(B: int = 1) -> Case:
    """Circle-plus-arc pieces with tangents from finite differences (open)."""
    o = synth.circle_arc_orbit(20, 9)
    H, W, p = 48, 40, 1.6
    desc = dict(n_views=o.n_views, det_rows=H, det_cols=W, n_mu=40, n_s=40, pitch=p, ds=p,
                vol_x=24, vol_y=24, vol_z=20, voxel=(1.0, 1.0, 1.0),
                vol_center=(0.0, 0.0, 0.0), closed_orbit=0)
    return Case("arc_open", desc, synth.projection_matrices(o, H, W, p), None, o, B)


def random_nn(B: int = 1) -> Case:
    """The random nearest-neighbour orbit (open, finite-difference tangents)."""
    o = synth.random_nn_orbit(30, seed=3)
    H, W, p = 40, 48, 1.6
    desc = dict(n_views=o.n_views, det_rows=H, det_cols=W, n_mu=36, n_s=44, pitch=p, ds=p,
                vol_x=24, vol_y=24, vol_z=20, voxel=(1.0, 1.0, 1.0),
                vol_center=(0.0, 0.0, 0.0), closed_orbit=0)
    return Case("random_nn", desc, synth.projection_matrices(o, H, W, p), o.vdl, o, B)


def phantom_projections(case: Case, seed: int = 0, n: int = 8) -> np.ndarray:
    """[B,V,H,W] exact line integrals of seeded ellipsoid phantoms (FP64)."""
    d = case.desc
    r = synth.fov_radius(d["det_rows"], d["det_cols"], d["pitch"], d["n_s"], d["ds"],
                         float(np.linalg.norm(case.orbit.sources[0])), case.orbit.sdd)
    out = []
    for b in range(case.B):
        blobs = synth.random_ellipsoids(np.random.default_rng(seed + b), n, r)
        out.append(synth.project_phantom(blobs, case.orbit, d["det_rows"], d["det_cols"],
                                         d["pitch"]))
    return np.stack(out)


def random_weights(case: Case, seed: int = 5) -> np.ndarray:
    d = case.desc
    rng = np.random.default_rng(seed)
    return rng.uniform(0.2, 0.8, size=(d["n_views"], d["n_mu"], d["n_s"]))


def rel_l2(a, b) -> float:
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))
