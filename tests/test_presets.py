"""The synthetic workload presets carry the paper's printed geometry."""
import json
import math
import os

import numpy as np

from paper_2410_14900_gb300 import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "paper_geometry.json")


def test_paper_shape_preset_matches_tables_1_and_2():
    t = json.load(open(GOLDEN))
    w = synth.workload("paper400")
    t1, t2 = t["table1"], t["table2"]
    assert list(w.vol_shape) == t1["volume_shape"]
    assert list(w.voxel) == t1["volume_spacing_mm"]
    assert w.n_views == t1["n_projections"]
    assert abs(np.linalg.norm(w.orbit.sources, axis=1) - t1["source_isocenter_mm"]).max() < 1e-9
    assert w.orbit.sdd == t1["source_detector_mm"]
    assert w.pitch == t1["detector_spacing_mm"] == t2["detector_spacing_mm"] == w.ds
    assert [w.det_cols, w.det_rows] == t1["detector_shape_cols_rows"] == t2["image_shape"]
    assert w.n_mu == t2["n_angles"] and w.n_s == t2["detector_bins"]
    # Table 2's 785 bins cover the detector diagonal
    assert w.n_s == math.ceil(math.hypot(w.det_cols, w.det_rows))


def test_orbits_have_the_stated_shapes():
    c = synth.circle_orbit(400)
    assert np.allclose(np.linalg.norm(c.sources, axis=1), synth.SID_MM)
    s = synth.sinusoid_orbit(360)
    assert abs(s.sources[:, 2].max() - 40.0) < 0.1
    ca = synth.circle_arc_orbit(360, 136)
    assert ca.n_views == 496 and not ca.closed
    arc = ca.sources[360:]
    assert np.allclose(arc[:, 1], 0.0)
    ang = np.degrees(np.arctan2(arc[:, 2], arc[:, 0]))
    assert abs(ang[0] + 30) < 1e-9 and abs(ang[-1] - 30) < 1e-9
    t = synth.tilted_sinusoid_orbit(400)
    tilt = np.degrees(np.arcsin(t.sources[:, 2] / synth.SID_MM))
    assert abs(tilt.max() - 20.0) < 1e-6 and abs(tilt.min() + 20.0) < 0.5
    # analytic tangents agree with finite differences of the positions
    for o in (c, s, t):
        fd = 0.5 * (np.roll(o.sources, -1, 0) - np.roll(o.sources, 1, 0))
        assert np.abs(fd - o.vdl).max() < 2e-3 * np.abs(o.vdl).max()


def test_random_nearest_neighbour_orbit():
    """Sec. 4.4's random orbit: points on the sphere band of +-10 degrees,
    chained by nearest neighbour, tangents from central differences."""
    o = synth.random_nn_orbit(120, seed=4)
    a = o.sources
    assert o.n_views == 120 and not o.closed
    assert np.allclose(np.linalg.norm(a, axis=1), synth.SID_MM)
    assert np.degrees(np.abs(np.arcsin(a[:, 2] / synth.SID_MM))).max() <= 10.0 + 1e-9
    for i in range(len(a) - 2):   # every next point is the nearest of the rest
        d = np.sum((a[i + 1:] - a[i]) ** 2, axis=1)
        assert d[0] == d.min()
    assert np.allclose(o.vdl[1:-1], 0.5 * (a[2:] - a[:-2]))
    assert np.allclose(o.vdl[0], a[1] - a[0]) and np.allclose(o.vdl[-1], a[-1] - a[-2])
    # detector frame: orthonormal, principal ray through the isocentre
    for lx, ly, lz, ai in zip(o.lx, o.ly, o.lz, a):
        F = np.stack([lx, ly, lz])
        assert np.allclose(F @ F.T, np.eye(3), atol=1e-12)
        assert np.allclose(lz, ai / np.linalg.norm(ai))


def test_phantom_line_integrals_match_quadrature():
    rng = np.random.default_rng(0)
    for kind in ("ellipsoid", "gauss"):
        b = synth.random_ellipsoids(rng, 1, 40.0, kind)[0]
        src = np.array([750.0, 0.0, 0.0])
        d = b.center - src + np.array([0.0, 0.3, -0.2]) * b.axes.min()
        d /= np.linalg.norm(d)
        t = np.linspace(600.0, 900.0, 300001)
        pts = src + t[:, None] * d
        T = (b.rot / b.axes[None, :]).T
        q = np.sum((pts - b.center) @ T.T * ((pts - b.center) @ T.T), -1)
        f = (q <= 1.0) * b.rho if kind == "ellipsoid" else b.rho * np.exp(-0.5 * q)
        quad = np.trapezoid(f, t)
        exact = synth._line_integrals_np([b], src, d[None])[0]
        assert abs(quad - exact) < 2e-3 * max(exact, 1e-3)
