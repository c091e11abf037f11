"""Seeded synthetic inputs for the Defrise-Clack filtered backprojection.

This module produces *inputs* only: source orbits, 3x4 projection matrices,
per-view orbit tangents a'(lambda)*dlambda, random ellipsoid / Gaussian-blob
phantoms, their exact cone-beam line integrals and optional Poisson noise.
It holds none of the reconstruction arithmetic (no cosine weights, Radon
transforms, redundancy weights or backprojection); the CPU oracle and the
CUDA library both take what it returns as plain arrays.

Conventions (shared by every consumer, stated here once):

* World coordinates in mm, isocentre at the origin, radians for angles.
* Detector frame per view (paper Fig. 1): origin O at the detector centre,
  l_x and l_y in the detector plane, l_z the unit vector pointing from the
  detector towards the source, source a = O + D*l_z.  The principal ray passes
  through the isocentre: l_z = a/|a|, l_y is world z projected orthogonally to
  l_z, l_x = l_y x l_z.
* Pixel (col j, row r) sits at O + (j - c_u)*p*l_x + (r - c_v)*p*l_y with
  c_u = (W-1)/2, c_v = (H-1)/2.
* A projection matrix maps a homogeneous world point to (j*w, r*w, w) where
  w is the depth of the point in front of the source along -l_z (mm).
* Projections are stored [V][H][W] (column index fastest); volumes [Z][Y][X].

Workload presets follow Tables 1-2 of the paper (geometry class: SID 750 mm,
SDD 1200 mm) at the sizes of the five benchmark configurations.
"""
from __future__ import annotations

import dataclasses
import math
from typing import List, Optional, Sequence

import numpy as np

try:  # torch is only needed for the fast (device) line-integral evaluation
    import torch
except Exception:  # pragma: no cover - torch is always present in this project
    torch = None

SID_MM = 750.0   # source to isocentre (Table 1)
SDD_MM = 1200.0  # source to detector (Table 1)


# --------------------------------------------------------------------------
# Orbits
# --------------------------------------------------------------------------
@dataclasses.dataclass
class Orbit:
    """Source positions, detector frames and tangents for one scan."""

    kind: str
    sources: np.ndarray      # [V,3] source positions a_i (mm)
    lx: np.ndarray           # [V,3]
    ly: np.ndarray           # [V,3]
    lz: np.ndarray           # [V,3]
    vdl: np.ndarray          # [V,3] a'(lambda_i) * dlambda_i (mm)
    sdd: float               # source-detector distance D (mm)
    closed: bool             # True when the orbit is a closed curve

    @property
    def n_views(self) -> int:
        return int(self.sources.shape[0])


def _frame(a: np.ndarray):
    """Detector frame for source positions a [V,3] (principal ray -> origin)."""
    lz = a / np.linalg.norm(a, axis=1, keepdims=True)
    ez = np.array([0.0, 0.0, 1.0])
    ly = ez[None, :] - (lz @ ez)[:, None] * lz
    ly /= np.linalg.norm(ly, axis=1, keepdims=True)
    lx = np.cross(ly, lz)
    return lx, ly, lz


def circle_orbit(n_views: int, sid: float = SID_MM, sdd: float = SDD_MM) -> Orbit:
    """Full circle in the z=0 plane, phi_i = 2*pi*i/V."""
    phi = 2.0 * math.pi * np.arange(n_views) / n_views
    a = np.stack([sid * np.cos(phi), sid * np.sin(phi), np.zeros_like(phi)], 1)
    dphi = 2.0 * math.pi / n_views
    vdl = np.stack([-sid * np.sin(phi), sid * np.cos(phi), np.zeros_like(phi)], 1) * dphi
    lx, ly, lz = _frame(a)
    return Orbit("circle", a, lx, ly, lz, vdl, sdd, True)


def sinusoid_orbit(n_views: int, sid: float = SID_MM, sdd: float = SDD_MM,
                   amp: float = 40.0) -> Orbit:
    """Circle of radius `sid` with an axial offset amp*sin(2*phi) (mm)."""
    phi = 2.0 * math.pi * np.arange(n_views) / n_views
    a = np.stack([sid * np.cos(phi), sid * np.sin(phi), amp * np.sin(2 * phi)], 1)
    dphi = 2.0 * math.pi / n_views
    vdl = np.stack([-sid * np.sin(phi), sid * np.cos(phi),
                    2.0 * amp * np.cos(2 * phi)], 1) * dphi
    lx, ly, lz = _frame(a)
    return Orbit("sinusoid", a, lx, ly, lz, vdl, sdd, True)


def tilted_sinusoid_orbit(n_views: int, sid: float = SID_MM, sdd: float = SDD_MM,
                          tilt_max_deg: float = 20.0, freq: float = 5.0) -> Orbit:
    """Sphere-surface sinusoid of Eq. 15: tilt phi = phi_max*cos(f*theta)."""
    th = -math.pi + 2.0 * math.pi * np.arange(n_views) / n_views
    tmax = math.radians(tilt_max_deg)
    ph = tmax * np.cos(freq * th)
    a = sid * np.stack([np.cos(ph) * np.cos(th), np.cos(ph) * np.sin(th), np.sin(ph)], 1)
    dth = 2.0 * math.pi / n_views
    dph = -tmax * freq * np.sin(freq * th)
    da = sid * np.stack([
        -np.sin(ph) * dph * np.cos(th) - np.cos(ph) * np.sin(th),
        -np.sin(ph) * dph * np.sin(th) + np.cos(ph) * np.cos(th),
        np.cos(ph) * dph], 1)
    lx, ly, lz = _frame(a)
    return Orbit("tilted_sinusoid", a, lx, ly, lz, da * dth, sdd, True)


def random_nn_orbit(n_views: int = 400, sid: float = SID_MM, sdd: float = SDD_MM,
                    tilt_deg: float = 10.0, seed: int = 0) -> Orbit:
    """Random points on the sphere band |tilt| <= tilt_deg (azimuth U[0, 2pi),
    tilt U[-tilt_deg, tilt_deg]), ordered into a path by nearest neighbour
    from the first point (Sec. 4.4).  Open orbit; tangents from central
    differences of the ordered positions (one-sided at the ends)."""
    rng = np.random.default_rng(seed)
    th = rng.uniform(0.0, 2.0 * math.pi, n_views)
    ph = np.radians(rng.uniform(-tilt_deg, tilt_deg, n_views))
    pts = sid * np.stack([np.cos(ph) * np.cos(th), np.cos(ph) * np.sin(th), np.sin(ph)], 1)
    order = [0]
    left = set(range(1, n_views))
    while left:
        last = pts[order[-1]]
        nxt = min(left, key=lambda j: float(np.sum((pts[j] - last) ** 2)))
        order.append(nxt)
        left.remove(nxt)
    a = pts[order]
    v = np.zeros_like(a)
    v[1:-1] = 0.5 * (a[2:] - a[:-2])
    v[0] = a[1] - a[0]
    v[-1] = a[-1] - a[-2]
    lx, ly, lz = _frame(a)
    return Orbit("random_nn", a, lx, ly, lz, v, sdd, False)


def circle_arc_orbit(n_circle: int = 360, n_arc: int = 136, sid: float = SID_MM,
                     sdd: float = SDD_MM, arc_deg: float = 60.0) -> Orbit:
    """Full circle plus a perpendicular arc through the circle point phi=0.

    The arc lies in the x-z plane, psi in [-arc/2, +arc/2], uniform with both
    end points included.  The two pieces are separate open segments, so the
    tangents are given analytically for every view.
    """
    circ = circle_orbit(n_circle, sid, sdd)
    half = math.radians(arc_deg) / 2.0
    psi = np.linspace(-half, half, n_arc)
    a_arc = np.stack([sid * np.cos(psi), np.zeros_like(psi), sid * np.sin(psi)], 1)
    dpsi = (2.0 * half) / (n_arc - 1)
    v_arc = np.stack([-sid * np.sin(psi), np.zeros_like(psi), sid * np.cos(psi)], 1) * dpsi
    a = np.concatenate([circ.sources, a_arc], 0)
    vdl = np.concatenate([circ.vdl, v_arc], 0)
    lx, ly, lz = _frame(a)
    return Orbit("circle_arc", a, lx, ly, lz, vdl, sdd, False)


def projection_matrices(orbit: Orbit, det_rows: int, det_cols: int,
                        pitch: float) -> np.ndarray:
    """[V,3,4] FP64 matrices P_i = A_i [I | -a_i] (see module docstring)."""
    V = orbit.n_views
    f = orbit.sdd / pitch
    cu = (det_cols - 1) / 2.0
    cv = (det_rows - 1) / 2.0
    P = np.zeros((V, 3, 4))
    for i in range(V):
        A = np.stack([f * orbit.lx[i] - cu * orbit.lz[i],
                      f * orbit.ly[i] - cv * orbit.lz[i],
                      -orbit.lz[i]], 0)
        P[i, :, :3] = A
        P[i, :, 3] = -A @ orbit.sources[i]
    return P


def pixel_rays(orbit: Orbit, i: int, det_rows: int, det_cols: int, pitch: float):
    """Unit ray directions [H,W,3] from source i through every pixel centre."""
    cu = (det_cols - 1) / 2.0
    cv = (det_rows - 1) / 2.0
    x = (np.arange(det_cols) - cu) * pitch
    y = (np.arange(det_rows) - cv) * pitch
    d = (x[None, :, None] * orbit.lx[i][None, None, :]
         + y[:, None, None] * orbit.ly[i][None, None, :]
         - orbit.sdd * orbit.lz[i][None, None, :])
    return d / np.linalg.norm(d, axis=2, keepdims=True)


# --------------------------------------------------------------------------
# Phantoms
# --------------------------------------------------------------------------
@dataclasses.dataclass
class Blob:
    """An ellipsoid (kind='ellipsoid') or a Gaussian blob (kind='gauss').

    Ellipsoid:  rho on {x : |A^-1 Q^T (x-c)| <= 1}.
    Gaussian:   rho * exp(-|A^-1 Q^T (x-c)|^2 / 2).
    A = diag(axes), Q a rotation matrix.
    """

    kind: str
    center: np.ndarray   # [3]
    axes: np.ndarray     # [3]
    rot: np.ndarray      # [3,3]
    rho: float


def random_rotation(rng: np.random.Generator) -> np.ndarray:
    q = rng.normal(size=4)
    q /= np.linalg.norm(q)
    w, x, y, z = q
    return np.array([
        [1 - 2 * (y * y + z * z), 2 * (x * y - z * w), 2 * (x * z + y * w)],
        [2 * (x * y + z * w), 1 - 2 * (x * x + z * z), 2 * (y * z - x * w)],
        [2 * (x * z - y * w), 2 * (y * z + x * w), 1 - 2 * (x * x + y * y)]])


def fov_radius(det_rows: int, det_cols: int, pitch: float, n_s: int, ds: float,
               sid: float = SID_MM, sdd: float = SDD_MM) -> float:
    """Radius of the sphere about the isocentre seen by every view.

    e is the radius of the largest disc about the detector centre inside both
    the detector and the s-range of the sinogram; the sphere subtends e.
    """
    e = 0.5 * min(det_cols * pitch, det_rows * pitch, n_s * ds)
    return sid * math.sin(math.atan(e / sdd))


def random_ellipsoids(rng: np.random.Generator, n: int, r_fov: float,
                      kind: str = "ellipsoid", axis_range=(0.05, 0.3),
                      margin: float = 0.95) -> List[Blob]:
    """n seeded objects fully inside margin*r_fov (densities U[0,1]).

    Semi-axes ~ U[axis_range]*r_fov; the centre is uniform in the ball whose
    radius leaves room for the largest semi-axis (3 sigma for Gaussians).
    """
    out = []
    for _ in range(n):
        axes = rng.uniform(axis_range[0], axis_range[1], size=3) * r_fov
        reach = axes.max() * (3.0 if kind == "gauss" else 1.0)
        rmax = max(margin * r_fov - reach, 0.0)
        d = rng.normal(size=3)
        d /= np.linalg.norm(d)
        c = d * rmax * rng.uniform() ** (1.0 / 3.0)
        out.append(Blob(kind, c, axes, random_rotation(rng), float(rng.uniform(0.0, 1.0))))
    return out


def _line_integrals_np(blobs: Sequence[Blob], src: np.ndarray, dirs: np.ndarray) -> np.ndarray:
    """Exact line integrals of the phantom along rays src + t*dirs (|dirs|=1)."""
    out = np.zeros(dirs.shape[:-1])
    for b in blobs:
        T = (b.rot / b.axes[None, :]).T           # A^-1 Q^T
        y0 = T @ (src - b.center)
        d = dirs @ T.T
        dd = np.sum(d * d, axis=-1)
        bd = d @ y0
        if b.kind == "ellipsoid":
            disc = bd * bd - dd * (y0 @ y0 - 1.0)
            out += b.rho * 2.0 * np.sqrt(np.maximum(disc, 0.0)) / dd
        else:
            q = y0 @ y0 - bd * bd / dd
            out += b.rho * math.sqrt(2.0 * math.pi) / np.sqrt(dd) * np.exp(-0.5 * q)
    return out


def project_phantom(blobs: Sequence[Blob], orbit: Orbit, det_rows: int, det_cols: int,
                    pitch: float, device: Optional[str] = None,
                    dtype=None) -> "np.ndarray | torch.Tensor":
    """Cone-beam projections g [V,H,W] of the phantom (exact line integrals).

    With device=None the result is an FP64 numpy array; otherwise a torch
    tensor evaluated on `device` in FP64 and cast to `dtype`.
    """
    V = orbit.n_views
    if device is None:
        g = np.zeros((V, det_rows, det_cols))
        for i in range(V):
            g[i] = _line_integrals_np(blobs, orbit.sources[i],
                                      pixel_rays(orbit, i, det_rows, det_cols, pitch))
        return g
    t = torch
    f64 = t.float64
    cu = (det_cols - 1) / 2.0
    cv = (det_rows - 1) / 2.0
    x = (t.arange(det_cols, device=device, dtype=f64) - cu) * pitch
    y = (t.arange(det_rows, device=device, dtype=f64) - cv) * pitch
    lx = t.as_tensor(orbit.lx, device=device, dtype=f64)
    ly = t.as_tensor(orbit.ly, device=device, dtype=f64)
    lz = t.as_tensor(orbit.lz, device=device, dtype=f64)
    a = t.as_tensor(orbit.sources, device=device, dtype=f64)
    out = t.empty((V, det_rows, det_cols), device=device, dtype=dtype or t.float32)
    for i in range(V):
        d = (x[None, :, None] * lx[i] + y[:, None, None] * ly[i] - orbit.sdd * lz[i])
        d = d / t.linalg.norm(d, dim=2, keepdim=True)
        acc = t.zeros((det_rows, det_cols), device=device, dtype=f64)
        for b in blobs:
            T = t.as_tensor((b.rot / b.axes[None, :]).T, device=device, dtype=f64)
            y0 = T @ (a[i] - t.as_tensor(b.center, device=device, dtype=f64))
            dv = d @ T.T
            dd = (dv * dv).sum(-1)
            bd = dv @ y0
            if b.kind == "ellipsoid":
                disc = bd * bd - dd * ((y0 * y0).sum() - 1.0)
                acc += b.rho * 2.0 * t.sqrt(t.clamp(disc, min=0.0)) / dd
            else:
                q = (y0 * y0).sum() - bd * bd / dd
                acc += b.rho * math.sqrt(2.0 * math.pi) / t.sqrt(dd) * t.exp(-0.5 * q)
        out[i] = acc.to(out.dtype)
    return out


def add_poisson_noise(g, photons: float, kappa: float, seed: int):
    """Poisson counts N ~ Poi(photons*exp(-kappa*g)); returns -ln(max(N,1)/photons)/kappa."""
    if torch is not None and isinstance(g, torch.Tensor):
        gen = torch.Generator(device=g.device)
        gen.manual_seed(seed)
        lam = photons * torch.exp(-kappa * g.double())
        n = torch.poisson(lam, generator=gen).clamp_(min=1.0)
        return (-torch.log(n / photons) / kappa).to(g.dtype)
    rng = np.random.default_rng(seed)
    n = np.maximum(rng.poisson(photons * np.exp(-kappa * g)), 1.0)
    return -np.log(n / photons) / kappa


def voxel_centers(shape_zyx, voxel, center=(0.0, 0.0, 0.0)):
    """World coordinates (x, y, z) 1-D arrays of the voxel centres."""
    nz, ny, nx = shape_zyx
    xs = center[0] + (np.arange(nx) - (nx - 1) / 2.0) * voxel[0]
    ys = center[1] + (np.arange(ny) - (ny - 1) / 2.0) * voxel[1]
    zs = center[2] + (np.arange(nz) - (nz - 1) / 2.0) * voxel[2]
    return xs, ys, zs


def phantom_volume(blobs: Sequence[Blob], shape_zyx, voxel, center=(0.0, 0.0, 0.0),
                   supersample: int = 2, device=None):
    """Ground-truth density on the voxel grid [Z,Y,X].

    Ellipsoids are averaged over supersample^3 sub-voxel points; Gaussian
    blobs are evaluated at the voxel centres.  device=None: FP64 numpy;
    otherwise an FP32 torch tensor evaluated (in FP32) on that device.
    """
    if device is not None:
        return _phantom_volume_torch(blobs, shape_zyx, voxel, center, supersample, device)
    nz, ny, nx = shape_zyx
    out = np.zeros((nz, ny, nx))
    xs, ys, zs = voxel_centers(shape_zyx, voxel, center)
    for b in blobs:
        T = (b.rot / b.axes[None, :]).T
        if b.kind == "gauss":
            Z, Y, X = np.meshgrid(zs, ys, xs, indexing="ij")
            pts = np.stack([X - b.center[0], Y - b.center[1], Z - b.center[2]], -1)
            q = np.einsum("ij,zyxj->zyxi", T, pts)
            out += b.rho * np.exp(-0.5 * np.sum(q * q, -1))
            continue
        ss = supersample
        offs = ((np.arange(ss) + 0.5) / ss - 0.5)
        acc = np.zeros_like(out)
        for oz in offs:
            for oy in offs:
                for ox in offs:
                    Z, Y, X = np.meshgrid(zs + oz * voxel[2], ys + oy * voxel[1],
                                          xs + ox * voxel[0], indexing="ij")
                    pts = np.stack([X - b.center[0], Y - b.center[1], Z - b.center[2]], -1)
                    q = np.einsum("ij,zyxj->zyxi", T, pts)
                    acc += (np.sum(q * q, -1) <= 1.0)
        out += b.rho * acc / ss ** 3
    return out


def _phantom_volume_torch(blobs, shape_zyx, voxel, center, ss, device):
    t = torch
    nz, ny, nx = shape_zyx
    xs, ys, zs = (t.as_tensor(a, dtype=t.float32, device=device)
                  for a in voxel_centers(shape_zyx, voxel, center))
    out = t.zeros((nz, ny, nx), dtype=t.float32, device=device)
    offs = [((k + 0.5) / ss - 0.5) for k in range(ss)]
    for b in blobs:
        T = t.as_tensor((b.rot / b.axes[None, :]).T, dtype=t.float32, device=device)
        c = t.as_tensor(b.center, dtype=t.float32, device=device)
        pts = [(0.0, 0.0, 0.0)] if b.kind == "gauss" else \
              [(ox, oy, oz) for oz in offs for oy in offs for ox in offs]
        acc = t.zeros_like(out)
        for (ox, oy, oz) in pts:
            X = (xs + ox * voxel[0] - c[0])[None, None, :]
            Y = (ys + oy * voxel[1] - c[1])[None, :, None]
            Z = (zs + oz * voxel[2] - c[2])[:, None, None]
            q = (T[0, 0] * X + T[0, 1] * Y + T[0, 2] * Z) ** 2 \
                + (T[1, 0] * X + T[1, 1] * Y + T[1, 2] * Z) ** 2 \
                + (T[2, 0] * X + T[2, 1] * Y + T[2, 2] * Z) ** 2
            acc += t.exp(-0.5 * q) if b.kind == "gauss" else (q <= 1.0).float()
        out += b.rho * acc / len(pts)
    return out


# --------------------------------------------------------------------------
# Workload presets
# --------------------------------------------------------------------------
@dataclasses.dataclass
class Workload:
    """Geometry and sizes of one reconstruction problem."""

    name: str
    orbit: Orbit
    det_rows: int
    det_cols: int
    pitch: float
    n_mu: int
    n_s: int
    ds: float
    vol_shape: tuple          # (nz, ny, nx)
    voxel: tuple              # (dx, dy, dz) mm
    vol_center: tuple = (0.0, 0.0, 0.0)
    batch: int = 1
    seed: int = 0
    n_objects: int = 10
    photons: Optional[float] = None

    @property
    def n_views(self) -> int:
        return self.orbit.n_views

    def matrices(self) -> np.ndarray:
        return projection_matrices(self.orbit, self.det_rows, self.det_cols, self.pitch)

    def r_fov(self) -> float:
        return fov_radius(self.det_rows, self.det_cols, self.pitch, self.n_s, self.ds,
                          float(np.linalg.norm(self.orbit.sources[0])), self.orbit.sdd)

    def desc_dict(self) -> dict:
        return dict(n_views=self.n_views, det_rows=self.det_rows, det_cols=self.det_cols,
                    n_mu=self.n_mu, n_s=self.n_s, pitch=self.pitch, ds=self.ds,
                    vol_x=self.vol_shape[2], vol_y=self.vol_shape[1], vol_z=self.vol_shape[0],
                    voxel=tuple(self.voxel), vol_center=tuple(self.vol_center),
                    closed_orbit=int(self.orbit.closed))

    def phantoms(self, kind: str = "ellipsoid") -> List[List[Blob]]:
        """One seeded phantom per batch item (seeds seed, seed+1, ...)."""
        return [random_ellipsoids(np.random.default_rng(self.seed + b), self.n_objects,
                                  self.r_fov(), kind) for b in range(self.batch)]


def _voxel_for(pitch: float, sid: float = SID_MM, sdd: float = SDD_MM) -> float:
    """Voxel size that maps one voxel at the isocentre onto one pixel."""
    return pitch * sid / sdd


def workload(name: str) -> Workload:
    """Named presets of the benchmark configurations (sizes of the paper's workload class)."""
    if name == "circle64":        # plain FP32 circle, small
        o = circle_orbit(64)
        return Workload(name, o, 64, 64, 2.0, 180, 64, 2.0, (64, 64, 64), (2.0, 2.0, 2.0),
                        seed=0, n_objects=10)
    if name == "sinusoid256":     # sinusoid, Poisson noise
        o = sinusoid_orbit(360)
        v = _voxel_for(1.2)
        return Workload(name, o, 256, 256, 1.2, 360, 256, 1.2, (256, 256, 256), (v, v, v),
                        seed=1, n_objects=20, photons=1e5)
    if name == "sinusoid256_train":
        o = sinusoid_orbit(360)
        v = _voxel_for(1.2)
        return Workload(name, o, 256, 256, 1.2, 360, 256, 1.2, (256, 256, 256), (v, v, v),
                        batch=4, seed=2, n_objects=20)
    if name == "circle_arc512":   # circle + arc, 512^3
        o = circle_arc_orbit(360, 136)
        v = _voxel_for(0.6)
        return Workload(name, o, 384, 512, 0.6, 720, 512, 0.6, (512, 512, 512), (v, v, v),
                        seed=6, n_objects=20)
    if name == "paper400":        # the paper's own shape (Tables 1-2)
        o = tilted_sinusoid_orbit(400)
        return Workload(name, o, 480, 620, 0.616, 360, 785, 0.616, (128, 512, 512),
                        (0.25, 0.25, 0.25), seed=7, n_objects=20)
    if name == "paper400_circle":
        o = circle_orbit(400)
        return Workload(name, o, 480, 620, 0.616, 360, 785, 0.616, (128, 512, 512),
                        (0.25, 0.25, 0.25), seed=7, n_objects=20)
    raise KeyError(name)


def batch_workloads(n: int = 12, seed: int = 100, max_views: int = 720,
                    max_det=(480, 616), sizes=(128, 192, 256, 384, 512),
                    min_views: int = 200, min_det: int = 256) -> List[Workload]:
    """Uneven problems for the batched launch: kinds cycle circle, sinusoid,
    circle plus arc; problem k uses seed + k for view count
    U{min_views..max_views}, detector W x H between min_det^2 and max_det
    (multiples of 8, same
    physical width as the 512-column preset), and a cubic volume from `sizes`
    over the same 192 mm field."""
    out = []
    kinds = ["circle", "sinusoid", "circle_arc"]
    for k in range(n):
        rng = np.random.default_rng(seed + k)
        kind = kinds[k % 3]
        V = int(rng.integers(min_views, max_views + 1))
        Wd = int(rng.integers(min_det // 8, max_det[1] // 8 + 1)) * 8
        Hd = int(rng.integers(min_det // 8, min(max_det[0], Wd) // 8 + 1)) * 8
        N = int(rng.choice(sizes))
        pitch = 0.6 * 512 / Wd
        if kind == "circle":
            o = circle_orbit(V)
        elif kind == "sinusoid":
            o = sinusoid_orbit(V)
        else:
            nc = max(2, int(round(V * 360 / 496)))
            o = circle_arc_orbit(nc, max(2, V - nc))
        n_mu = 360 if Wd <= 384 else 720
        vox = 192.0 / N
        out.append(Workload(f"batch{k}_{kind}", o, Hd, Wd, pitch, n_mu, Wd, pitch, (N, N, N),
                            (vox, vox, vox), seed=seed + k, n_objects=20))
    return out


def scaled_workload(name: str, views: Optional[int] = None, det=None, vol=None,
                    n_mu: Optional[int] = None, n_s: Optional[int] = None) -> Workload:
    """A preset with some sizes overridden (for small parity cases)."""
    w = workload(name)
    if views is not None:
        kind = w.orbit.kind
        if kind == "circle":
            w.orbit = circle_orbit(views)
        elif kind == "sinusoid":
            w.orbit = sinusoid_orbit(views)
        elif kind == "circle_arc":
            w.orbit = circle_arc_orbit(max(views * 360 // 496, 2), max(views * 136 // 496, 2))
        elif kind == "tilted_sinusoid":
            w.orbit = tilted_sinusoid_orbit(views)
    if det is not None:
        scale = w.det_cols / det[1]
        w.det_rows, w.det_cols = det
        w.pitch *= scale
        w.ds *= scale
    if n_s is not None:
        w.ds = w.ds * w.n_s / n_s
        w.n_s = n_s
    if n_mu is not None:
        w.n_mu = n_mu
    if vol is not None:
        scale = w.vol_shape[2] / vol[2]
        w.vol_shape = tuple(vol)
        w.voxel = tuple(v * scale for v in w.voxel)
    return w
