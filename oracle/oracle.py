"""FP64 CPU oracle of the Defrise-Clack filtered backprojection (numpy API).

TEST INFRASTRUCTURE ONLY: imported by the tests, by the smoke check and by
the CPU-baseline leg of the benchmark; never by the product path.  The
arithmetic lives in dc_oracle.c (plain C, FP64); this module only builds it
with gcc and marshals numpy arrays.  It shares no code with the CUDA library.

Section/equation references are to Ye et al., "DRACO: Differentiable
Reconstruction for Arbitrary CBCT Orbits" (arXiv 2410.14900).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "dc_oracle.c")
_LIB = os.path.join(_HERE, "libdc_oracle.so")
_lock = threading.Lock()
_lib = None

GEO_N = 32
G_P, G_A, G_LX, G_LY, G_LZ, G_D, G_CU, G_CV, G_V = 0, 12, 15, 18, 21, 24, 25, 26, 27


def build(force: bool = False) -> str:
    """Compile dc_oracle.c into libdc_oracle.so next to it (gcc, OpenMP)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-fopenmp", "-shared", "-fPIC", _SRC,
                               "-o", tmp, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def lib():
    global _lib
    with _lock:
        if _lib is None:
            _lib = ctypes.CDLL(build())
    return _lib


_D = ctypes.POINTER(ctypes.c_double)


def _p(a):
    return None if a is None else a.ctypes.data_as(_D)


def _f64(a):
    return None if a is None else np.ascontiguousarray(a, dtype=np.float64)


def num_threads() -> int:
    return int(lib().orc_num_threads())


class Geometry:
    """Per-view geometry recovered from the projection matrices (Fig. 1)."""

    def __init__(self, desc: dict, P: np.ndarray, vdl=None):
        self.desc = dict(desc)
        V = desc["n_views"]
        P = _f64(np.asarray(P).reshape(V, 12))
        ctr = _f64(np.asarray(desc.get("vol_center", (0.0, 0.0, 0.0))))
        self.geo = np.zeros((V, GEO_N))
        rc = lib().orc_setup_geometry(ctypes.c_int(V), ctypes.c_double(desc["pitch"]),
                                      _p(ctr), _p(P), _p(_f64(vdl)),
                                      ctypes.c_int(int(desc.get("closed_orbit", 1))),
                                      _p(self.geo))
        if rc != 0:
            raise ValueError("projection matrix is singular, skewed or has non-square pixels")

    # convenient views of the record
    def source(self, i):
        return self.geo[i, G_A:G_A + 3]

    def frame(self, i):
        g = self.geo[i]
        return g[G_LX:G_LX + 3], g[G_LY:G_LY + 3], g[G_LZ:G_LZ + 3]

    def D(self, i):
        return self.geo[i, G_D]

    def principal_point(self, i):
        return self.geo[i, G_CU], self.geo[i, G_CV]

    def tangent(self, i):
        return self.geo[i, G_V:G_V + 3]

    def matrix(self, i):
        return self.geo[i, G_P:G_P + 12].reshape(3, 4)

    # sizes
    @property
    def V(self):
        return self.desc["n_views"]

    @property
    def H(self):
        return self.desc["det_rows"]

    @property
    def W(self):
        return self.desc["det_cols"]


def _ci(x):
    return ctypes.c_int(int(x))


def _cd(x):
    return ctypes.c_double(float(x))


# ---------------------------------------------------------------- per view
def cosine_weight(geom: Geometry, i: int, g: np.ndarray) -> np.ndarray:
    """w_cos * g for view i (Eq. 7)."""
    d = geom.desc
    g = _f64(g)
    out = np.empty_like(g)
    lib().orc_cosine_weight(_ci(d["det_rows"]), _ci(d["det_cols"]), _cd(d["pitch"]),
                            _p(geom.geo[i]), _p(g), _p(out))
    return out


def detector_weight(geom: Geometry, i: int, h: np.ndarray) -> np.ndarray:
    """w_d * h for view i (Eq. 11)."""
    d = geom.desc
    h = _f64(h)
    out = np.empty_like(h)
    lib().orc_detector_weight(_ci(d["det_rows"]), _ci(d["det_cols"]), _cd(d["pitch"]),
                              _p(geom.geo[i]), _p(h), _p(out))
    return out


def radon(img: np.ndarray, pitch: float, n_mu: int, n_s: int, ds: float,
          cu=None, cv=None) -> np.ndarray:
    """Joseph A2d of an [H,W] image -> [n_mu, n_s] line sums (Eq. 7)."""
    img = _f64(img)
    H, W = img.shape
    cu = (W - 1) / 2.0 if cu is None else cu
    cv = (H - 1) / 2.0 if cv is None else cv
    R = np.empty((n_mu, n_s))
    lib().orc_radon(_ci(H), _ci(W), _cd(pitch), _cd(cu), _cd(cv), _ci(n_mu), _ci(n_s),
                    _cd(ds), _p(img), _p(R))
    return R


def radon_T(R: np.ndarray, H: int, W: int, pitch: float, ds: float,
            cu=None, cv=None) -> np.ndarray:
    """Literal transpose of `radon` (no scale)."""
    R = _f64(R)
    n_mu, n_s = R.shape
    cu = (W - 1) / 2.0 if cu is None else cu
    cv = (H - 1) / 2.0 if cv is None else cv
    img = np.zeros((H, W))
    lib().orc_radon_T(_ci(H), _ci(W), _cd(pitch), _cd(cu), _cd(cv), _ci(n_mu), _ci(n_s),
                      _cd(ds), _p(R), _p(img))
    return img


def _deriv(name, x, ds):
    x = _f64(x)
    out = np.empty_like(x)
    getattr(lib(), name)(_ci(x.shape[0]), _ci(x.shape[1]), _cd(ds), _p(x), _p(out))
    return out


def deriv_f(R, ds):
    return _deriv("orc_deriv_f", R, ds)


def deriv_f_T(y, ds):
    return _deriv("orc_deriv_f_T", y, ds)


def deriv_b(Q, ds):
    return _deriv("orc_deriv_b", Q, ds)


def deriv_b_T(y, ds):
    return _deriv("orc_deriv_b_T", y, ds)


def redundancy_K(geom: Geometry, i: int) -> np.ndarray:
    """K = -(1/4pi^2)|v.theta|/sqrt(s^2+D^2) on the half grid (Eq. 10)."""
    d = geom.desc
    out = np.empty((d["n_mu"], d["n_s"]))
    lib().orc_redundancy_K(_ci(d["n_mu"]), _ci(d["n_s"]), _cd(d["ds"]), _p(geom.geo[i]),
                           _p(out))
    return out


def grangeat(geom: Geometry, i: int, g: np.ndarray) -> np.ndarray:
    """S = w_sino D_f A2d w_cos g for view i, on s_{k+1/2} (Eq. 7)."""
    d = geom.desc
    S = np.empty((d["n_mu"], d["n_s"]))
    lib().orc_grangeat(_ci(d["det_rows"]), _ci(d["det_cols"]), _cd(d["pitch"]),
                       _ci(d["n_mu"]), _ci(d["n_s"]), _cd(d["ds"]), _p(geom.geo[i]),
                       _p(_f64(g)), _p(S))
    return S


# ------------------------------------------------------------ whole operators
def filter(geom: Geometry, g: np.ndarray, Wred=None, views=None) -> np.ndarray:
    """g^F = w_d A2d^T D_b w_red S (Eq. 11) for g [B][nv][H][W].

    `views` selects which views of the geometry the nv input images belong to
    (default: all, in order).  Wred [V][n_mu][n_s] or None (=1/2).
    """
    d = geom.desc
    g = _f64(g)
    if g.ndim == 3:
        g = g[None]
    B, nv = g.shape[:2]
    vsel = None if views is None else np.ascontiguousarray(views, dtype=np.int32)
    out = np.empty_like(g)
    lib().orc_filter(_ci(B), _ci(nv),
                     None if vsel is None else vsel.ctypes.data_as(ctypes.POINTER(ctypes.c_int)),
                     _ci(d["det_rows"]), _ci(d["det_cols"]), _cd(d["pitch"]), _ci(d["n_mu"]),
                     _ci(d["n_s"]), _cd(d["ds"]), _p(geom.geo), _p(g), _p(_f64(Wred)), _p(out))
    return out


def filter_adjoint(geom: Geometry, g: np.ndarray, G: np.ndarray, Wred=None,
                   want_grad_g=True, want_grad_W=True):
    """Reverse mode of `filter`: returns (dL/dg, dL/dW) for dL/dg^F = G."""
    d = geom.desc
    g = _f64(g)
    G = _f64(G)
    if g.ndim == 3:
        g, G = g[None], G[None]
    B, V = g.shape[:2]
    gg = np.empty_like(g) if want_grad_g else None
    gW = np.empty((V, d["n_mu"], d["n_s"])) if want_grad_W else None
    lib().orc_filter_adjoint(_ci(B), _ci(V), _ci(d["det_rows"]), _ci(d["det_cols"]),
                             _cd(d["pitch"]), _ci(d["n_mu"]), _ci(d["n_s"]), _cd(d["ds"]),
                             _p(geom.geo), _p(g), _p(_f64(Wred)), _p(G), _p(gg), _p(gW))
    return gg, gW


def _vol_args(d):
    vox = _f64(np.asarray(d["voxel"], dtype=np.float64))
    ctr = _f64(np.asarray(d.get("vol_center", (0.0, 0.0, 0.0)), dtype=np.float64))
    return vox, ctr


def backproject(geom: Geometry, gF: np.ndarray, relu=False, vol=None) -> np.ndarray:
    """f = A3d^T g^F (Eq. 5), [B][Z][Y][X]; adds into `vol` if given."""
    d = geom.desc
    gF = _f64(gF)
    if gF.ndim == 3:
        gF = gF[None]
    B = gF.shape[0]
    nx, ny, nz = d["vol_x"], d["vol_y"], d["vol_z"]
    accum = vol is not None
    out = _f64(vol).copy() if accum else np.empty((B, nz, ny, nx))
    vox, ctr = _vol_args(d)
    lib().orc_backproject(_ci(B), _ci(d["n_views"]), _ci(d["det_rows"]), _ci(d["det_cols"]),
                          _ci(nx), _ci(ny), _ci(nz), _p(vox), _p(ctr), _p(geom.geo), _p(gF),
                          _ci(accum), _ci(relu), _p(out))
    return out


def backproject_points(geom: Geometry, gF: np.ndarray, flat_idx: np.ndarray,
                       relu=False) -> np.ndarray:
    """A3d^T g^F at selected flat voxel indices of one volume (gF [V][H][W])."""
    d = geom.desc
    gF = _f64(gF)
    idx = np.ascontiguousarray(flat_idx, dtype=np.int64)
    out = np.empty(idx.shape[0])
    vox, ctr = _vol_args(d)
    lib().orc_backproject_points(_ci(d["n_views"]), _ci(d["det_rows"]), _ci(d["det_cols"]),
                                 _ci(d["vol_x"]), _ci(d["vol_y"]), _ci(d["vol_z"]), _p(vox),
                                 _p(ctr), _p(geom.geo), _p(gF), _ci(idx.shape[0]),
                                 idx.ctypes.data_as(ctypes.POINTER(ctypes.c_long)),
                                 _ci(relu), _p(out))
    return out


def backproject_adjoint(geom: Geometry, grad_vol: np.ndarray) -> np.ndarray:
    """(A3d^T)^T grad_vol -> [B][V][H][W]."""
    d = geom.desc
    gv = _f64(grad_vol)
    if gv.ndim == 3:
        gv = gv[None]
    B = gv.shape[0]
    out = np.empty((B, d["n_views"], d["det_rows"], d["det_cols"]))
    vox, ctr = _vol_args(d)
    lib().orc_backproject_adjoint(_ci(B), _ci(d["n_views"]), _ci(d["det_rows"]),
                                  _ci(d["det_cols"]), _ci(d["vol_x"]), _ci(d["vol_y"]),
                                  _ci(d["vol_z"]), _p(vox), _p(ctr), _p(geom.geo), _p(gv),
                                  _p(out))
    return out


def crofton_weights(geom: Geometry, segments=None, m: int = 2, taper: int = 5) -> np.ndarray:
    """Smooth Crofton weights of Eq. 9 for every (view, mu, s_{k+1/2}).

    segments: list of (first_view, closed) for the orbit's pieces (default:
    one piece, closed as the descriptor says).
    """
    d = geom.desc
    V = d["n_views"]
    if segments is None:
        segments = [(0, bool(d.get("closed_orbit", 1)))]
    st = np.ascontiguousarray([s[0] for s in segments], dtype=np.int32)
    cl = np.ascontiguousarray([int(bool(s[1])) for s in segments], dtype=np.int32)
    out = np.empty((V, d["n_mu"], d["n_s"]))
    IP = ctypes.POINTER(ctypes.c_int)
    lib().orc_crofton_weights(_ci(V), _ci(d["n_mu"]), _ci(d["n_s"]), _cd(d["ds"]), _p(geom.geo),
                              _ci(len(segments)), st.ctypes.data_as(IP), cl.ctypes.data_as(IP),
                              _ci(m), _ci(taper), _p(out))
    return out


def gauss_smooth(W: np.ndarray, sigma: float = 20.0, radius: int = 60,
                 adjoint: bool = False) -> np.ndarray:
    """The Gaussian filter layer on the redundancy weight (Sec. 3.1): per
    view, separable along mu and s over the valid entries k < n_s - 1, unit-sum
    taps, mirror ends.  adjoint=True applies the transpose."""
    W = np.ascontiguousarray(W, dtype=np.float64)
    V, n_mu, n_s = W.shape
    out = np.empty_like(W)
    lib().orc_gauss_smooth(_ci(V), _ci(n_mu), _ci(n_s), _cd(sigma), _ci(radius),
                           _ci(int(bool(adjoint))), _p(W), _p(out))
    return out


def reconstruct(geom: Geometry, g: np.ndarray, Wred=None, relu=False) -> np.ndarray:
    """Eq. 12: f = A3d^T w_d A2d^T D w_red w_sino D A2d w_cos g."""
    return backproject(geom, filter(geom, g, Wred), relu=relu)
