"""Python binding of the C ABI in include/dracogb.h (argument marshalling only).

Every function has the name of its C entry point and forwards torch CUDA
tensors as raw device pointers on the current torch stream; all arithmetic
runs in the CUDA library.  Layouts (Ye et al., DRACO, Eq. 12):

    g, g^F : [B, V, H, W]          volume : [B, Z, Y, X]
    W      : [V, n_mu, n_s]        S, R   : [B, V, n_mu, n_s]
"""
from __future__ import annotations

import ctypes
from typing import Optional

import numpy as np
import torch

from . import _lib
from ._lib import (DC_ACCUM, DC_BF16, DC_F16, DC_F32, DC_F32X2, DC_KAHAN, DC_PERSISTENT_FILTER,
                   DC_RELU, check)

# storage forms of g^F: code, torch dtype; "f32x2" holds (value, right
# difference) FP32 pairs in a trailing dimension of 2
_DTYPES = {"f32": (DC_F32, torch.float32), "bf16": (DC_BF16, torch.bfloat16),
           "f16": (DC_F16, torch.float16), "f32x2": (DC_F32X2, torch.float32)}


def gF_shape(geom: "Geometry", B: int, dtype: str = "f32") -> tuple:
    """Shape of g^F in a storage form."""
    shp = (B, geom.V, geom.H, geom.W)
    return shp + (2,) if dtype == "f32x2" else shp


def _gF_code(gF: torch.Tensor) -> int:
    if gF.dtype == torch.float32 and gF.dim() == 5:
        return DC_F32X2
    return {torch.float32: DC_F32, torch.bfloat16: DC_BF16, torch.float16: DC_F16}[gF.dtype]


def _ptr(t: Optional[torch.Tensor]):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


def _stream():
    return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)


def _need(t: torch.Tensor, name: str, dtype, shape):
    if not isinstance(t, torch.Tensor):
        raise TypeError(f"{name} must be a torch.Tensor")
    if not t.is_cuda:
        raise ValueError(f"{name} must be a CUDA tensor")
    if t.dtype != dtype:
        raise ValueError(f"{name} must be {dtype}, got {t.dtype}")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    if tuple(t.shape) != tuple(shape):
        raise ValueError(f"{name} has shape {tuple(t.shape)}, expected {tuple(shape)}")


class Geometry:
    """Owner of a dc_geometry handle (dc_setup_geometry / dc_destroy_geometry)."""

    def __init__(self, desc: dict, P, vdl=None):
        L = _lib.load()
        d = _lib.dc_geometry_desc()
        d.n_views, d.det_rows, d.det_cols = desc["n_views"], desc["det_rows"], desc["det_cols"]
        d.n_mu, d.n_s = desc["n_mu"], desc["n_s"]
        d.pitch, d.ds = desc["pitch"], desc["ds"]
        d.vol_x, d.vol_y, d.vol_z = desc["vol_x"], desc["vol_y"], desc["vol_z"]
        for t in range(3):
            d.voxel[t] = desc["voxel"][t]
            d.vol_center[t] = desc.get("vol_center", (0.0, 0.0, 0.0))[t]
        d.closed_orbit = int(desc.get("closed_orbit", 1))
        self.desc = dict(desc)
        P = np.ascontiguousarray(P, dtype=np.float64)
        if P.size != 12 * d.n_views:
            raise ValueError("P must hold n_views 3x4 matrices")
        v = None if vdl is None else np.ascontiguousarray(vdl, dtype=np.float64)
        if v is not None and v.size != 3 * d.n_views:
            raise ValueError("vdl must hold n_views 3-vectors")
        h = ctypes.c_void_p()
        rc = L.dc_setup_geometry(ctypes.byref(d), P.ctypes.data_as(ctypes.c_void_p),
                                 None if v is None else v.ctypes.data_as(ctypes.c_void_p),
                                 ctypes.byref(h))
        check(rc, "dc_setup_geometry")
        self._h = h
        self._lib = L

    @property
    def handle(self):
        if self._h is None:
            raise RuntimeError("geometry already destroyed")
        return self._h

    def close(self):
        if getattr(self, "_h", None) is not None:
            self._lib.dc_destroy_geometry(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

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

    @property
    def vol_shape(self):
        return (self.desc["vol_z"], self.desc["vol_y"], self.desc["vol_x"])

    @property
    def sino_shape(self):
        return (self.desc["n_mu"], self.desc["n_s"])


def dc_setup_geometry(desc: dict, P, vdl=None) -> Geometry:
    return Geometry(desc, P, vdl)


def dc_destroy_geometry(geom: Geometry):
    geom.close()


def dc_get_view_geometry(geom: Geometry) -> np.ndarray:
    out = np.zeros((geom.V, _lib.DC_VIEW_GEO_N))
    check(_lib.load().dc_get_view_geometry(geom.handle, out.ctypes.data_as(ctypes.c_void_p)),
          "dc_get_view_geometry")
    return out


def dc_filter(geom: Geometry, g: torch.Tensor, W: Optional[torch.Tensor] = None,
              dtype: str = "f32", out: Optional[torch.Tensor] = None,
              scale: Optional[torch.Tensor] = None, S_out: Optional[torch.Tensor] = None):
    """g^F = w_d A2d^T D_b (W K) w_sino D_f A2d w_cos g (Eq. 11).  Returns (g^F, scale).
    With S_out ([B, V, n_mu, n_s]) Grangeat's S is kept there for the reverse mode."""
    B = g.shape[0]
    _need(g, "g", torch.float32, (B, geom.V, geom.H, geom.W))
    if W is not None:
        _need(W, "W", torch.float32, (geom.V,) + geom.sino_shape)
    code, tdt = _DTYPES[dtype]
    if out is None:
        out = torch.empty(gF_shape(geom, B, dtype), device=g.device, dtype=tdt)
    _need(out, "gF", tdt, gF_shape(geom, B, dtype))
    if code == DC_F16 and scale is None:
        scale = torch.empty((B, geom.V), device=g.device, dtype=torch.float32)
    if S_out is not None:
        _need(S_out, "S_out", torch.float32, (B, geom.V) + geom.sino_shape)
        rc = _lib.load().dc_filter_with_s(geom.handle, B, _ptr(g), _ptr(W), _ptr(out), code,
                                          _ptr(scale if code == DC_F16 else None), _ptr(S_out),
                                          _stream())
        check(rc, "dc_filter_with_s")
    else:
        rc = _lib.load().dc_filter(geom.handle, B, _ptr(g), _ptr(W), _ptr(out), code,
                                   _ptr(scale if code == DC_F16 else None), _stream())
        check(rc, "dc_filter")
    return out, (scale if code == DC_F16 else None)


def dc_filter_adjoint(geom: Geometry, grad_gF: torch.Tensor, g: Optional[torch.Tensor],
                      W: Optional[torch.Tensor] = None, want_grad_g: bool = True,
                      want_grad_W: bool = True, view_chunk: int = 0,
                      S: Optional[torch.Tensor] = None):
    """Reverse mode of dc_filter: returns (dL/dg or None, dL/dW or None).
    With S (kept by dc_filter(..., S_out=...)) g is not needed: the line-sum
    pass that recomputes S is skipped."""
    B = grad_gF.shape[0]
    shp = (B, geom.V, geom.H, geom.W)
    _need(grad_gF, "grad_gF", torch.float32, shp)
    if S is not None:
        _need(S, "S", torch.float32, (B, geom.V) + geom.sino_shape)
    else:
        _need(g, "g", torch.float32, shp)
    if W is not None:
        _need(W, "W", torch.float32, (geom.V,) + geom.sino_shape)
    dev = grad_gF.device
    gg = torch.empty(shp, device=dev, dtype=torch.float32) if want_grad_g else None
    gW = (torch.empty((geom.V,) + geom.sino_shape, device=dev, dtype=torch.float32)
          if want_grad_W else None)
    if S is not None:
        rc = _lib.load().dc_filter_adjoint_from_s(geom.handle, B, _ptr(grad_gF), _ptr(S), _ptr(W),
                                                  _ptr(gg), _ptr(gW), int(view_chunk), _stream())
        check(rc, "dc_filter_adjoint_from_s")
    else:
        rc = _lib.load().dc_filter_adjoint(geom.handle, B, _ptr(grad_gF), _ptr(g), _ptr(W),
                                           _ptr(gg), _ptr(gW), int(view_chunk), _stream())
        check(rc, "dc_filter_adjoint")
    return gg, gW


def dc_backproject(geom: Geometry, gF: torch.Tensor, scale: Optional[torch.Tensor] = None,
                   out: Optional[torch.Tensor] = None, accum: bool = False,
                   kahan: bool = False, relu: bool = False) -> torch.Tensor:
    """f = A3d^T g^F (Eq. 5), optional ReLU; g^F in f32, f32x2 ([..., 2] pairs),
    bf16 or f16 (+scale)."""
    B = gF.shape[0]
    code = _gF_code(gF)
    _need(gF, "gF", gF.dtype, (B, geom.V, geom.H, geom.W) + ((2,) if code == DC_F32X2 else ()))
    if code == DC_F16:
        if scale is None:
            raise ValueError("f16 g^F needs its scale")
        _need(scale, "scale", torch.float32, (B, geom.V))
    if out is None:
        if accum:
            raise ValueError("accum needs an output volume")
        out = torch.empty((B,) + geom.vol_shape, device=gF.device, dtype=torch.float32)
    _need(out, "vol", torch.float32, (B,) + geom.vol_shape)
    flags = (DC_ACCUM if accum else 0) | (DC_KAHAN if kahan else 0) | (DC_RELU if relu else 0)
    rc = _lib.load().dc_backproject(geom.handle, B, _ptr(gF), code,
                                    _ptr(scale if code == DC_F16 else None), _ptr(out),
                                    flags, _stream())
    check(rc, "dc_backproject")
    return out


def dc_backproject_adjoint(geom: Geometry, grad_vol: torch.Tensor,
                           relu_vol: Optional[torch.Tensor] = None) -> torch.Tensor:
    """(A3d^T)^T grad_vol -> [B, V, H, W]; masked where relu_vol <= 0 if given."""
    B = grad_vol.shape[0]
    _need(grad_vol, "grad_vol", torch.float32, (B,) + geom.vol_shape)
    if relu_vol is not None:
        _need(relu_vol, "relu_vol", torch.float32, (B,) + geom.vol_shape)
    out = torch.empty((B, geom.V, geom.H, geom.W), device=grad_vol.device, dtype=torch.float32)
    rc = _lib.load().dc_backproject_adjoint(geom.handle, B, _ptr(grad_vol), _ptr(relu_vol),
                                            _ptr(out), _stream())
    check(rc, "dc_backproject_adjoint")
    return out


def dc_grangeat(geom: Geometry, g: torch.Tensor) -> torch.Tensor:
    """S = w_sino D_f A2d w_cos g on the half grid (Eq. 7)."""
    B = g.shape[0]
    _need(g, "g", torch.float32, (B, geom.V, geom.H, geom.W))
    S = torch.empty((B, geom.V) + geom.sino_shape, device=g.device, dtype=torch.float32)
    check(_lib.load().dc_grangeat(geom.handle, B, _ptr(g), _ptr(S), _stream()), "dc_grangeat")
    return S


def dc_radon2d(geom: Geometry, img: torch.Tensor) -> torch.Tensor:
    """Joseph A2d of per-view detector images."""
    B = img.shape[0]
    _need(img, "img", torch.float32, (B, geom.V, geom.H, geom.W))
    R = torch.empty((B, geom.V) + geom.sino_shape, device=img.device, dtype=torch.float32)
    check(_lib.load().dc_radon2d(geom.handle, B, _ptr(img), _ptr(R), _stream()), "dc_radon2d")
    return R


def dc_radon2d_adjoint(geom: Geometry, R: torch.Tensor) -> torch.Tensor:
    """Exact transpose of dc_radon2d."""
    B = R.shape[0]
    _need(R, "R", torch.float32, (B, geom.V) + geom.sino_shape)
    img = torch.empty((B, geom.V, geom.H, geom.W), device=R.device, dtype=torch.float32)
    check(_lib.load().dc_radon2d_adjoint(geom.handle, B, _ptr(R), _ptr(img), _stream()),
          "dc_radon2d_adjoint")
    return img


def dc_crofton_weights(geom: Geometry, segments=None, m: int = 2, taper: int = 5) -> torch.Tensor:
    """Smooth Crofton weights of Eq. 9, [V, n_mu, n_s], usable as W.

    segments: list of (first_view, closed) pieces of the orbit (None: one
    piece, closed as the descriptor says).
    """
    W = torch.empty((geom.V,) + geom.sino_shape, device="cuda", dtype=torch.float32)
    if segments:
        st = (ctypes.c_int * len(segments))(*[int(s[0]) for s in segments])
        cl = (ctypes.c_int * len(segments))(*[int(bool(s[1])) for s in segments])
        n = len(segments)
    else:
        st = cl = None
        n = 0
    check(_lib.load().dc_crofton_weights(geom.handle, n, st, cl, int(m), int(taper), _ptr(W),
                                         _stream()), "dc_crofton_weights")
    return W


def dc_gauss_smooth(W: torch.Tensor, sigma: float = 20.0, radius: int = 60,
                    adjoint: bool = False, out: torch.Tensor = None,
                    work: torch.Tensor = None) -> torch.Tensor:
    """The Gaussian filter layer on the redundancy weight (Sec. 3.1), or its
    transpose: W is [V, n_mu, n_s] FP32 on the GPU."""
    if not isinstance(W, torch.Tensor) or W.dim() != 3:
        raise ValueError("W must be a [V, n_mu, n_s] tensor")
    _need(W, "W", torch.float32, tuple(W.shape))
    out = torch.empty_like(W) if out is None else out
    work = torch.empty_like(W) if work is None else work
    _need(out, "out", torch.float32, tuple(W.shape))
    _need(work, "work", torch.float32, tuple(W.shape))
    V, n_mu, n_s = W.shape
    check(_lib.load().dc_gauss_smooth(V, n_mu, n_s, float(sigma), int(radius),
                                      int(bool(adjoint)), _ptr(W), _ptr(out), _ptr(work),
                                      _stream()), "dc_gauss_smooth")
    return out


def dc_deriv(geom: Geometry, x: torch.Tensor, kind: str = "f") -> torch.Tensor:
    """The s-derivatives alone on [B, V, n_mu, n_s] sinograms: kind "f"
    (D_f), "fT", "b" (D_b) or "bT"."""
    B = x.shape[0]
    _need(x, "x", torch.float32, (B, geom.V) + geom.sino_shape)
    out = torch.empty_like(x)
    code = {"f": 0, "fT": 1, "b": 2, "bT": 3}[kind]
    check(_lib.load().dc_deriv(geom.handle, B, _ptr(x), _ptr(out), code, _stream()), "dc_deriv")
    return out


def dc_sync_status(geom: Geometry):
    """Wait for the current stream; raise if a device-side wait timed out."""
    check(_lib.load().dc_sync_status(geom.handle, _stream()), "dc_sync_status")


def dc_geometry_set_tuning(geom: Geometry, chunk_images: int = 0, bp_nz: int = 0):
    check(_lib.load().dc_geometry_set_tuning(geom.handle, int(chunk_images), int(bp_nz)),
          "dc_geometry_set_tuning")


def dc_geometry_get_tuning(geom: Geometry) -> dict:
    a, c, z = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
    check(_lib.load().dc_geometry_get_tuning(geom.handle, ctypes.byref(a), ctypes.byref(c),
                                             ctypes.byref(z)), "dc_geometry_get_tuning")
    return {"chunk_images": a.value, "chunk_capacity": c.value, "bp_nz": z.value}


class Batch:
    """A batch of reconstruction problems (dc_batch_create / dc_batch_run).

    run() filters every problem and backprojects all of them with one
    persistent kernel; it allocates nothing, so it can be captured in a CUDA
    graph (capture()) and replayed (replay()).
    """

    def __init__(self, geoms, dtype: str = "f32", kahan: bool = False, relu: bool = False,
                 persistent_filter: bool = False):
        L = _lib.load()
        self.geoms = list(geoms)
        arr = (ctypes.c_void_p * len(self.geoms))(*[g.handle for g in self.geoms])
        flags = ((DC_KAHAN if kahan else 0) | (DC_RELU if relu else 0)
                 | (DC_PERSISTENT_FILTER if persistent_filter else 0))
        h = ctypes.c_void_p()
        check(L.dc_batch_create(len(self.geoms), arr, _DTYPES[dtype][0], flags, ctypes.byref(h)),
              "dc_batch_create")
        self._h = h
        self._lib = L
        self.graph = None

    def set_bp_nz(self, nz: int):
        check(self._lib.dc_batch_set_bp_nz(self._h, int(nz)), "dc_batch_set_bp_nz")

    def run(self, g_list, vol_list, W_list=None):
        n = len(self.geoms)
        for i, (geom, g, v) in enumerate(zip(self.geoms, g_list, vol_list)):
            _need(g, f"g[{i}]", torch.float32, (geom.V, geom.H, geom.W))
            _need(v, f"vol[{i}]", torch.float32, geom.vol_shape)
        gp = (ctypes.c_void_p * n)(*[t.data_ptr() for t in g_list])
        vp = (ctypes.c_void_p * n)(*[t.data_ptr() for t in vol_list])
        wp = None
        if W_list is not None:
            wp = (ctypes.c_void_p * n)(*[0 if t is None else t.data_ptr() for t in W_list])
        check(self._lib.dc_batch_run(self._h, gp, wp, vp, _stream()), "dc_batch_run")

    def capture(self, g_list, vol_list, W_list=None):
        """Record one run into a CUDA graph (after one eager run, which sets
        the kernels' shared-memory attributes outside the capture)."""
        self.run(g_list, vol_list, W_list)
        torch.cuda.synchronize()
        self.graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(self.graph):
            self.run(g_list, vol_list, W_list)
        return self.graph

    def replay(self):
        self.graph.replay()

    def close(self):
        if getattr(self, "_h", None) is not None:
            self.graph = None
            self._lib.dc_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def reconstruct(geom: Geometry, g: torch.Tensor, W: Optional[torch.Tensor] = None,
                dtype: str = "f32", kahan: bool = False, relu: bool = False) -> torch.Tensor:
    """Eq. 12: f = A3d^T w_d A2d^T D w_red w_sino D A2d w_cos g."""
    gF, sc = dc_filter(geom, g, W, dtype)
    return dc_backproject(geom, gF, sc, kahan=kahan, relu=relu)


def dc_reconstruct_host(geom: Geometry, g_host: torch.Tensor, vol_host: torch.Tensor,
                        W: Optional[torch.Tensor] = None, dtype: str = "f32",
                        kahan: bool = False, relu: bool = False, n_slabs: int = 0,
                        g_dev: Optional[torch.Tensor] = None, gF: Optional[torch.Tensor] = None,
                        scale: Optional[torch.Tensor] = None,
                        vol_dev: Optional[torch.Tensor] = None, device="cuda") -> torch.Tensor:
    """Eq. 12 from host projections [B, V, H, W] into the host volume
    [B, Z, Y, X], the transfers overlapped with the kernels (pin both host
    tensors for the overlap).  Device buffers are made when not given."""
    if g_host.is_cuda or vol_host.is_cuda:
        raise ValueError("g_host and vol_host must be host tensors")
    B = g_host.shape[0]
    shp = (B, geom.V, geom.H, geom.W)
    for t, name, s in ((g_host, "g_host", shp), (vol_host, "vol_host", (B,) + geom.vol_shape)):
        if t.dtype != torch.float32 or not t.is_contiguous() or tuple(t.shape) != s:
            raise ValueError(f"{name} must be contiguous float32 of shape {s}")
    code, tdt = _DTYPES[dtype]
    if W is not None:
        _need(W, "W", torch.float32, (geom.V,) + geom.sino_shape)
    g_dev = torch.empty(shp, device=device, dtype=torch.float32) if g_dev is None else g_dev
    gF = torch.empty(gF_shape(geom, B, dtype), device=device, dtype=tdt) if gF is None else gF
    vol_dev = torch.empty((B,) + geom.vol_shape, device=device) if vol_dev is None else vol_dev
    if code == DC_F16 and scale is None:
        scale = torch.empty((B, geom.V), device=device, dtype=torch.float32)
    _need(g_dev, "g_dev", torch.float32, shp)
    _need(gF, "gF", tdt, gF_shape(geom, B, dtype))
    _need(vol_dev, "vol_dev", torch.float32, (B,) + geom.vol_shape)
    flags = (DC_KAHAN if kahan else 0) | (DC_RELU if relu else 0)
    check(_lib.load().dc_reconstruct_host(geom.handle, B, g_host.data_ptr(), _ptr(W), _ptr(g_dev),
                                          _ptr(gF), code,
                                          _ptr(scale if code == DC_F16 else None), _ptr(vol_dev),
                                          vol_host.data_ptr(), flags, int(n_slabs), _stream()),
          "dc_reconstruct_host")
    return vol_host
