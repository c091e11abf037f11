"""The C-ABI library builds for sm_103a, loads without a GPU and exports every
entry point include/dracogb.h declares; host-side argument checks work."""
import ctypes
import os
import re

import pytest

from paper_2410_14900_gb300 import build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "dracogb.h")


def declared_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(dc_[a-z0-9_]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    return ctypes.CDLL(build.build())


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("dc_setup_geometry", "dc_destroy_geometry", "dc_filter",
                     "dc_filter_adjoint", "dc_backproject", "dc_backproject_adjoint"):
        assert required in names


def test_library_exports_every_declared_symbol(lib):
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_argument_errors_without_a_gpu(lib):
    from paper_2410_14900_gb300 import _lib as L
    h = L.load()
    out = ctypes.c_void_p()
    assert h.dc_setup_geometry(None, None, None, ctypes.byref(out)) == L.DC_ERR_ARG
    assert b"NULL" in h.dc_last_error()
    d = L.dc_geometry_desc()
    d.n_views = 0
    P = (ctypes.c_double * 12)()
    assert h.dc_setup_geometry(ctypes.byref(d), P, None, ctypes.byref(out)) == L.DC_ERR_ARG
    d.n_views, d.det_rows, d.det_cols, d.n_mu, d.n_s = 1, 8, 8, 4, 8
    d.vol_x = d.vol_y = d.vol_z = 4
    d.pitch, d.ds = 1.0, 1.0
    d.voxel[0] = d.voxel[1] = d.voxel[2] = 1.0
    P[0] = float("nan")
    assert h.dc_setup_geometry(ctypes.byref(d), P, None, ctypes.byref(out)) == L.DC_ERR_ARG
    assert b"non-finite" in h.dc_last_error()
    for f in ("dc_filter", "dc_backproject", "dc_grangeat", "dc_radon2d"):
        assert getattr(h, f)  # resolvable
    assert h.dc_filter(None, 1, None, None, None, 0, None, None) == L.DC_ERR_ARG
    assert h.dc_backproject(None, 1, None, 0, None, None, 0, None) == L.DC_ERR_ARG
    assert h.dc_backproject_adjoint(None, 1, None, None, None, None) == L.DC_ERR_ARG
    assert h.dc_filter_adjoint(None, 1, None, None, None, None, None, 0, None) == L.DC_ERR_ARG
    assert h.dc_sync_status(None, None) == L.DC_ERR_ARG
    for code in range(6):
        assert h.dc_status_string(code).startswith(b"DC_")
    h.dc_destroy_geometry(None)  # NULL is ignored


def test_no_cpu_fallback_when_library_is_missing(tmp_path, monkeypatch):
    """The binding raises instead of computing anything on the CPU."""
    from paper_2410_14900_gb300 import _lib as L
    monkeypatch.setattr(L, "_lib", None)
    monkeypatch.setattr(L._build, "LIB", str(tmp_path / "absent.so"))
    with pytest.raises(RuntimeError, match="missing"):
        L.load()
