"""Projection of a scalar pixel field onto a mesh -- the oracle of
mesh_project (test infrastructure, used only by the tests, the smoke check
and the benchmark's CPU baseline).

Wraps ``oracle/sbmt_project.c``: per triangle the mean of the
piecewise-constant pixel field over the triangle (clipping against each
pixel square, Sec. 3.3's projection of the bitmap's scalar fields onto each
triangle), per vertex the bilinear interpolation between pixel centres.
Both in double precision, one plain loop each.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "sbmt_project.c")
_LIB = os.path.join(_HERE, "_build", "libproject.so")
_lib = None


def build(force: bool = False) -> str:
    os.makedirs(os.path.dirname(_LIB), exist_ok=True)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + ".tmp.%d" % os.getpid()
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-shared", "-fPIC", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build())
        lib.sbmt_oracle_tri_box_area.restype = ctypes.c_double
        lib.sbmt_oracle_tri_box_area.argtypes = [ctypes.c_void_p] + [ctypes.c_double] * 4
        lib.sbmt_oracle_project_triangles.restype = None
        lib.sbmt_oracle_project_triangles.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64,
                                                      ctypes.c_void_p, ctypes.c_int, ctypes.c_int, ctypes.c_void_p]
        lib.sbmt_oracle_vertex_values.restype = None
        lib.sbmt_oracle_vertex_values.argtypes = [ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p, ctypes.c_int,
                                                  ctypes.c_int, ctypes.c_void_p]
        _lib = lib
    return _lib


def _field(f) -> np.ndarray:
    f = np.ascontiguousarray(np.asarray(f, dtype=np.float32))
    if f.ndim != 2:
        raise ValueError("the field must be a 2-D array")
    return f


def tri_box_area(tri_xy, x0, x1, y0, y1) -> float:
    """Area of a triangle (3 x 2 points) inside the box [x0, x1] x [y0, y1]."""
    t = np.ascontiguousarray(np.asarray(tri_xy, dtype=np.float64).reshape(6))
    return _load().sbmt_oracle_tri_box_area(t.ctypes.data, x0, x1, y0, y1)


def project_triangles(xy, tri, field) -> np.ndarray:
    """Mean of the pixel field over each triangle (0 outside the image)."""
    f = _field(field)
    xy = np.ascontiguousarray(np.asarray(xy, dtype=np.float64))
    tri = np.ascontiguousarray(np.asarray(tri, dtype=np.int32))
    out = np.zeros(len(tri), dtype=np.float64)
    _load().sbmt_oracle_project_triangles(xy.ctypes.data, tri.ctypes.data, len(tri), f.ctypes.data, f.shape[1],
                                          f.shape[0], out.ctypes.data)
    return out


def vertex_values(xy, field) -> np.ndarray:
    """Bilinear interpolation of the pixel field at each vertex (clamped)."""
    f = _field(field)
    xy = np.ascontiguousarray(np.asarray(xy, dtype=np.float64))
    out = np.zeros(len(xy), dtype=np.float64)
    _load().sbmt_oracle_vertex_values(xy.ctypes.data, len(xy), f.ctypes.data, f.shape[1], f.shape[0],
                                      out.ctypes.data)
    return out
