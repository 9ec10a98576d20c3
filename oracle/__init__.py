"""CPU oracle for the SBMT hot path -- TEST INFRASTRUCTURE ONLY.

This package wraps ``oracle/sbmt_oracle.cpp``, a plain single-threaded exact
CPU statement of the method (boundary extraction, base grid, Alg. 1 events,
frozen registry, canonical key and App. G lookup, Tier-G greedy rule,
labels).  Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s
cpu_baseline / reference leg may import it; the product path never does, and
it shares no code with the CUDA library.

Functions whose parity is pinned by the paper (see the tests): ``alg1``
(single-segment atoms of Fig. "lookup_table"), ``line_meet`` (App. F printed
intersection points), ``local_patch`` / ``template`` (App. G triangle lists).
The Tier-G greedy rule (``greedy``) has no counterpart in the paper; it is
pinned only by invariants and brute force ("parity unpinned" by the paper).
``region3`` (Region III of Alg. 3's schedule: Alg. 2 on the preprocessed
mesh) is pinned by reproducing the plain mesh on the unmoved base mesh, by
the invariants of an embedding, and by hand-built degenerate cells against
App. G and Fig. "lookup_table".
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "sbmt_oracle.cpp")
_OUT_DIR = os.path.join(_HERE, "_build")
_LIB = os.path.join(_OUT_DIR, "liboracle.so")


def build(force: bool = False) -> str:
    """Compile the oracle shared library (g++ -O2) if missing or stale.  No
    floating-point contraction: every product and sum is rounded on its own,
    as written, on every host (GCC fuses them by default for C++ on Arm)."""
    os.makedirs(_OUT_DIR, exist_ok=True)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + ".tmp.%d" % os.getpid()
        subprocess.check_call(["g++", "-O2", "-std=c++17", "-ffp-contract=off", "-shared", "-fPIC", "-o", tmp, _SRC])
        os.replace(tmp, _LIB)
    return _LIB


class _Mesh(ctypes.Structure):
    _fields_ = [
        ("n_vertices", ctypes.c_int64),
        ("n_triangles", ctypes.c_int64),
        ("n_cells", ctypes.c_int64),
        ("n_cut_cells", ctypes.c_int64),
        ("n_tierG_cells", ctypes.c_int64),
        ("n_vertices_grid", ctypes.c_int64),
        ("xy", ctypes.POINTER(ctypes.c_double)),
        ("tri", ctypes.POINTER(ctypes.c_int32)),
        ("label", ctypes.POINTER(ctypes.c_uint16)),
        ("code", ctypes.POINTER(ctypes.c_uint16)),
        ("n_segments", ctypes.c_int64),
        ("seg", ctypes.POINTER(ctypes.c_int32)),
        ("n_events", ctypes.c_int64),
        ("ev", ctypes.POINTER(ctypes.c_int64)),
        ("cut", ctypes.POINTER(ctypes.c_int64)),
    ]


_lib = None


def _load():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build())
        lib.oracle_mesh_bitmap.restype = ctypes.c_int
        lib.oracle_mesh_bitmap.argtypes = [ctypes.c_void_p, ctypes.c_int32, ctypes.c_int32, ctypes.c_int64,
                                           ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32,
                                           ctypes.c_int32, ctypes.POINTER(_Mesh)]
        lib.oracle_mesh_free.argtypes = [ctypes.POINTER(_Mesh)]
        lib.oracle_last_error.restype = ctypes.c_char_p
        lib.oracle_alg1.restype = ctypes.c_int
        lib.oracle_alg1.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]
        lib.oracle_line_meet.restype = ctypes.c_int
        lib.oracle_line_meet.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]
        lib.oracle_local_patch.restype = ctypes.c_int
        lib.oracle_local_patch.argtypes = [ctypes.c_void_p, ctypes.c_int32, ctypes.c_void_p, ctypes.c_int32,
                                           ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int32]
        lib.oracle_template.restype = ctypes.c_int
        lib.oracle_template.argtypes = [ctypes.c_int32, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int32]
        lib.oracle_base_mesh.restype = ctypes.c_int
        lib.oracle_base_mesh.argtypes = [ctypes.c_int32] * 6 + [ctypes.POINTER(ctypes.c_int64)] * 2 + [
            ctypes.POINTER(ctypes.POINTER(ctypes.c_double)), ctypes.POINTER(ctypes.POINTER(ctypes.c_int32))]
        lib.oracle_free.argtypes = [ctypes.c_void_p]
        lib.oracle_check_mesh.restype = ctypes.c_int
        lib.oracle_check_mesh.argtypes = [ctypes.c_void_p] + [ctypes.c_int32] * 4 + [ctypes.c_int64] * 2 + [
            ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p, ctypes.c_void_p]
        lib.oracle_brute.restype = ctypes.c_int64
        lib.oracle_brute.argtypes = [ctypes.c_int32] * 4 + [ctypes.c_int64] * 2
        lib.oracle_region3.restype = ctypes.c_int
        lib.oracle_region3.argtypes = [ctypes.c_void_p, ctypes.c_int32, ctypes.c_int32, ctypes.c_int64,
                                       ctypes.c_int32, ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p,
                                       ctypes.c_int64, ctypes.c_int32, ctypes.POINTER(_Mesh)]
        lib.oracle_brute_general.restype = ctypes.c_int64
        lib.oracle_brute_general.argtypes = [ctypes.c_int32] * 6 + [ctypes.c_int64] * 2
        lib.oracle_greedy.restype = ctypes.c_int
        lib.oracle_greedy.argtypes = [ctypes.c_void_p, ctypes.c_int32, ctypes.c_void_p, ctypes.c_int32,
                                      ctypes.c_void_p, ctypes.c_int32]
        _lib = lib
    return _lib


class OracleError(RuntimeError):
    pass


def _copy(ptr, n, dtype):
    if n == 0:
        return np.zeros(0, dtype=dtype)
    return np.ctypeslib.as_array(ptr, shape=(n,)).astype(dtype, copy=True)


def mesh_bitmap(img: np.ndarray, h_num: int, h_den: int = 1, origin2x: int = 0, origin2y: int = 0) -> dict:
    """Mesh a 2-D uint8/uint16 label image (row y = image row).  Returns numpy
    arrays: xy (V,2) f64, tri (T,3) i32 CCW, label (T,) u16 (0xFFFF outside the
    image), code (T,) u16, seg (n,7), ev (n,3), cut (n,5) and counts."""
    lib = _load()
    img = np.ascontiguousarray(img)
    if img.ndim != 2 or img.dtype not in (np.uint8, np.uint16):
        raise ValueError("img must be a 2-D uint8 or uint16 array")
    H, W = img.shape
    m = _Mesh()
    rc = lib.oracle_mesh_bitmap(img.ctypes.data, W, H, img.strides[0], img.dtype.itemsize, h_num, h_den,
                                origin2x, origin2y, ctypes.byref(m))
    if rc != 0:
        raise OracleError("oracle_mesh_bitmap failed (%d): %s" % (rc, lib.oracle_last_error().decode()))
    try:
        out = dict(
            n_vertices=m.n_vertices, n_triangles=m.n_triangles, n_cells=m.n_cells, n_cut_cells=m.n_cut_cells,
            n_tierG_cells=m.n_tierG_cells, n_vertices_grid=m.n_vertices_grid,
            xy=_copy(m.xy, 2 * m.n_vertices, np.float64).reshape(-1, 2),
            tri=_copy(m.tri, 3 * m.n_triangles, np.int32).reshape(-1, 3),
            label=_copy(m.label, m.n_triangles, np.uint16),
            code=_copy(m.code, m.n_triangles, np.uint16),
            seg=_copy(m.seg, 7 * m.n_segments, np.int32).reshape(-1, 7),
            ev=_copy(m.ev, 3 * m.n_events, np.int64).reshape(-1, 3),
            cut=_copy(m.cut, 5 * m.n_cut_cells, np.int64).reshape(-1, 5),
        )
    finally:
        lib.oracle_mesh_free(ctypes.byref(m))
    return out


def _pts(points) -> np.ndarray:
    """Points as (x, x_sqrt3, y, y_sqrt3) integer quadruples: x + x_sqrt3*sqrt(3)."""
    a = np.ascontiguousarray(np.asarray(points, dtype=np.int64).reshape(-1, 4))
    return a


def alg1(tri, seg):
    """Alg. 1 for triangle ``tri`` (3 points, CCW) and segment ``seg`` (2
    points).  Returns (kinds for AB, BC, CA; bitmask AB=2, BC=4, CA=8)."""
    lib = _load()
    t, s = _pts(tri), _pts(seg)
    kinds = np.zeros(3, dtype=np.int32)
    mask = lib.oracle_alg1(t.ctypes.data, s.ctypes.data, kinds.ctypes.data)
    return kinds, mask


def line_meet(pq, uv):
    """Intersection point of lines PQ and UV (same units as the inputs)."""
    lib = _load()
    a, b = _pts(pq), _pts(uv)
    out = np.zeros(2, dtype=np.float64)
    ok = lib.oracle_line_meet(a.ctypes.data, b.ctypes.data, out.ctypes.data)
    return out if ok else None


def local_patch(nev, nchain, ce):
    """Key and Tier-T patch of a cell from its combinatorial description.
    Returns dict(key, sigma, klass, mask, tierG, tri (n,3) local indices)."""
    lib = _load()
    nev = np.ascontiguousarray(np.asarray(nev, dtype=np.int32))
    ce = np.ascontiguousarray(np.asarray(ce, dtype=np.int32).reshape(-1, 2))
    info = np.zeros(5, dtype=np.int32)
    cap = 64
    tri = np.zeros(3 * cap, dtype=np.int32)
    n = lib.oracle_local_patch(nev.ctypes.data, nchain, ce.ctypes.data, ce.shape[0], info.ctypes.data,
                               tri.ctypes.data, cap)
    if n < 0:
        raise OracleError(lib.oracle_last_error().decode())
    return dict(key=int(info[0]), sigma=int(info[1]), klass=int(info[2]), mask=int(info[3]),
                tierG=int(info[4]), tri=tri[: 3 * n].reshape(-1, 3).copy())


def template(key: int):
    """(canonical code, template label triples) of a Tier-T key, or None."""
    lib = _load()
    code = ctypes.c_int32(0)
    tri = np.zeros(3 * 64, dtype=np.int32)
    n = lib.oracle_template(key, ctypes.byref(code), tri.ctypes.data, 64)
    if n <= 0:
        return None
    return int(code.value), tri[: 3 * n].reshape(-1, 3).copy()


def greedy(points, constraints):
    """Tier-G greedy triangulation of explicit points with constraint edges."""
    lib = _load()
    p = _pts(points)
    c = np.ascontiguousarray(np.asarray(constraints, dtype=np.int32).reshape(-1, 2))
    cap = 4 * p.shape[0] + 8
    tri = np.zeros(3 * cap, dtype=np.int32)
    n = lib.oracle_greedy(p.ctypes.data, p.shape[0], c.ctypes.data, c.shape[0], tri.ctypes.data, cap)
    if n < 0:
        raise OracleError("greedy failed")
    return tri[: 3 * n].reshape(-1, 3).copy()


def base_mesh(width: int, height: int, h_num: int, h_den: int = 1, origin2x: int = 0, origin2y: int = 0):
    """The base mesh T0 (Sec. 3.3): lattice vertex coordinates (V, 2) in
    vertex-id order and the cells' corners A, B, C (C, 3) in cell-id order."""
    lib = _load()
    nv, nc = ctypes.c_int64(0), ctypes.c_int64(0)
    xy = ctypes.POINTER(ctypes.c_double)()
    tri = ctypes.POINTER(ctypes.c_int32)()
    rc = lib.oracle_base_mesh(width, height, h_num, h_den, origin2x, origin2y, ctypes.byref(nv), ctypes.byref(nc),
                              ctypes.byref(xy), ctypes.byref(tri))
    if rc != 0:
        raise OracleError("oracle_base_mesh failed (%d): %s" % (rc, lib.oracle_last_error().decode()))
    try:
        return (_copy(xy, 2 * nv.value, np.float64).reshape(-1, 2), _copy(tri, 3 * nc.value, np.int32).reshape(-1, 3))
    finally:
        lib.oracle_free(ctypes.cast(xy, ctypes.c_void_p))
        lib.oracle_free(ctypes.cast(tri, ctypes.c_void_p))


def brute(width: int, height: int, h_num: int, h_den: int = 1, first: int = 0, stride: int = 1) -> int:
    """Mesh every binary width x height bitmap (bit k of its number = pixel k,
    row-major; from `first`, every `stride`-th) at h = h_num / h_den and check
    each mesh against the invariants of any correct output (orientation,
    closure, Euler characteristic, exact total and per-label areas, boundary
    conformity).  Returns the number checked; raises on the first failure."""
    r = _load().oracle_brute(width, height, h_num, h_den, first, stride)
    if r < 0:
        raise OracleError(_load().oracle_last_error().decode())
    return r


def check_mesh(img: np.ndarray, h_num: int, h_den: int, mesh: dict) -> int:
    """The invariants of brute() for one mesh of a binary bitmap: 0, or the
    number of the failed check (the message in last_error())."""
    lib = _load()
    img = np.ascontiguousarray(img, dtype=np.uint8)
    xy = np.ascontiguousarray(mesh["xy"], dtype=np.float64)
    tri = np.ascontiguousarray(mesh["tri"], dtype=np.int32)
    lab = np.ascontiguousarray(mesh["label"], dtype=np.uint16)
    return lib.oracle_check_mesh(img.ctypes.data, img.shape[1], img.shape[0], h_num, h_den, mesh["n_cells"],
                                 len(xy), xy.ctypes.data, len(tri), tri.ctypes.data, lab.ctypes.data)


def region3(img: np.ndarray, xy: np.ndarray, tri: np.ndarray, plant: int = 0) -> dict:
    """Region III of Alg. 3's schedule: Alg. 2 (the template retriangulation)
    of the counter-clockwise triangle mesh (xy (V, 2) f64, tri (C, 3)) against
    the image's boundary, each cell on its own.  Returns the embedded mesh as
    mesh_bitmap does (xy, tri, label, code and counts; n_events, n_inside).
    plant != 0 plants one of the oracle's test mistakes."""
    lib = _load()
    img = np.ascontiguousarray(img)
    if img.ndim != 2 or img.dtype not in (np.uint8, np.uint16):
        raise ValueError("img must be a 2-D uint8 or uint16 array")
    H, W = img.shape
    xy = np.ascontiguousarray(xy, dtype=np.float64)
    tri = np.ascontiguousarray(tri, dtype=np.int32)
    m = _Mesh()
    rc = lib.oracle_region3(img.ctypes.data, W, H, img.strides[0], img.dtype.itemsize, xy.ctypes.data, len(xy),
                            tri.ctypes.data, len(tri), plant, ctypes.byref(m))
    if rc != 0:
        raise OracleError("oracle_region3 failed (%d): %s" % (rc, lib.oracle_last_error().decode()))
    try:
        out = dict(
            n_vertices=m.n_vertices, n_triangles=m.n_triangles, n_cells=m.n_cells, n_cut_cells=m.n_cut_cells,
            n_tierG_cells=m.n_tierG_cells, n_vertices_grid=m.n_vertices_grid, n_events=m.n_events,
            n_inside=m.n_vertices - m.n_vertices_grid - m.n_events,
            xy=_copy(m.xy, 2 * m.n_vertices, np.float64).reshape(-1, 2),
            tri=_copy(m.tri, 3 * m.n_triangles, np.int32).reshape(-1, 3),
            label=_copy(m.label, m.n_triangles, np.uint16),
            code=_copy(m.code, m.n_triangles, np.uint16),
        )
    finally:
        lib.oracle_mesh_free(ctypes.byref(m))
    return out


def mesh_general(img: np.ndarray, h_num: int, h_den: int = 1, origin2x: int = 0, origin2y: int = 0) -> dict:
    """The general path, for any integer origin (an odd origin2x / origin2y
    puts the lattice on pixel lines): the base mesh, then Region III."""
    H, W = img.shape
    xy0, cells = base_mesh(W, H, h_num, h_den, origin2x, origin2y)
    out = region3(img, xy0, cells)
    out["base_xy"], out["base_tri"] = xy0, cells
    return out


def brute_general(width: int, height: int, h_num: int, h_den: int = 1, origin2x: int = -1, origin2y: int = -1,
                  first: int = 0, stride: int = 1) -> int:
    """brute() for the general path at the given origin: every binary bitmap
    (from first, every stride-th) meshed as mesh_general does and checked
    against the invariants.  Returns the number checked; raises on a failure."""
    r = _load().oracle_brute_general(width, height, h_num, h_den, origin2x, origin2y, first, stride)
    if r < 0:
        raise OracleError(_load().oracle_last_error().decode())
    return r


def last_error() -> str:
    return _load().oracle_last_error().decode()
