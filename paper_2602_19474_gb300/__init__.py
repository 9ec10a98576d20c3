"""GB300 (sm_103a) implementation of the data-parallel hot path of Structured
Bitmap-to-Mesh Triangulation (arXiv 2602.19474).

This module is a thin ctypes binding of the C interface in include/sbmt.h
(same names: mesh_create, mesh_bitmap, mesh_batch, mesh_query, mesh_release,
mesh_destroy, mesh_stage).  It only marshals arguments: every step of the
meshing runs in the CUDA kernels of libsbmt.so.  There is no CPU fallback;
loading fails with an error if the library has not been built.

PyTorch is used for device buffers: images may be passed as CUDA tensors,
and finished meshes are exposed as zero-copy CUDA tensors.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from ._build import LIB as _LIB_PATH
from ._build import build as build_library

SBMT_OK = 0
SBMT_EINVAL = -1
SBMT_ENOMEM = -2
SBMT_EPENDING = -3
SBMT_ETIMEDOUT = -4
SBMT_ECAPACITY = -5
SBMT_EPROTO = -6
SBMT_ECUDA = -7
SBMT_EINTERNAL = -8
SBMT_ENOENT = -9
SBMT_ECANCELED = -10
SBMT_U8, SBMT_U16, SBMT_F32 = 1, 2, 4
SBMT_PLAIN, SBMT_PREPROCESS = 0, 1
SBMT_EXPLICIT, SBMT_COMPACT = 0, 1
SBMT_KEEP_STAGES = 1
SBMT_DEBUG_STALL_SCAN = 2

EXPORTS = ("mesh_create", "mesh_bitmap", "mesh_batch", "mesh_autotune", "mesh_tuning", "mesh_set_tuning",
           "mesh_query", "mesh_release", "mesh_destroy", "mesh_stage", "mesh_profile", "mesh_profile_read", "mesh_quality", "mesh_project",
           "mesh_preprocess", "mesh_preprocess_info", "mesh_retriangulate", "mesh_import", "mesh_heat", "mesh_check", "mesh_footprint", "mesh_bound", "server_create",
           "server_submit", "server_wait", "server_cancel", "server_release", "server_stats", "server_destroy",
           "sbmt_last_error", "sbmt_server_last_error")


class sbmt_image(ctypes.Structure):
    _fields_ = [("width", ctypes.c_int32), ("height", ctypes.c_int32), ("pitch_bytes", ctypes.c_int64),
                ("dtype", ctypes.c_int32), ("data", ctypes.c_void_p), ("on_device", ctypes.c_int32)]


class sbmt_params(ctypes.Structure):
    _fields_ = [("h_num", ctypes.c_int32), ("h_den", ctypes.c_int32), ("origin2x", ctypes.c_int32),
                ("origin2y", ctypes.c_int32), ("mode", ctypes.c_int32), ("a", ctypes.c_double),
                ("b", ctypes.c_double), ("c", ctypes.c_double), ("format", ctypes.c_int32),
                ("flags", ctypes.c_int32)]


class sbmt_mesh_view(ctypes.Structure):
    _fields_ = [("n_vertices", ctypes.c_int64), ("n_triangles", ctypes.c_int64), ("n_cells", ctypes.c_int64),
                ("n_cut_cells", ctypes.c_int64), ("n_tierG_cells", ctypes.c_int64), ("n_segments", ctypes.c_int64),
                ("n_events", ctypes.c_int64), ("n_inside_vertices", ctypes.c_int64),
                ("n_lattice_vertices", ctypes.c_int64), ("n_tierG_triangles", ctypes.c_int64), ("xy", ctypes.c_void_p),
                ("tri", ctypes.c_void_p), ("label", ctypes.c_void_p), ("code", ctypes.c_void_p),
                ("status", ctypes.c_int32), ("format", ctypes.c_int32), ("n_patch_triangles", ctypes.c_int64),
                ("cell_label", ctypes.c_void_p), ("cell_code", ctypes.c_void_p), ("patch_cell", ctypes.c_void_p),
                ("patch_off", ctypes.c_void_p)]


class sbmt_quality(ctypes.Structure):
    _fields_ = [("triangles", ctypes.c_int64), ("min_angle_deg", ctypes.c_double), ("min_area", ctypes.c_double),
                ("slivers", ctypes.c_int64), ("equilateral", ctypes.c_int64), ("area_mean", ctypes.c_double),
                ("area_var", ctypes.c_double), ("ar_median", ctypes.c_double), ("ar_p95", ctypes.c_double),
                ("ar_max", ctypes.c_double), ("angle_hist", ctypes.c_int64 * 30)]


class sbmt_pre_info(ctypes.Structure):
    _fields_ = [("n_lattice_vertices", ctypes.c_int64), ("n_points", ctypes.c_int64), ("n_snapped", ctypes.c_int64),
                ("n_repelled", ctypes.c_int64), ("n_candidate_points", ctypes.c_int64),
                ("n_eliminated", ctypes.c_int64), ("n_split_cells", ctypes.c_int64), ("a_px", ctypes.c_double),
                ("b_px", ctypes.c_double), ("c_px", ctypes.c_double), ("status", ctypes.c_void_p),
                ("snap", ctypes.c_void_p), ("elim", ctypes.c_void_p)]


class sbmt_heat_params(ctypes.Structure):
    _fields_ = [("label", ctypes.c_int32), ("alpha", ctypes.c_double), ("dt", ctypes.c_double),
                ("steps", ctypes.c_int32), ("x0", ctypes.c_double), ("y0", ctypes.c_double),
                ("sigma", ctypes.c_double), ("amplitude", ctypes.c_double), ("tol", ctypes.c_double),
                ("max_iterations", ctypes.c_int32)]


class sbmt_server_config(ctypes.Structure):
    _fields_ = [("hbm_budget", ctypes.c_size_t), ("max_batch", ctypes.c_int32), ("workers", ctypes.c_int32),
                ("oom_every", ctypes.c_int32)]


class sbmt_request_info(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int32), ("batch_size", ctypes.c_int32), ("queued_ms", ctypes.c_double),
                ("total_ms", ctypes.c_double)]


class sbmt_server_stats(ctypes.Structure):
    _fields_ = [("submitted", ctypes.c_int64), ("completed", ctypes.c_int64), ("failed", ctypes.c_int64),
                ("cancelled", ctypes.c_int64), ("batches", ctypes.c_int64), ("queued", ctypes.c_int64),
                ("reserved_bytes", ctypes.c_int64), ("peak_reserved_bytes", ctypes.c_int64),
                ("budget_bytes", ctypes.c_int64)]


class SbmtError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__("sbmt error %d: %s" % (code, msg))
        self.code = code


_lib = None


def library_path() -> str:
    return _LIB_PATH


def load(path: str | None = None) -> ctypes.CDLL:
    """Load libsbmt.so (built in-tree by build_library())."""
    global _lib
    if _lib is not None:
        return _lib
    path = path or _LIB_PATH
    if not os.path.exists(path):
        raise RuntimeError("libsbmt.so is not built (%s); run paper_2602_19474_gb300.build_library()" % path)
    lib = ctypes.CDLL(path)
    vp, i32, i64 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64
    lib.mesh_create.argtypes = [ctypes.POINTER(vp), ctypes.c_int, ctypes.c_size_t, vp]
    lib.mesh_bitmap.argtypes = [vp, ctypes.POINTER(sbmt_image), ctypes.POINTER(sbmt_params),
                                ctypes.POINTER(ctypes.c_uint64)]
    lib.mesh_batch.argtypes = [vp, ctypes.POINTER(sbmt_image), ctypes.c_int, ctypes.POINTER(sbmt_params),
                               ctypes.c_int, ctypes.POINTER(ctypes.c_uint64)]
    lib.mesh_autotune.argtypes = [vp, ctypes.POINTER(sbmt_image), ctypes.c_int, ctypes.POINTER(sbmt_params),
                                  ctypes.c_int, ctypes.c_int]
    lib.mesh_tuning.argtypes = [vp, ctypes.POINTER(sbmt_image), ctypes.c_int, ctypes.POINTER(sbmt_params),
                                ctypes.c_int, ctypes.POINTER(ctypes.c_int32)]
    lib.mesh_set_tuning.argtypes = [vp, ctypes.POINTER(sbmt_image), ctypes.c_int, ctypes.POINTER(sbmt_params),
                                    ctypes.c_int, ctypes.POINTER(ctypes.c_int32)]
    lib.mesh_query.argtypes = [vp, ctypes.c_uint64, ctypes.c_int, ctypes.POINTER(sbmt_mesh_view)]
    lib.mesh_release.argtypes = [vp, ctypes.c_uint64]
    lib.mesh_destroy.argtypes = [vp]
    lib.mesh_stage.argtypes = [vp, ctypes.c_uint64, ctypes.c_int, vp, i64, ctypes.POINTER(i64)]
    lib.mesh_profile.argtypes = [vp, ctypes.c_int]
    lib.mesh_profile_read.argtypes = [vp, ctypes.c_int, ctypes.c_int, ctypes.POINTER(ctypes.c_char_p),
                                      ctypes.POINTER(ctypes.c_double), ctypes.POINTER(i64),
                                      ctypes.POINTER(ctypes.c_int)]
    lib.mesh_quality.argtypes = [vp, ctypes.c_uint64, ctypes.POINTER(sbmt_quality)]
    lib.mesh_project.argtypes = [vp, ctypes.c_uint64, ctypes.POINTER(sbmt_image), vp, vp]
    lib.mesh_preprocess.argtypes = [vp, ctypes.POINTER(sbmt_image), ctypes.POINTER(sbmt_params),
                                    ctypes.POINTER(ctypes.c_uint64)]
    lib.mesh_preprocess_info.argtypes = [vp, ctypes.c_uint64, ctypes.POINTER(sbmt_pre_info)]
    lib.mesh_retriangulate.argtypes = [vp, ctypes.POINTER(sbmt_image), ctypes.c_uint64, ctypes.POINTER(ctypes.c_uint64)]
    lib.mesh_import.argtypes = [vp, vp, ctypes.c_int64, vp, ctypes.c_int64, ctypes.POINTER(ctypes.c_uint64)]
    lib.mesh_heat.argtypes = [vp, ctypes.c_uint64, ctypes.POINTER(sbmt_heat_params), vp, vp, vp]
    lib.mesh_check.argtypes = [ctypes.POINTER(sbmt_image), ctypes.POINTER(sbmt_params)]
    lib.mesh_footprint.argtypes = [vp, ctypes.c_uint64, ctypes.POINTER(ctypes.c_size_t)]
    lib.mesh_bound.argtypes = [ctypes.POINTER(sbmt_image), ctypes.POINTER(sbmt_params), ctypes.POINTER(ctypes.c_size_t)]
    lib.server_create.argtypes = [ctypes.POINTER(vp), ctypes.c_int, ctypes.POINTER(sbmt_server_config)]
    lib.server_submit.argtypes = [vp, ctypes.POINTER(sbmt_image), ctypes.POINTER(sbmt_params),
                                  ctypes.POINTER(ctypes.c_uint64)]
    lib.server_wait.argtypes = [vp, ctypes.c_uint64, ctypes.c_int, ctypes.POINTER(sbmt_mesh_view),
                                ctypes.POINTER(sbmt_request_info)]
    lib.server_cancel.argtypes = [vp, ctypes.c_uint64]
    lib.server_release.argtypes = [vp, ctypes.c_uint64]
    lib.server_stats.argtypes = [vp, ctypes.POINTER(sbmt_server_stats)]
    lib.server_destroy.argtypes = [vp]
    for f in ("mesh_check", "mesh_footprint", "mesh_bound", "mesh_retriangulate", "mesh_import", "server_create", "server_submit", "server_wait", "server_cancel",
              "server_release", "server_stats", "server_destroy"):
        getattr(lib, f).restype = ctypes.c_int
    lib.sbmt_server_last_error.restype = ctypes.c_char_p
    lib.sbmt_last_error.restype = ctypes.c_char_p
    for f in ("mesh_create", "mesh_bitmap", "mesh_batch", "mesh_autotune", "mesh_tuning", "mesh_set_tuning",
              "mesh_query", "mesh_release", "mesh_destroy",
              "mesh_stage", "mesh_profile", "mesh_profile_read", "mesh_quality", "mesh_project", "mesh_preprocess",
              "mesh_preprocess_info", "mesh_heat"):
        getattr(lib, f).restype = ctypes.c_int
    del i32
    _lib = lib
    return lib


def _check(rc: int):
    if rc != SBMT_OK:
        raise SbmtError(rc, load().sbmt_last_error().decode())


def _image(img) -> tuple[sbmt_image, object]:
    """sbmt_image for a numpy array (host) or a CUDA tensor (device); returns
    the struct and the object that keeps the memory alive."""
    if isinstance(img, np.ndarray):
        a = np.ascontiguousarray(img)
        if a.ndim != 2 or a.dtype not in (np.uint8, np.uint16):
            raise ValueError("image must be a 2-D uint8 or uint16 array")
        return sbmt_image(a.shape[1], a.shape[0], a.strides[0], a.itemsize, a.ctypes.data, 0), a
    import torch

    t = img
    if not (isinstance(t, torch.Tensor) and t.is_cuda and t.dim() == 2 and t.dtype in (torch.uint8, torch.int16)
            or isinstance(t, torch.Tensor) and t.is_cuda and t.dim() == 2 and str(t.dtype) == "torch.uint16"):
        raise ValueError("device image must be a 2-D CUDA tensor of uint8 or 16-bit integers")
    if t.stride(1) != 1:
        t = t.contiguous()
    item = t.element_size()
    return sbmt_image(t.shape[1], t.shape[0], t.stride(0) * item, item, t.data_ptr(), 1), t


def _params(h_num: int, h_den: int = 1, origin2x: int = 0, origin2y: int = 0, keep_stages: bool = False,
            mode: int = SBMT_PLAIN, format: int = SBMT_EXPLICIT) -> sbmt_params:
    return sbmt_params(h_num, h_den, origin2x, origin2y, mode, 0.0, 0.0, 0.0, format,
                       SBMT_KEEP_STAGES if keep_stages else 0)


# ---------------------------------------------------------------------------
# C-ABI names
# ---------------------------------------------------------------------------
def mesh_create(device: int = 0, pool_bytes: int = 0, stream: int | None = None) -> int:
    ctx = ctypes.c_void_p()
    _check(load().mesh_create(ctypes.byref(ctx), device, pool_bytes, stream))
    return ctx.value


def mesh_bitmap(ctx: int, img, h_num: int, h_den: int = 1, origin2x: int = 0, origin2y: int = 0,
                keep_stages: bool = False, mode: int = SBMT_PLAIN, format: int = SBMT_EXPLICIT, flags: int = 0) -> int:
    im, keep = _image(img)
    pr = _params(h_num, h_den, origin2x, origin2y, keep_stages, mode, format)
    pr.flags |= flags
    out = ctypes.c_uint64()
    _check(load().mesh_bitmap(ctx, ctypes.byref(im), ctypes.byref(pr), ctypes.byref(out)))
    del keep
    return out.value


def mesh_preprocess(ctx: int, img, h_num: int, h_den: int = 1, a: float = 0.26, b: float = 0.125, c: float = 0.183,
                    origin2x: int = 0, origin2y: int = 0) -> int:
    """Alg. 3's preprocessed mesh of one image (thresholds relative to the
    reference edge sqrt(0.45) px); a handle for mesh_query and
    mesh_preprocess_info."""
    im, keep = _image(img)
    pr = sbmt_params(h_num, h_den, origin2x, origin2y, SBMT_PREPROCESS, float(a), float(b), float(c), SBMT_EXPLICIT, 0)
    out = ctypes.c_uint64()
    _check(load().mesh_preprocess(ctx, ctypes.byref(im), ctypes.byref(pr), ctypes.byref(out)))
    del keep
    return out.value


def mesh_preprocessed(ctx: int, img, h_num: int, h_den: int = 1, a: float = 0.26, b: float = 0.125, c: float = 0.183,
                      origin2x: int = 0, origin2y: int = 0) -> int:
    """Alg. 3 in full through mesh_bitmap (mode SBMT_PREPROCESS): Regions
    I-II, then Region III on the preprocessed mesh; the embedded mesh."""
    im, keep = _image(img)
    pr = sbmt_params(h_num, h_den, origin2x, origin2y, SBMT_PREPROCESS, float(a), float(b), float(c), SBMT_EXPLICIT, 0)
    out = ctypes.c_uint64()
    _check(load().mesh_bitmap(ctx, ctypes.byref(im), ctypes.byref(pr), ctypes.byref(out)))
    del keep
    return out.value


def mesh_retriangulate(ctx: int, img, base: int) -> int:
    """Region III: Alg. 2 on the explicit mesh `base` against img's boundary."""
    im, keep = _image(img)
    out = ctypes.c_uint64()
    _check(load().mesh_retriangulate(ctx, ctypes.byref(im), base, ctypes.byref(out)))
    del keep
    return out.value


def mesh_import(ctx: int, xy, tri) -> int:
    """An explicit mesh handle from host arrays xy (n, 2) and tri (m, 3)."""
    xy = np.ascontiguousarray(xy, dtype=np.float64).reshape(-1, 2)
    tri = np.ascontiguousarray(tri, dtype=np.int32).reshape(-1, 3)
    out = ctypes.c_uint64()
    _check(load().mesh_import(ctx, xy.ctypes.data, len(xy), tri.ctypes.data, len(tri), ctypes.byref(out)))
    return out.value


def mesh_preprocess_info(ctx: int, mesh: int) -> sbmt_pre_info:
    v = sbmt_pre_info()
    _check(load().mesh_preprocess_info(ctx, mesh, ctypes.byref(v)))
    return v


def pre_info_numpy(info: sbmt_pre_info) -> dict:
    """Host copies of a preprocessed mesh's records (status, snap, elim)."""
    import torch

    def dev(ptr, shape, typestr):
        return torch.as_tensor(_CudaArray(ptr, shape, typestr, None), device="cuda").cpu().numpy()

    V, E = info.n_lattice_vertices, info.n_eliminated
    return {
        "status": dev(info.status, (V,), "|u1") if V else np.zeros(0, np.uint8),
        "snap": dev(info.snap, (V,), "<i4") if V else np.zeros(0, np.int32),
        "elim": dev(info.elim, (E, 3), "<i4") if E else np.zeros((0, 3), np.int32),
        "n_points": info.n_points, "n_snapped": info.n_snapped, "n_repelled": info.n_repelled,
        "n_candidate_points": info.n_candidate_points, "n_split_cells": info.n_split_cells,
        "thresholds_px": (info.a_px, info.b_px, info.c_px),
    }


def _batch_args(imgs, h_num, h_den, keep_stages=False, format=SBMT_EXPLICIT, flags=0):
    n = len(imgs)
    ims, keeps = zip(*[_image(i) for i in imgs]) if n else ((), ())
    arr = (sbmt_image * max(n, 1))(*ims)
    hn = list(h_num) if isinstance(h_num, (list, tuple, np.ndarray)) else [h_num]
    hd = list(h_den) if isinstance(h_den, (list, tuple, np.ndarray)) else [h_den] * len(hn)
    prs = (sbmt_params * len(hn))(*[_params(int(a), int(b), keep_stages=keep_stages, format=format)
                                       for a, b in zip(hn, hd)])
    for p in prs:
        p.flags |= flags
    return n, arr, prs, len(hn), keeps


def mesh_batch(ctx: int, imgs, h_num, h_den=1, keep_stages: bool = False, format: int = SBMT_EXPLICIT,
               flags: int = 0) -> list[int]:
    n, arr, prs, npr, keeps = _batch_args(imgs, h_num, h_den, keep_stages, format, flags)
    out = (ctypes.c_uint64 * max(n, 1))()
    _check(load().mesh_batch(ctx, arr, n, prs, npr, out))
    del keeps
    return [out[k] for k in range(n)]


def mesh_autotune(ctx: int, imgs, h_num, h_den=1, repeats: int = 2) -> None:
    """Tune the batched path for the size class of this batch (persists to
    the tuning file); the meshes it makes are released."""
    n, arr, prs, npr, keeps = _batch_args(imgs, h_num, h_den)
    _check(load().mesh_autotune(ctx, arr, n, prs, npr, repeats))
    del keeps


def mesh_tuning(ctx: int, imgs, h_num, h_den=1) -> dict:
    """The launch parameters mesh_batch uses for this batch."""
    n, arr, prs, npr, keeps = _batch_args(imgs, h_num, h_den)
    o = (ctypes.c_int32 * 4)()
    _check(load().mesh_tuning(ctx, arr, n, prs, npr, o))
    del keeps
    return {"cut_blocks_per_sm": o[0], "tierg_blocks_per_sm": o[1], "fork": o[2], "graph": o[3]}


def mesh_set_tuning(ctx: int, imgs, h_num, h_den=1, cut_blocks_per_sm: int = 8, tierg_blocks_per_sm: int = 24,
                    fork: int = 1, graph: int = 0) -> None:
    """Set the launch parameters of this batch's size class (this context only)."""
    n, arr, prs, npr, keeps = _batch_args(imgs, h_num, h_den)
    v = (ctypes.c_int32 * 4)(cut_blocks_per_sm, tierg_blocks_per_sm, fork, graph)
    _check(load().mesh_set_tuning(ctx, arr, n, prs, npr, v))
    del keeps


def mesh_query(ctx: int, mesh: int, wait_ms: int = -1) -> sbmt_mesh_view:
    v = sbmt_mesh_view()
    rc = load().mesh_query(ctx, mesh, wait_ms, ctypes.byref(v))
    if rc in (SBMT_EPENDING, SBMT_ETIMEDOUT):
        return None
    _check(rc)
    return v


def mesh_release(ctx: int, mesh: int) -> None:
    _check(load().mesh_release(ctx, mesh))


def mesh_destroy(ctx: int) -> None:
    _check(load().mesh_destroy(ctx))


def mesh_stage(ctx: int, mesh: int, stage: int) -> np.ndarray:
    width = {1: (8, np.int32), 2: (4, np.int64), 3: (5, np.int64), 4: (1, np.int64)}[stage]
    n = ctypes.c_int64(0)
    _check(load().mesh_stage(ctx, mesh, stage, None, 0, ctypes.byref(n)))
    buf = np.zeros((max(n.value, 1), width[0]), dtype=width[1])
    _check(load().mesh_stage(ctx, mesh, stage, buf.ctypes.data, n.value, ctypes.byref(n)))
    return buf[: min(n.value, 1024) if stage == 4 else n.value]


def mesh_quality(ctx: int, mesh: int) -> dict:
    """Quality measures of a finished mesh, computed on the device."""
    q = sbmt_quality()
    _check(load().mesh_quality(ctx, mesh, ctypes.byref(q)))
    out = {k: getattr(q, k) for k, _ in sbmt_quality._fields_ if k != "angle_hist"}
    out["angle_hist"] = [int(x) for x in q.angle_hist]
    return out


def _field(field) -> tuple[sbmt_image, object]:
    """sbmt_image (SBMT_F32) for a float32 numpy array or CUDA tensor."""
    if isinstance(field, np.ndarray):
        a = np.ascontiguousarray(field, dtype=np.float32)
        if a.ndim != 2:
            raise ValueError("the field must be 2-D")
        return sbmt_image(a.shape[1], a.shape[0], a.strides[0], SBMT_F32, a.ctypes.data, 0), a
    import torch

    t = field
    if not (isinstance(t, torch.Tensor) and t.is_cuda and t.dim() == 2 and t.dtype == torch.float32):
        raise ValueError("a device field must be a 2-D float32 CUDA tensor")
    if t.stride(1) != 1:
        t = t.contiguous()
    return sbmt_image(t.shape[1], t.shape[0], t.stride(0) * 4, SBMT_F32, t.data_ptr(), 1), t


def mesh_project(ctx: int, mesh: int, field, tri_value=None, vertex_value=None) -> None:
    """Project a float32 pixel field onto a finished mesh: per-triangle means
    into ``tri_value`` and bilinear vertex values into ``vertex_value`` (float32
    CUDA tensors of n_triangles / n_vertices elements, or None).  Enqueued on
    the context's stream; mesh_query on the mesh waits for it."""
    fi, keep = _field(field)

    def ptr(t):
        if t is None:
            return None
        if not (t.is_cuda and t.dtype.itemsize == 4 and t.is_contiguous()):
            raise ValueError("outputs must be contiguous float32 CUDA tensors")
        return t.data_ptr()

    _check(load().mesh_project(ctx, mesh, ctypes.byref(fi), ptr(tri_value), ptr(vertex_value)))
    del keep


def mesh_heat(ctx: int, mesh: int, label: int, alpha: float, dt: float, steps: int, x0: float, y0: float,
              sigma: float, amplitude: float = 100.0, tol: float = 1e-10, max_iterations: int = 10000, u=None):
    """Heat diffusion on the triangles of one label (App. H); returns (u as a
    CUDA float64 tensor over the mesh's vertices, peaks per step, CG
    iterations per step)."""
    import torch

    v = mesh_query(ctx, mesh, -1)
    if u is None:
        u = torch.empty(v.n_vertices, dtype=torch.float64, device="cuda")
    pr = sbmt_heat_params(label, alpha, dt, steps, x0, y0, sigma, amplitude, tol, max_iterations)
    peaks = (ctypes.c_double * max(steps, 1))()
    its = (ctypes.c_int32 * max(steps, 1))()
    _check(load().mesh_heat(ctx, mesh, ctypes.byref(pr), ctypes.c_void_p(u.data_ptr()), peaks, its))
    return u, [peaks[k] for k in range(steps)], [its[k] for k in range(steps)]


def mesh_profile(ctx: int, enable: bool) -> None:
    _check(load().mesh_profile(ctx, 1 if enable else 0))


def mesh_profile_read(ctx: int, reset: bool = False) -> dict:
    """{kernel name: (milliseconds, launches)} accumulated while tracing."""
    cap = 32
    names = (ctypes.c_char_p * cap)()
    ms = (ctypes.c_double * cap)()
    cnt = (ctypes.c_int64 * cap)()
    n = ctypes.c_int(0)
    _check(load().mesh_profile_read(ctx, 1 if reset else 0, cap, names, ms, cnt, ctypes.byref(n)))
    return {names[k].decode(): (ms[k], cnt[k]) for k in range(min(n.value, cap))}


# ---------------------------------------------------------------------------
# device views of a finished mesh
# ---------------------------------------------------------------------------
class _CudaArray:
    """__cuda_array_interface__ wrapper so torch can view library memory."""

    def __init__(self, ptr: int, shape, typestr: str, owner):
        self.__cuda_array_interface__ = {"shape": tuple(shape), "typestr": typestr, "data": (ptr, False),
                                         "version": 3, "strides": None}
        self._owner = owner


def view_tensors(view: sbmt_mesh_view, owner=None) -> dict:
    """Zero-copy torch CUDA tensors of a finished mesh (valid until release)."""
    import torch

    def dev(ptr, shape, typestr):
        return torch.as_tensor(_CudaArray(ptr, shape, typestr, owner), device="cuda")

    if view.format == SBMT_COMPACT:
        V, T, C, K = view.n_vertices - view.n_lattice_vertices, view.n_patch_triangles, view.n_cells, view.n_cut_cells
        return {
            "xy": dev(view.xy, (V, 2), "<f8"),
            "tri": dev(view.tri, (T, 3), "<i4"),
            "label": dev(view.label, (T,), "<i2"),
            "code": dev(view.code, (T,), "<i2"),
            "cell_label": dev(view.cell_label, (C,), "<i2"),
            "cell_code": dev(view.cell_code, (C,), "<i2"),
            "patch_cell": dev(view.patch_cell, (K,), "<i4"),
            "patch_off": dev(view.patch_off, (K + 1,), "<i4"),
        }
    V, T = view.n_vertices, view.n_triangles
    return {
        "xy": dev(view.xy, (V, 2), "<f8"),
        "tri": dev(view.tri, (T, 3), "<i4"),
        "label": dev(view.label, (T,), "<i2"),
        "code": dev(view.code, (T,), "<i2"),
    }


def view_numpy(view: sbmt_mesh_view) -> dict:
    """Host copies of a finished mesh."""
    t = view_tensors(view)
    out = {
        "xy": t["xy"].cpu().numpy(),
        "tri": t["tri"].cpu().numpy(),
        "label": t["label"].cpu().numpy().view(np.uint16),
        "code": t["code"].cpu().numpy().view(np.uint16),
    }
    if view.format == SBMT_COMPACT:
        out.update(cell_label=t["cell_label"].cpu().numpy().view(np.uint16),
                   cell_code=t["cell_code"].cpu().numpy().view(np.uint16),
                   patch_cell=t["patch_cell"].cpu().numpy().view(np.uint32),
                   patch_off=t["patch_off"].cpu().numpy().view(np.uint32),
                   n_triangles=view.n_triangles, n_vertices=view.n_vertices, n_patch_triangles=view.n_patch_triangles)
    out.update({
        "format": view.format,
        "n_cells": view.n_cells,
        "n_cut_cells": view.n_cut_cells,
        "n_tierG_cells": view.n_tierG_cells,
        "n_segments": view.n_segments,
        "n_events": view.n_events,
        "n_inside_vertices": view.n_inside_vertices,
        "n_lattice_vertices": view.n_lattice_vertices,
        "n_tierG_triangles": view.n_tierG_triangles,
    })
    return out


class Context:
    """Convenience owner of a context handle."""

    def __init__(self, device: int = 0, pool_bytes: int = 0, stream: int | None = None):
        self.handle = mesh_create(device, pool_bytes, stream)

    def mesh(self, img, h_num, h_den=1, **kw) -> int:
        return mesh_bitmap(self.handle, img, h_num, h_den, **kw)

    def result(self, mesh: int) -> dict:
        return view_numpy(mesh_query(self.handle, mesh, -1))

    def close(self):
        if self.handle:
            mesh_destroy(self.handle)
            self.handle = None

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()


# ---------------------------------------------------------------------------
# serving
# ---------------------------------------------------------------------------
def _scheck(rc: int):
    if rc != SBMT_OK:
        raise SbmtError(rc, load().sbmt_server_last_error().decode())


def mesh_check(img, h_num: int, h_den: int = 1) -> int:
    """SBMT_OK, or the code mesh_bitmap would return for bad arguments."""
    im, keep = _image(img)
    pr = _params(h_num, h_den)
    rc = load().mesh_check(ctypes.byref(im), ctypes.byref(pr))
    del keep
    return rc


def mesh_bound(img, h_num: int, h_den: int = 1) -> int:
    """A request's reservation before its boundary is counted (bytes)."""
    im, keep = _image(img)
    pr = _params(h_num, h_den)
    b = ctypes.c_size_t(0)
    _scheck(load().mesh_bound(ctypes.byref(im), ctypes.byref(pr), ctypes.byref(b)))
    del keep
    return b.value


def mesh_footprint(ctx: int, mesh: int) -> int:
    b = ctypes.c_size_t(0)
    _check(load().mesh_footprint(ctx, mesh, ctypes.byref(b)))
    return b.value


def server_create(device: int = 0, hbm_budget: int = 0, max_batch: int = 0, workers: int = 0,
                  oom_every: int = 0) -> int:
    srv = ctypes.c_void_p()
    cfg = sbmt_server_config(hbm_budget, max_batch, workers, oom_every)
    _scheck(load().server_create(ctypes.byref(srv), device, ctypes.byref(cfg)))
    return srv.value


def server_submit(srv: int, img, h_num: int, h_den: int = 1) -> int:
    """Queue one request; a CUDA tensor image must stay alive until the
    request is done (a numpy image is copied)."""
    im, keep = _image(img)
    pr = _params(h_num, h_den)
    rid = ctypes.c_uint64()
    _scheck(load().server_submit(srv, ctypes.byref(im), ctypes.byref(pr), ctypes.byref(rid)))
    del keep
    return rid.value


def server_wait(srv: int, rid: int, wait_ms: int = -1):
    """(view or None while pending, info dict); raises on a failed request."""
    v, info = sbmt_mesh_view(), sbmt_request_info()
    rc = load().server_wait(srv, rid, wait_ms, ctypes.byref(v), ctypes.byref(info))
    if rc in (SBMT_EPENDING, SBMT_ETIMEDOUT):
        return None, None
    d = {"status": info.status, "batch_size": info.batch_size, "queued_ms": info.queued_ms,
         "total_ms": info.total_ms}
    _scheck(rc)
    return v, d


def server_cancel(srv: int, rid: int) -> None:
    _scheck(load().server_cancel(srv, rid))


def server_release(srv: int, rid: int) -> None:
    _scheck(load().server_release(srv, rid))


def server_stats(srv: int) -> dict:
    st = sbmt_server_stats()
    _scheck(load().server_stats(srv, ctypes.byref(st)))
    return {k: getattr(st, k) for k, _ in sbmt_server_stats._fields_}


def server_destroy(srv: int) -> None:
    _scheck(load().server_destroy(srv))
