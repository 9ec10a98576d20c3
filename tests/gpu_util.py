"""Helpers for the GPU tests: run the CUDA path through the C interface and
compare its output with the CPU oracle element by element."""
from __future__ import annotations

import numpy as np

import oracle
import paper_2602_19474_gb300 as sb

_CTX = None


def ctx():
    global _CTX
    if _CTX is None:
        sb.build_library()
        _CTX = sb.mesh_create(0)
    return _CTX


def gpu_mesh(img, h_num, h_den=1, stages=False, on_device=False):
    c = ctx()
    src = img
    if on_device:
        import torch

        src = torch.from_numpy(img.astype(np.int16) if img.dtype == np.uint16 else img).cuda()
    m = sb.mesh_bitmap(c, src, h_num, h_den, keep_stages=stages)
    v = sb.mesh_query(c, m, -1)
    out = sb.view_numpy(v)
    if stages:
        out["seg"] = sb.mesh_stage(c, m, 1)
        out["ev"] = sb.mesh_stage(c, m, 2)
        out["cut"] = sb.mesh_stage(c, m, 3)
    sb.mesh_release(c, m)
    return out


def assert_same_mesh(g, o, h, W=None, stages=False):
    """Bit-exact connectivity, labels and codes in the canonical order;
    coordinates within 1e-6 h."""
    assert g["n_cells"] == o["n_cells"]
    assert g["n_cut_cells"] == o["n_cut_cells"]
    assert g["n_tierG_cells"] == o["n_tierG_cells"]
    assert g["tri"].shape == o["tri"].shape, (g["tri"].shape, o["tri"].shape)
    assert g["xy"].shape == o["xy"].shape
    bad = np.nonzero((g["tri"] != o["tri"]).any(axis=1))[0]
    assert len(bad) == 0, "first differing triangle %d: gpu %s oracle %s" % (bad[0], g["tri"][bad[0]], o["tri"][bad[0]])
    assert np.array_equal(g["label"], o["label"])
    assert np.array_equal(g["code"], o["code"])
    err = np.abs(g["xy"] - o["xy"]).max() if len(o["xy"]) else 0.0
    assert err <= 1e-6 * h, err
    if stages:
        # segments: same set (the device emits them in any order)
        og = o["seg"].copy()
        og[:, 4:6][og[:, 4:6] == 0x10000] = 0xFFFF
        a = np.unique(og[:, :7], axis=0)
        b = np.unique(g["seg"][:, :7], axis=0)
        assert np.array_equal(a, b)
        # events: same vertex ids on the same grid edges, crossed by the same segment
        oseg = o["seg"][o["ev"][:, 1]].astype(np.int64)
        corner = oseg[:, 1] * (W + 1) + oseg[:, 0]
        exp = np.stack([o["ev"][:, 0], o["ev"][:, 2], corner, oseg[:, 2]], axis=1)
        assert np.array_equal(exp, g["ev"])
        # cut cells: id, code, triangles, inside vertices, outside-regime flag
        assert np.array_equal(g["cut"], o["cut"])


def assert_window_matches_crop(img, g, hn, hd, x0, y0, w, hh):
    """Full-size parity on a window: mesh the crop [x0, x0+w) x [y0, y0+hh)
    with the oracle on the same lattice (grid origin moved by the crop
    offset) and require that every triangle lying inside the crop's interior
    window (2h + 2 px from its border, where the crop border cannot reach)
    is in both meshes with the same vertices in the same order, label and
    code."""
    from scipy.spatial import cKDTree

    h = hn / hd
    crop = np.ascontiguousarray(img[y0:y0 + hh, x0:x0 + w])
    o = oracle.mesh_bitmap(crop, hn, hd, origin2x=-2 * x0, origin2y=-2 * y0)
    oxy = o["xy"] + np.array([x0, y0], dtype=np.float64)
    m = 2 * h + 2
    lo = np.array([x0 - 0.5 + m, y0 - 0.5 + m])
    hi = np.array([x0 + w - 0.5 - m, y0 + hh - 0.5 - m])

    def select(xy, tri):
        P = xy[tri]
        return np.all((P >= lo) & (P <= hi), axis=(1, 2))

    gs = select(g["xy"], g["tri"])
    os_ = select(oxy, o["tri"])
    assert gs.sum() == os_.sum() and gs.sum() > 0, (gs.sum(), os_.sum())
    tree = cKDTree(oxy)
    d, idx = tree.query(g["xy"][g["tri"][gs]].reshape(-1, 2))
    assert d.max() <= 1e-6 * h, d.max()
    gt = idx.reshape(-1, 3).astype(np.int64)
    a = np.concatenate([gt, g["label"][gs, None].astype(np.int64), g["code"][gs, None].astype(np.int64)], axis=1)
    b = np.concatenate([o["tri"][os_].astype(np.int64), o["label"][os_, None].astype(np.int64),
                        o["code"][os_, None].astype(np.int64)], axis=1)
    a = a[np.lexsort(a.T[::-1])]
    b = b[np.lexsort(b.T[::-1])]
    bad = np.nonzero((a != b).any(axis=1))[0]
    assert len(bad) == 0, "window (%d,%d): first mismatch gpu %s oracle %s" % (x0, y0, a[bad[0]], b[bad[0]])
    return int(gs.sum())


def exact_area_checks(img, g, h):
    """Properties that hold at any size: every triangle CCW, total area equal
    to the cells' area, per-label area equal to the pixel count."""
    import math

    from mesh_checks import signed_areas

    area = signed_areas(g["xy"], g["tri"])
    assert (area > 0).all()
    total = g["n_cells"] * math.sqrt(3) / 4 * h * h
    assert abs(area.sum() - total) <= 1e-9 * total
    per = np.bincount(g["label"].astype(np.int64), weights=area, minlength=65536)
    cnt = np.bincount(img.ravel().astype(np.int64), minlength=65536)
    lab = np.nonzero(cnt)[0]
    assert np.allclose(per[lab], cnt[lab], rtol=0, atol=1e-9 * img.size + 1e-6)
